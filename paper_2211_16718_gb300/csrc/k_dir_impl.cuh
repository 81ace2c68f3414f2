// Fused per-direction pass of the right-hand side (arXiv 2211.16718, Sec. 2.2):
// for every grid line along direction D, component-wise WENO5 reconstruction of
// u and f_D (left- and right-biased, Jiang-Shu weights), Roe flux with Harten's
// entropy fix at every interface, conservative difference of the interface
// fluxes, 4th-order central divergence of the viscous flux along D, and the
// accumulation / Runge-Kutta stage epilogue.
//
// One CTA owns a tile of TP points along D times W lines (periodic halo of 3
// points each side, fetched with wrapped indices).  Everything is staged in
// shared memory and computed in five phases separated by barriers:
//   A  load state, primitives, viscous flux; point fluxes f_D        [NP x W]
//   B  smoothness indicators of every 3-point window for the 9
//      reconstructed scalars (u_0..u_4, f_1..f_4)                      [9 x NW x W]
//   C  left/right WENO5 reconstructions of the 9 scalars at every
//      interface (MODE 1: as their double-float sum and jump)          [9 x NI x W]
//   D  Roe flux at every interface                                     [NI x W]
//   E  flux difference + viscous divergence + epilogue, global writes  [TP x W]
// The mass flux f_0 = (rho u_D) is the momentum component u_{1+D} itself, so its
// reconstructions are those of u_{1+D}.
//
// With b_k = 4(eps + beta_k) and B_k = b_k^2, the weights are
// omega_k = (c_k/B_k) / sum_j (c_j/B_j) = c_k prod_{m!=k} B_m / sum_j c_j prod_{m!=j} B_m.
// The three squared indicators of a window serve the left-biased reconstruction
// at one interface and the right-biased one at another, so each is computed once.
//
// MODE 0 (all FP64): fhat = sum_k omega_k F_k with one FP64 division.
// MODE 1 (FP64 values, double-float weights): since sum omega = 1,
//   fhat = F_2 + omega_1 (F_1 - F_2) + omega_3 (F_3 - F_2),
// where F_1 - F_2 and F_3 - F_2 are third differences of the data (FP64, from the
// window second differences s) and the weights, which only multiply these small
// differences, are evaluated in double-float arithmetic (~48 bits) on the FP32
// pipe.  The reconstructed values themselves are never formed: the Roe flux needs
// fhat_L + fhat_R = P_i + P_{i+1} + (dL + dR) and the jump fhat_R - fhat_L =
// (P_{i+1} - P_i) + dR - dL, both kept in double-float, so the FP64 pipe sees
// only the first differences, the point sums and one combination per flux
// component.  The result agrees with the all-FP64 evaluation to rounding.
// Phases A2, B and C of MODE 1 take two lines of the tile per item and run their
// double-float arithmetic on both at once with the packed FP32 instructions
// (df2.cuh): each lane computes what a one-line evaluation would, with half the
// issued instructions.
#include <math.h>

#include <type_traits>

#pragma once

#include "df.cuh"
#include "df2.cuh"
#include "k_dir_common.cuh"
#include "k_point_impl.cuh"
#include "ns3d_internal.cuh"

namespace ns3d {

constexpr int NQ = 9;             // reconstructed scalars

// Tile plan of a direction pass: TP points along the pencil times W lines.
// Shared memory in 8-byte words (doubles, or double-float pairs in MODE 1):
//   MODE 0: Q [NQ][NP*W] point values, ROE [5][NP*W] sqrt(rho), u, v, w, H,
//           FV [4][NP*W] viscous flux, B [NQ][3][NW*W] squared indicators,
//           R [18][NI*W] interface values, later [5][NI*W] interface fluxes.
//   MODE 1: Q [NQ][NP*W], dead after phase A2: ROE [5][NP*W] and FV [4][NP*W] then
//           arrive there by cp.async (as FP64) while phases B and C run;
//           B [NQ][3][NW*W/2] squared indicators, dead after phase C: the epilogue
//           operands then arrive there; S [NQ][NW*W/2] third differences;
//           G [NQ][NG*W/2] first differences (B, S, G: double-float values of the two
//           lines of a line pair side by side, 16 bytes (hi0, hi1, lo0, lo1), indexed
//           like the lines with W/2 line pairs); R [10][NI*W]: jumps du of u_0..u_4
//           (double-float, slots 0-4) and the sums of the five flux scalars
//           (FP64, slots 5-9), later [5][NI*W] interface fluxes.
//   The MODE 1 plan of a 24 x 4 tile is 57.2 KB, so that four CTAs of 256 threads
//   (64 registers) share an SM.  MODE 1 tiles have an even number of lines.
template <int MODE, int TP_, int W_>
struct Plan {
  static constexpr int TP = TP_;                    // points per tile along the pencil
  static constexpr int W = W_;                      // lines per tile
  static constexpr int THREADS = (MODE == 0) ? 128 : 256;  // MODE 1: 8 warps share the tile (latency hiding)
  static constexpr int MIN_CTAS = (MODE == 0) ? 3 : 4;     // resident CTAs per SM the registers allow
  static constexpr int NP = TP + 6;                 // points incl. 3-point halo each side
  static constexpr int NW = TP + 4;                 // 3-point windows centred at -2 .. TP+1
  static constexpr int NI = TP + 1;                 // interfaces -1/2 .. TP-1/2
  static constexpr int NG = NP - 1;                 // first differences
  static constexpr int OFF_Q = 0;
  static constexpr int OFF_ROE = (MODE == 1) ? OFF_Q : OFF_Q + NQ * NP * W;
  static constexpr int OFF_FV = OFF_ROE + 5 * NP * W;
  static constexpr int OFF_B = (MODE == 1) ? OFF_Q + NQ * NP * W : OFF_FV + 4 * NP * W;
  static constexpr int OFF_S = OFF_B + NQ * 3 * NW * W;  // MODE 1: third differences
  static constexpr int OFF_G = OFF_S + (MODE == 1 ? NQ * NW * W : 0);
  static constexpr int OFF_R = OFF_G + (MODE == 1 ? NQ * NG * W : 0);
  static constexpr int R_SLOTS = (MODE == 1) ? 10 : 18;
  static constexpr int WORDS = OFF_R + R_SLOTS * NI * W;
  static constexpr int BYTES = WORDS * 8;
  static_assert(MODE == 0 || OFF_FV + 4 * NP * W <= OFF_B, "ROE and FV fit the dead point values");
};

// Index of conserved component c among the reconstructed scalars.  MODE 0 keeps
// the order u_0..u_4, f_1..f_4.  MODE 1 stores the normal momentum u_{1+D} fifth,
// (u_0, u_{1+T1}, u_{1+T2}, u_4, u_{1+D}, f_1..f_4), so that scalars 0-4 are the
// conserved variables and scalars 4-8 the five flux components (f_0 = u_{1+D}).
template <int MODE, int D>
__host__ __device__ constexpr int scalar_of(int c) {
  if (MODE == 0 || c == 0) return c;
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  return (c == 1 + D) ? 4 : (c == 1 + T1) ? 1 : (c == 1 + T2) ? 2 : 3;
}

__device__ __forceinline__ double weno_combine(double B1, double B2, double B3, double F1, double F2, double F3) {
  const double p23 = B2 * B3;
  const double t13 = 6.0 * (B1 * B3);
  const double t12 = 3.0 * (B1 * B2);
  const double num = fma(p23, F1, fma(t13, F2, t12 * F3));
  const double den = p23 + t13 + t12;
  return num / den;
}

// Range of the squared indicators inside which df2_offset needs no rescaling: products of
// two stay below 2^80, so that they times a third difference (below 2^12 for such tiles,
// since |third difference| <= 4 |first differences| <= 4 B^(1/4)) and the denominator times
// the candidate difference stay inside the float range; and above 2^-100, so that their
// TwoProd error terms stay normal floats and the products keep full precision.
constexpr float DFW_LO = 0x1p-50f, DFW_HI = 0x1p40f;

// Offset of one reconstruction from its candidate-2 value, in double-float, from the three
// squared scaled indicators B_k (candidate order 1, 2, 3) and three differences:
//   d = e/6 + omega_1/3 * ta + omega_3/6 * tb,   omega_k = c_k prod_{m!=k} B_m / den,
// over the common denominator 6 den = 6 (B2 B3 + 6 B1 B3 + 3 B1 B2):
//   d = [den * e + 2 B2 B3 * ta + 3 B1 B2 * tb] / (6 den)        (one division).
// Left-biased: e = 2 g2 + g1, ta = s0 - s1, tb = s1 - s2; right-biased (mirrored):
// e = -(2 g2 + g3), ta = s3 - s2, tb = -(s1 - s2).
// SCALE: rescale the B_k by a common power of two first (the weights are scale-free);
// without it every B_k must lie in [DFW_LO, DFW_HI).
// Evaluated for two lines at once (two-lane double-float; each lane exactly as the
// one-lane evaluation, its scale chosen from its own B_k).
template <bool SCALE = true>
__device__ __forceinline__ df2 df2_offset(df2 B1, df2 B2, df2 B3, df2 e, df2 ta, df2 tb) {
  if (SCALE) {
    const int E0 = max(exponent_of(B1.hi.x), max(exponent_of(B2.hi.x), exponent_of(B3.hi.x)));
    const int E1 = max(exponent_of(B1.hi.y), max(exponent_of(B2.hi.y), exponent_of(B3.hi.y)));
    const float2 sc = make_float2(pow2f(-E0), pow2f(-E1));
    B1 = df2_scale(B1, sc);
    B2 = df2_scale(B2, sc);
    B3 = df2_scale(B3, sc);
  }
  const df2 p23 = df2_mul_u(B2, B3);
  const df2 p13 = df2_mul_u(B1, B3);
  const df2 p12 = df2_mul_u(B1, B2);
  const df2 den = df2_add_pos_u(p23, df2_add_pos_u(df2_mul_f_u(p13, 6.0f), df2_mul_f_u(p12, 3.0f)));
  const df2 num = df2_add_fast(df2_mul_u(den, e),
                               df2_add_fast(df2_twice(df2_mul_u(p23, ta)), df2_mul_f_u(df2_mul_u(p12, tb), 3.0f)));
  return df2_div(num, df2_mul_f_u(den, 6.0f));
}

// One tile (tx, ty, tz) of the direction-D pass, executed by the whole CTA on the
// shared memory sm (PL::BYTES).  Used by the standalone kernels (one tile per CTA),
// the batched kernels and the persistent ensemble kernel (many tiles per CTA,
// with a barrier between tiles).  NC selects read-only-cache loads, valid only when
// the inputs are not written during the kernel (false in the persistent kernel).
template <int D, int MODE, int TP_, int W_, bool NC = true>
__device__ __forceinline__ void dir_tile(const DirArgs& a, double* sm, int tx, int ty, int tz) {
  using PL = Plan<MODE, TP_, W_>;
  constexpr int TP = PL::TP, NP = PL::NP, NW = PL::NW, NI = PL::NI, W = PL::W;
  constexpr int W2 = (W + 1) / 2;  // line pairs (MODE 1)
  static_assert(MODE == 0 || W % 2 == 0, "MODE 1 tiles pair their lines");
  const int nD = a.g.n[D];
  constexpr int AX = (D == 0) ? 1 : 0;   // axis of the W lines
  constexpr int BX = (D == 2) ? 1 : 2;   // axis of blockIdx.z
  const int na = a.g.n[AX];
  const int nx = a.g.n[0], ny = a.g.n[1];
  const long long N = a.g.N;
  const int s0 = tx * TP;
  const int a0 = ty * W;
  const int bz = tz;
  const int tid = threadIdx.x;

  auto flat = [&](int c, int la) -> long long {
    int idx[3];
    idx[D] = c;
    idx[AX] = la;
    idx[BX] = bz;
    return ((long long)idx[2] * ny + idx[1]) * nx + idx[0];
  };

  // ---- A: load --------------------------------------------------------------
  for (int item = tid; item < NP * W; item += PL::THREADS) {
    int pos, line;
    tile_split<D, W>(item, NP, pos, line);
    const int c = wrap_idx(s0 - 3 + pos, nD);
    const int la = min(a0 + line, na - 1);
    const long long p = flat(c, la);
    double U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = ldx<NC>(a.u + v * N + p);
    const double vx = ldx<NC>(a.pm + PM_U * N + p), vy = ldx<NC>(a.pm + PM_V * N + p), vz = ldx<NC>(a.pm + PM_W * N + p);
    const double pr = ldx<NC>(a.pm + PM_P * N + p);
    const double un = (D == 0) ? vx : (D == 1) ? vy : vz;
    const int s = tile_idx<D, W>(pos, line, NP);
    double* q = sm + PL::OFF_Q;
#pragma unroll
    for (int v = 0; v < 5; ++v) q[scalar_of<MODE, D>(v) * NP * W + s] = U[v];
    q[5 * NP * W + s] = (D == 0) ? fma(U[1], un, pr) : U[1] * un;
    q[6 * NP * W + s] = (D == 1) ? fma(U[2], un, pr) : U[2] * un;
    q[7 * NP * W + s] = (D == 2) ? fma(U[3], un, pr) : U[3] * un;
    q[8 * NP * W + s] = (U[4] + pr) * un;
    if (MODE == 0) {  // MODE 1 fetches these after phase A2 (cp.async into the dead point values)
      double* r = sm + PL::OFF_ROE;
      r[0 * NP * W + s] = ldx<NC>(a.pm + PM_SR * N + p);
      r[1 * NP * W + s] = vx;
      r[2 * NP * W + s] = vy;
      r[3 * NP * W + s] = vz;
      r[4 * NP * W + s] = ldx<NC>(a.pm + PM_H * N + p);
      if (a.fv != nullptr) {
        double* f = sm + PL::OFF_FV;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) f[cc * NP * W + s] = ldx<NC>(a.fv + (long long)(a.fv_dstride * D + cc) * N + p);
      }
    }
  }
  __syncthreads();

  // ---- A2 (MODE 1): first differences g_j = q_{j+1} - q_j in FP64, kept as double-float,
  //      and the point values q_j of the five flux scalars copied to interface j - 2
  constexpr int PF0 = (MODE == 1) ? PL::THREADS - NP * W : 0;  // first prefetching thread (MODE 1)
  static_assert(MODE == 0 || NP * W <= PL::THREADS, "one prefetched point per thread");
  if constexpr (MODE == 1) {
    constexpr int NG = PL::NG;
    const double* q = sm + PL::OFF_Q;
    float4* G = reinterpret_cast<float4*>(sm + PL::OFF_G);
    double* R = sm + PL::OFF_R;
    // one item per line pair (lines 2 lp, 2 lp + 1), stored as (hi0, hi1, lo0, lo1)
    for (int item = tid; item < NQ * NG * W2; item += PL::THREADS) {
      const int m = item / (NG * W2);
      int j, lp;
      tile_split<D, W2>(item - m * NG * W2, NG, j, lp);
      const double* qm = q + m * NP * W;
      const int l0 = 2 * lp, l1 = l0 + 1;
      const double qa0 = qm[tile_idx<D, W>(j, l0, NP)], qb0 = qm[tile_idx<D, W>(j + 1, l0, NP)];
      const double qa1 = qm[tile_idx<D, W>(j, l1, NP)], qb1 = qm[tile_idx<D, W>(j + 1, l1, NP)];
      const df g0 = d2df_bits(qb0 - qa0), g1 = d2df_bits(qb1 - qa1);
      G[m * NG * W2 + tile_idx<D, W2>(j, lp, NG)] = make_float4(g0.hi, g1.hi, g0.lo, g1.lo);
      if (m >= 4 && j >= 2 && j < NI + 2) {
        R[(1 + m) * NI * W + tile_idx<D, W>(j - 2, l0, NI)] = qa0;
        R[(1 + m) * NI * W + tile_idx<D, W>(j - 2, l1, NI)] = qa1;
      }
    }
    __syncthreads();
    // the point values are dead: fetch the Roe-average inputs and the viscous flux into
    // their space while phases B and C run.  One point per thread, on the last NP*W
    // threads (those with the fewest phase-C items), which also convert their Roe
    // inputs to double-float in place before the barrier that ends phase C.
    if (tid >= PF0) {
      int pos, line;
      tile_split<D, W>(tid - PF0, NP, pos, line);
      const long long p = flat(wrap_idx(s0 - 3 + pos, nD), min(a0 + line, na - 1));
      const int sp = tile_idx<D, W>(pos, line, NP);
      double* r = sm + PL::OFF_ROE + sp;
      cp_async8(r + 0 * NP * W, a.pm + PM_SR * N + p);
      cp_async8(r + 1 * NP * W, a.pm + PM_U * N + p);
      cp_async8(r + 2 * NP * W, a.pm + PM_V * N + p);
      cp_async8(r + 3 * NP * W, a.pm + PM_W * N + p);
      cp_async8(r + 4 * NP * W, a.pm + PM_H * N + p);
      if (a.fv != nullptr) {
        double* f = sm + PL::OFF_FV + sp;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) cp_async8(f + cc * NP * W, a.fv + (long long)(a.fv_dstride * D + cc) * N + p);
      }
    }
    cp_async_commit();
  }

  // ---- B: squared scaled smoothness indicators of every window ----------------
  int need_scale = 0;
  if constexpr (MODE == 0) {
    const double* q = sm + PL::OFF_Q;
    for (int item = tid; item < NQ * NW * W; item += PL::THREADS) {
      const int m = item / (NW * W);
      int w, line;
      tile_split<D, W>(item - m * NW * W, NW, w, line);
      const int o = tile_idx<D, W>(w, line, NW);
      const double* qm = q + m * NP * W;
      const double x = qm[tile_idx<D, W>(w, line, NP)];
      const double y = qm[tile_idx<D, W>(w + 1, line, NP)];
      const double z = qm[tile_idx<D, W>(w + 2, line, NP)];
      const double gm = y - x, gp = z - y, s = gp - gm;
      double* bw = sm + PL::OFF_B;
      const double aa = fma((13.0 / 3.0) * s, s, a.eps4);
      const double u1 = fma(3.0, gp, -gm);   // x - 4y + 3z
      const double u2 = gm + gp;             // z - x
      const double u3 = fma(-3.0, gm, gp);   // 3x - 4y + z
      const double b1 = fma(u1, u1, aa), b2 = fma(u2, u2, aa), b3 = fma(u3, u3, aa);
      bw[(m * 3 + 0) * NW * W + o] = b1 * b1;
      bw[(m * 3 + 1) * NW * W + o] = b2 * b2;
      bw[(m * 3 + 2) * NW * W + o] = b3 * b3;
    }
  } else {
    // one item per line pair: two-lane double-float arithmetic (packed FP32 instructions)
    int range_bad = 0;
    float4* bw = reinterpret_cast<float4*>(sm + PL::OFF_B);
    float4* S = reinterpret_cast<float4*>(sm + PL::OFF_S);
    const df2 c133 = df2_splat(df{a.c133_hi, a.c133_lo});
    const df2 eps4 = df2_splat(df{a.eps4_hi, a.eps4_lo});
    for (int item = tid; item < NQ * NW * W2; item += PL::THREADS) {
      const int m = item / (NW * W2);
      int w, lp;
      tile_split<D, W2>(item - m * NW * W2, NW, w, lp);
      const int o = tile_idx<D, W2>(w, lp, NW);
      const float4* G = reinterpret_cast<const float4*>(sm + PL::OFF_G) + m * PL::NG * W2;
      const df2 dgm = df2_from4(G[tile_idx<D, W2>(w, lp, PL::NG)]);
      const df2 dgp = df2_from4(G[tile_idx<D, W2>(w + 1, lp, PL::NG)]);
      const df2 ds = df2_add_fast(dgp, df2_neg(dgm));  // second difference s_w
      // third difference T_w = s_w - s_{w+1} (phase C needs T_f, T_{f+1}, T_{f+2}; the last
      // window has no s_{w+1} in the tile and its T is never read)
      df2 T{f2splat(0.0f), f2splat(0.0f)};
      if (w + 2 < PL::NG) {
        const df2 g2 = df2_from4(G[tile_idx<D, W2>(w + 2, lp, PL::NG)]);
        T = df2_add_fast(ds, df2_neg(df2_add_fast(g2, df2_neg(dgp))));
      }
      S[m * NW * W2 + o] = df2_to4(T);
      // scaled indicators b_k = u_k^2 + aa, aa = (13/3) s^2 + 4 eps, with u_2 = z - x and
      // u_1 = x - 4y + 3z = u_2 + 2s, u_3 = 3x - 4y + z = 2s - u_2:
      //   b_2 = u_2^2 + aa,  b_{1,3} = (b_2 + 4 s^2) +- 4 u_2 s   (b_k >= aa >= (13/3) s^2, so
      // b_2 + 4 s^2 <= ~3 b_{1,3}: no harmful cancellation)
      const df2 s2 = df2_sqr_u(ds);
      const df2 aa = df2_add_pos_u(df2_mul_u(s2, c133), eps4);
      const df2 u2 = df2_add_fast(dgm, dgp);
      const df2 b2 = df2_add_pos_u(df2_sqr_u(u2), aa);
      // Fast2Sum order with margins: b_2 >= aa >= (13/12) 4 s^2, and
      // pq = u_2^2 + (4 + 13/3) s^2 + 4 eps >= 1.44 |4 u_2 s| (minimum over u_2)
      const df2 pq = df2_add_ordered_u(b2, df2_twice(df2_twice(s2)));
      const df2 r4 = df2_twice(df2_twice(df2_mul_u(u2, ds)));
      const df2 B1 = df2_sqr_u(df2_add_ordered(pq, r4));
      const df2 B2 = df2_sqr_u(b2);
      const df2 B3 = df2_sqr_u(df2_add_ordered(pq, df2_neg(r4)));
      bw[(m * 3 + 0) * NW * W2 + o] = df2_to4(B1);
      bw[(m * 3 + 1) * NW * W2 + o] = df2_to4(B2);
      bw[(m * 3 + 2) * NW * W2 + o] = df2_to4(B3);
      // the float exponent range bounds the indicators (differences of the data
      // up to ~1e9); beyond it the host reports NS3D_ERANGE instead of a NaN
      const float bmax0 = fmaxf(B1.hi.x, fmaxf(B2.hi.x, B3.hi.x));
      const float bmax1 = fmaxf(B1.hi.y, fmaxf(B2.hi.y, B3.hi.y));
      const float bmin0 = fminf(B1.hi.x, fminf(B2.hi.x, B3.hi.x));
      const float bmin1 = fminf(B1.hi.y, fminf(B2.hi.y, B3.hi.y));
      range_bad |= !(bmax0 < 1e36f) || !(bmax1 < 1e36f);
      need_scale |= !(bmax0 < DFW_HI && bmin0 >= DFW_LO && bmax1 < DFW_HI && bmin1 >= DFW_LO);
    }
    if (__any_sync(0xffffffffu, range_bad) && (tid & 31) == 0) atomicOr(a.status, ST_DF_RANGE);
  }
  // one CTA-wide decision: rescaled weights only for tiles with extreme indicators
  const bool tile_scale = __syncthreads_or(need_scale) != 0;

  // ---- C: left/right WENO5 reconstructions at every interface -------------------
  if constexpr (MODE == 0) {
    const double* q = sm + PL::OFF_Q;
    double* rec = sm + PL::OFF_R;
    for (int item = tid; item < NQ * NI * W; item += PL::THREADS) {
      const int m = item / (NI * W);
      int f, line;
      tile_split<D, W>(item - m * NI * W, NI, f, line);
      const double* qm = q + m * NP * W;
      const double P0 = qm[tile_idx<D, W>(f, line, NP)], P1 = qm[tile_idx<D, W>(f + 1, line, NP)];
      const double P2 = qm[tile_idx<D, W>(f + 2, line, NP)], P3 = qm[tile_idx<D, W>(f + 3, line, NP)];
      const double P4 = qm[tile_idx<D, W>(f + 4, line, NP)], P5 = qm[tile_idx<D, W>(f + 5, line, NP)];
      // third-order candidates at the interface between P2 and P3
      const double xR = fma(11.0 / 6.0, P2, fma(-7.0 / 6.0, P1, (1.0 / 3.0) * P0));
      const double eR = fma(1.0 / 3.0, P3, fma(5.0 / 6.0, P2, (-1.0 / 6.0) * P1));
      const double eL = fma(-1.0 / 6.0, P4, fma(5.0 / 6.0, P3, (1.0 / 3.0) * P2));
      const double xL = fma(1.0 / 3.0, P5, fma(-7.0 / 6.0, P4, (11.0 / 6.0) * P3));
      const double* b = sm + PL::OFF_B + m * 3 * NW * W;
      const double B1f = b[0 * NW * W + tile_idx<D, W>(f, line, NW)];
      const double B2f1 = b[1 * NW * W + tile_idx<D, W>(f + 1, line, NW)];
      const double B3f2 = b[2 * NW * W + tile_idx<D, W>(f + 2, line, NW)];
      const double B3f3 = b[2 * NW * W + tile_idx<D, W>(f + 3, line, NW)];
      const double B2f2 = b[1 * NW * W + tile_idx<D, W>(f + 2, line, NW)];
      const double B1f1 = b[0 * NW * W + tile_idx<D, W>(f + 1, line, NW)];
      const int o = tile_idx<D, W>(f, line, NI);
      rec[(2 * m) * NI * W + o] = weno_combine(B1f, B2f1, B3f2, xR, eR, eL);
      rec[(2 * m + 1) * NI * W + o] = weno_combine(B3f3, B2f2, B1f1, xL, eL, eR);
    }
  } else {
    // fhat_L = P2 + dL, fhat_R = P3 + dR with the offsets (differences only)
    //   dL =  (2 g2 + g1)/6 + w1 (s0 - s1) + w3 (s1 - s2)      [w1 = omega_1/3, w3 = omega_3/6]
    //   dR = -(2 g2 + g3)/6 + v1 (s3 - s2) - v3 (s1 - s2)
    // (candidate 2 minus the point value, and F1 - F2, F3 - F2 as third differences),
    // evaluated in double-float on the FP32 pipe.  The interface values are never
    // formed in FP64: the Roe flux needs only
    //   du    = g2 + dR - dL       (fhat_R - fhat_L, for the u-scalars; double-float)
    //   fhat_L + fhat_R = 2 P2 + (g2 + dL + dR)   (for the flux scalars; FP64)
    // One item per line pair, in two-lane double-float arithmetic.
    float2* rf = reinterpret_cast<float2*>(sm + PL::OFF_R);
    auto phase_c = [&](auto scaled) {
      constexpr bool SCALE = decltype(scaled)::value;
      for (int item = tid; item < NQ * NI * W2; item += PL::THREADS) {
        const int m = item / (NI * W2);
        int f, lp;
        tile_split<D, W2>(item - m * NI * W2, NI, f, lp);
        const float4* S = reinterpret_cast<const float4*>(sm + PL::OFF_S) + m * NW * W2;
        const float4* G = reinterpret_cast<const float4*>(sm + PL::OFF_G) + m * PL::NG * W2;
        const float4* b = reinterpret_cast<const float4*>(sm + PL::OFF_B) + m * 3 * NW * W2;
        auto ldS = [&](int w) { return df2_from4(S[tile_idx<D, W2>(w, lp, NW)]); };
        auto ldG = [&](int j) { return df2_from4(G[tile_idx<D, W2>(j, lp, PL::NG)]); };
        auto ld = [&](int k, int w) { return df2_from4(b[k * NW * W2 + tile_idx<D, W2>(w, lp, NW)]); };
        // third differences (phase B): s0 - s1 = T_f, s1 - s2 = T_{f+1}, s3 - s2 = -T_{f+2}
        const df2 t0 = ldS(f), tC = ldS(f + 1), t2 = df2_neg(ldS(f + 2));
        const df2 g1 = ldG(f + 1), g2 = ldG(f + 2), g3 = ldG(f + 3);
        const df2 g22 = df2_twice(g2);
        const df2 dL = df2_offset<SCALE>(ld(0, f), ld(1, f + 1), ld(2, f + 2), df2_add_fast(g22, g1), t0, tC);
        const df2 dR = df2_offset<SCALE>(ld(2, f + 3), ld(1, f + 2), ld(0, f + 1), df2_neg(df2_add_fast(g22, g3)), t2,
                                         df2_neg(tC));
        const int o0 = tile_idx<D, W>(f, 2 * lp, NI), o1 = tile_idx<D, W>(f, 2 * lp + 1, NI);
        if (m < 5) {
          const df2 du = df2_add_fast(g2, df2_add_fast(dR, df2_neg(dL)));
          rf[m * NI * W + o0] = make_float2(du.hi.x, du.lo.x);
          rf[m * NI * W + o1] = make_float2(du.hi.y, du.lo.y);
        }
        if (m >= 4) {  // flux scalar: fhat_L + fhat_R = 2 P2 + (g2 + dL + dR), P2 copied in phase A2
          const df2 t = df2_add_fast(g2, df2_add_fast(dL, dR));
          double* F = sm + PL::OFF_R + (1 + m) * NI * W;
          F[o0] = fma(2.0, F[o0], f2d_bits(t.hi.x)) + f2d_bits(t.lo.x);
          F[o1] = fma(2.0, F[o1], f2d_bits(t.hi.y)) + f2d_bits(t.lo.y);
        }
      }
    };
    if (tile_scale)
      phase_c(std::true_type{});
    else
      phase_c(std::false_type{});
    cp_async_wait_all();  // this thread's ROE / FV copies; the barrier publishes them
    if (tid >= PF0) {  // velocities to double-float, in place (sqrt(rho) and H arrive as
                       // double-float: planes of the NS3D_FP64 primitive layout)
      int pos, line;
      tile_split<D, W>(tid - PF0, NP, pos, line);
      double* r = sm + PL::OFF_ROE + tile_idx<D, W>(pos, line, NP);
#pragma unroll
      for (int k = 1; k < 4; ++k) {
        const df x = d2df_bits(r[k * NP * W]);
        reinterpret_cast<float2*>(r)[k * NP * W] = make_float2(x.hi, x.lo);
      }
    }
  }
  __syncthreads();

  // ---- epilogue operands: fetched asynchronously into the (now unused) indicator
  //      space while phase D runs; each thread later reads only its own point's slots.
  //      cp.async.ca reads through L1 like a plain load, so in the persistent kernel (NC
  //      false), where the operands were written by other CTAs before the last grid-wide
  //      barrier, it sees them exactly as the plain loads it replaces would.
  static_assert(PL::TP * PL::W <= PL::THREADS, "one epilogue point per thread");
  static_assert(15 * PL::TP * PL::W <= NQ * 3 * PL::NW * PL::W, "prefetch slots fit the indicator space");
  double* pre = sm + PL::OFF_B + 15 * tid;
  if (tid < TP * W) {
    int pp, line;
    tile_split<D, W>(tid, TP, pp, line);
    if (s0 + pp < nD && a0 + line < na) epilogue_prefetch(a, flat(s0 + pp, a0 + line), pre);
  }
  cp_async_commit();

  // ---- D: Roe flux at every interface -------------------------------------------
  {
    const double gm1 = a.gamma - 1.0;
    const double* r = sm + PL::OFF_ROE;
    double* rec = sm + PL::OFF_R;
    int bad = 0, range_bad = 0;
    for (int item = tid; item < NI * W; item += PL::THREADS) {
      int f, line;
      tile_split<D, W>(item, NI, f, line);
      const int o = tile_idx<D, W>(f, line, NI);
      const int sa = tile_idx<D, W>(f + 2, line, NP), sb = tile_idx<D, W>(f + 3, line, NP);
      if (MODE == 1) {
        // Roe dissipation X|Lambda|X^{-1} du in double-float from the double-float jumps
        // du of phase C and the double-float Roe-average inputs; the flux, already divided
        // by dx for phase E, is (fhat_L + fhat_R)/(2 dx) - diss/(2 dx): two FP64 operations
        // per component
        const float2* rf = reinterpret_cast<const float2*>(r);
        auto ldr = [&](int k, int sp) { const float2 v = rf[k * NP * W + sp]; return df{v.x, v.y}; };
        const float2* rj = reinterpret_cast<const float2*>(rec);
        df du[5];
        double fs[5];  // fhat_L + fhat_R of the five flux components (f_0 = u_{1+D})
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const float2 j = rj[scalar_of<MODE, D>(v) * NI * W + o];
          du[v] = df{j.x, j.y};
          fs[v] = rec[(5 + v) * NI * W + o];
        }
        const df ra = ldr(0, sa), rb = ldr(0, sb);
        const df rsum = df_add_pos(ra, rb);
        const df rs = df_div(df{1.0f, 0.0f}, rsum);
        const df wa = df_mul_u(ra, rs), wb = df_mul_u(rb, rs);
        df V[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) V[m] = df_add_fast(df_mul_u(wa, ldr(1 + m, sa)), df_mul_u(wb, ldr(1 + m, sb)));
        const df H = df_add_pos(df_mul_u(wa, ldr(4, sa)), df_mul_u(wb, ldr(4, sb)));
        const df q2 = df_add_pos_u(df_sqr_u(V[0]), df_add_pos_u(df_sqr_u(V[1]), df_sqr_u(V[2])));
        const df q2h = df{0.5f * q2.hi, 0.5f * q2.lo};
        const df c2 = df_mul(df_add_fast(H, df_neg(q2h)), df{a.gm1_hi, a.gm1_lo});
        bad |= !(c2.hi > 0.0f);
        range_bad |= !(c2.hi > 1e-30f && c2.hi < 1e30f && rsum.hi > 1e-30f && rsum.hi < 1e30f);
        const df c = df_sqrt(c2);
        const df rc = df_div(df{1.0f, 0.0f}, c);
        constexpr int T1 = (D == 0) ? 1 : 0;
        constexpr int T2 = (D == 2) ? 1 : 2;
        const df un = V[D], vt1 = V[T1], vt2 = V[T2];
        const df b1 = df_mul_u(df{a.gm1_hi, a.gm1_lo}, df_sqr_u(rc));
        const df vdm = df_add_fast(df_mul_u(V[0], du[1]), df_add_fast(df_mul_u(V[1], du[2]), df_mul_u(V[2], du[3])));
        const df phi = df_mul_u(b1, df_add_fast(df_add_fast(df_mul_u(q2h, du[0]), du[4]), df_neg(vdm)));
        const df a2 = df_add_fast(du[0], df_neg(phi));
        const df a3 = df_add_fast(du[1 + T1], df_neg(df_mul_u(vt1, du[0])));
        const df a4 = df_add_fast(du[1 + T2], df_neg(df_mul_u(vt2, du[0])));
        const df ach0 = df_mul_u(df_add_fast(df_mul_u(un, du[0]), df_neg(du[1 + D])), rc);
        const df ach = df{0.5f * ach0.hi, 0.5f * ach0.lo};
        const df ph = df{0.5f * phi.hi, 0.5f * phi.lo};
        const df a1 = df_add_fast(ph, ach), a5 = df_add_fast(ph, df_neg(ach));
        df l1 = df_abs(df_add_fast(un, df_neg(c))), l5 = df_abs(df_add_fast(un, c));
        const df l2 = df_abs(un);
        const df delta = df_mul(c, df{a.hd_hi, a.hd_lo});
        if (df_lt(l1, delta)) l1 = df_div(df_add_pos_u(df_sqr_u(l1), df_sqr_u(delta)), df_twice(delta));
        if (df_lt(l5, delta)) l5 = df_div(df_add_pos_u(df_sqr_u(l5), df_sqr_u(delta)), df_twice(delta));
        const df A1 = df_mul_u(l1, a1), A2 = df_mul_u(l2, a2), A3 = df_mul_u(l2, a3), A4 = df_mul_u(l2, a4);
        const df A5 = df_mul_u(l5, a5);
        const df S = df_add_fast(A1, A5);
        const df d0 = df_add_fast(S, A2);
        const df cD = df_mul_u(c, df_add_fast(A5, df_neg(A1)));
        df diss[5];
        diss[0] = d0;
        diss[1 + D] = df_add_fast(df_mul_u(d0, un), cD);
        diss[1 + T1] = df_add_fast(df_mul_u(d0, vt1), A3);
        diss[1 + T2] = df_add_fast(df_mul_u(d0, vt2), A4);
        diss[4] = df_add_fast(df_add_fast(df_mul_u(S, H), df_mul_u(cD, un)),
                              df_add_fast(df_mul_u(A2, q2h), df_add_fast(df_mul_u(A3, vt1), df_mul_u(A4, vt2))));
        const df mhr = df_neg(d2df_bits(a.g.hrh[D]));
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const df t = df_mul(diss[v], mhr);
          rec[v * NI * W + o] = fma(a.g.hrh[D], fs[v], f2d_bits(t.hi)) + f2d_bits(t.lo);
        }
        continue;
      }
      double uL[5], uR[5], fL[5], fR[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        uL[v] = rec[(2 * v) * NI * W + o];
        uR[v] = rec[(2 * v + 1) * NI * W + o];
      }
#pragma unroll
      for (int v = 1; v < 5; ++v) {
        fL[v] = rec[(2 * (4 + v)) * NI * W + o];
        fR[v] = rec[(2 * (4 + v) + 1) * NI * W + o];
      }
      fL[0] = uL[1 + D];
      fR[0] = uR[1 + D];
      const double ra = r[sa], rb = r[sb];
      const double rsum = ra + rb;
      // MODE 1: FP32-seeded Newton reciprocals (FP64 accurate, ~4 FP64 operations
      // instead of ~9 for the IEEE division); MODE 0: IEEE division and square root
      const double rs = (MODE == 1) ? rcp_newton(rsum) : 1.0 / rsum;
      const double wa = ra * rs, wb = rb * rs;
      double V[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) V[m] = fma(wa, r[(1 + m) * NP * W + sa], wb * r[(1 + m) * NP * W + sb]);
      const double H = fma(wa, r[4 * NP * W + sa], wb * r[4 * NP * W + sb]);
      const double q2h = 0.5 * fma(V[0], V[0], fma(V[1], V[1], V[2] * V[2]));
      const double c2 = gm1 * (H - q2h);
      bad |= !(c2 > 0.0);
      double c, rc;
      if (MODE == 1) {
        // the float seeds need c^2 and sqrt(rho_a) + sqrt(rho_b) inside the float range
        range_bad |= !(c2 > 1e-36 && c2 < 1e36 && rsum > 1e-36 && rsum < 1e36);
        rc = rsqrt_newton(c2);
        c = c2 * rc;
      } else {
        c = sqrt(c2);
        rc = 1.0 / c;
      }
      double du[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) du[v] = uR[v] - uL[v];
      constexpr int T1 = (D == 0) ? 1 : 0;
      constexpr int T2 = (D == 2) ? 1 : 2;
      const double un = V[D], vt1 = V[T1], vt2 = V[T2];
      const double b1 = gm1 * (rc * rc);
      const double vdm = fma(V[0], du[1], fma(V[1], du[2], V[2] * du[3]));
      const double phi = b1 * (fma(q2h, du[0], du[4]) - vdm);
      const double a2 = du[0] - phi;
      const double a3 = fma(-vt1, du[0], du[1 + T1]);
      const double a4 = fma(-vt2, du[0], du[1 + T2]);
      const double ach = 0.5 * (fma(un, du[0], -du[1 + D]) * rc);
      const double ph = 0.5 * phi;
      const double a1 = ph + ach, a5 = ph - ach;
      double l1 = fabs(un - c), l5 = fabs(un + c);
      const double l2 = fabs(un);
      const double delta = a.hdelta * c;
      if (l1 < delta) l1 = (l1 * l1 + delta * delta) / (2.0 * delta);
      if (l5 < delta) l5 = (l5 * l5 + delta * delta) / (2.0 * delta);
      const double A1 = l1 * a1, A2 = l2 * a2, A3 = l2 * a3, A4 = l2 * a4, A5 = l5 * a5;
      const double S = A1 + A5;
      const double d0 = S + A2;
      const double cD = c * (A5 - A1);
      double diss[5];
      diss[0] = d0;
      diss[1 + D] = fma(d0, un, cD);
      diss[1 + T1] = fma(d0, vt1, A3);
      diss[1 + T2] = fma(d0, vt2, A4);
      diss[4] = fma(S, H, fma(cD, un, fma(A2, q2h, fma(A3, vt1, A4 * vt2))));
#pragma unroll
      for (int v = 0; v < 5; ++v) rec[v * NI * W + o] = 0.5 * (fL[v] + fR[v] - diss[v]);
    }
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(a.status, ST_NONPHYS);
    if (MODE == 1 && __any_sync(0xffffffffu, range_bad) && (tid & 31) == 0) atomicOr(a.status, ST_DF_RANGE);
  }
  __syncthreads();

  // ---- E: conservative difference + viscous divergence + epilogue ----------------
  cp_async_wait_all();
  {
    const double rdx = a.g.rh[D];
    const double r12 = a.g.r12h[D];
    const double* F = sm + PL::OFF_R;
    const double* fvs = sm + PL::OFF_FV;
    for (int item = tid; item < TP * W; item += PL::THREADS) {
      int pp, line;
      tile_split<D, W>(item, TP, pp, line);
      if (s0 + pp >= nD || a0 + line >= na) continue;
      double cv[5];
      const int op = tile_idx<D, W>(pp + 1, line, NI), om = tile_idx<D, W>(pp, line, NI);
      if (MODE == 1) {  // interface fluxes already divided by dx; viscous fluxes double-float
#pragma unroll
        for (int v = 0; v < 5; ++v) cv[v] = F[v * NI * W + om] - F[v * NI * W + op];
        if (a.fv != nullptr) {
          const df r12d = d2df_bits(r12);
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const float2* fc = reinterpret_cast<const float2*>(fvs + cc * NP * W);
            auto ld = [&](int j) { const float2 v = fc[tile_idx<D, W>(j, line, NP)]; return df{v.x, v.y}; };
            const df t = d4_dfv(ld(pp + 1), ld(pp + 2), ld(pp + 4), ld(pp + 5), r12d);
            cv[1 + cc] = (cv[1 + cc] + f2d_bits(t.hi)) + f2d_bits(t.lo);
          }
        }
        dir_epilogue_pre(a, flat(s0 + pp, a0 + line), cv, pre);
        continue;
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) cv[v] = (F[v * NI * W + om] - F[v * NI * W + op]) * rdx;
      if (a.fv != nullptr) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const double* fc = fvs + cc * NP * W;
          const double d1 = fc[tile_idx<D, W>(pp + 4, line, NP)] - fc[tile_idx<D, W>(pp + 2, line, NP)];
          const double d2 = fc[tile_idx<D, W>(pp + 5, line, NP)] - fc[tile_idx<D, W>(pp + 1, line, NP)];
          cv[1 + cc] = fma(fma(8.0, d1, -d2), r12, cv[1 + cc]);
        }
      }
      const long long p = flat(s0 + pp, a0 + line);
      dir_epilogue_pre(a, p, cv, pre);
    }
  }
}

}  // namespace ns3d
