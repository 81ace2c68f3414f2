// FP32-bulk direction pass (precision NS3D_FP32_BULK): the fused WENO5 + Roe +
// conservative difference + viscous divergence of k_dir.cu with the primitive
// variables, point fluxes, smoothness indicators, weights, interface values, the
// Roe flux and the viscous interface flux in FP32 (arXiv 2211.16718, Sec. 2.2
// arithmetic unchanged, precision reduced).  The total interface flux is widened
// to FP64 before the conservative difference, so the sums over the grid still
// telescope exactly; the accumulation / RK stage update and the state stay FP64.
//
// Layout of one tile (TP points along the pencil x W lines, 256 threads):
//  A   load the state (FP64, converted to FP32 by bit manipulation) at the tile's
//      points and a 3-point halo, form the primitive variables and point fluxes in
//      registers (no primitive planes are read), and the viscous flux of this
//      direction (FP32 planes of the viscous kernel);
//  BC  one item = one scalar on one line over SEG consecutive interfaces: the
//      SEG + 5 point values are read once (vector loads) and slid through in
//      registers: the window indicators, the left- and right-biased WENO5 values,
//      and their jump (conserved variables) or sum (flux components);
//  D   per interface: Roe average, wave strengths with Harten's fix, the central
//      part, the viscous interface flux (-f_{i-1} + 7 f_i + 7 f_{i+1} - f_{i+2})/12,
//      divided by dx and widened to FP64;
//  E   per point: FP64 difference of its two interface fluxes, then the
//      accumulation / RK epilogue (its operands prefetched by cp.async during D; in the y
//      and z passes a thread takes two x-adjacent points and moves 16-byte pairs).
#include <math.h>

#include "df.cuh"
#include "k_dir_common.cuh"
#include "ns3d_internal.cuh"

namespace ns3d {

namespace {

constexpr int THREADS = 256;
constexpr int TP = 27, W = 8;   // 27 points: 19 tiles cover 512 (513), 38 cover 1024 (1026)
constexpr int NP = TP + 6;      // positions per line: 3-point halo on each side
constexpr int NI = TP + 1;      // interfaces per line
constexpr int SEG = 4;          // interfaces per reconstruction item
constexpr int NSEG = NI / SEG;  // 7
static_assert(NI % SEG == 0, "whole segments");
constexpr int NQ = 9;           // reconstructed scalars: 5 conserved, 4 flux components (f_0 = u_{1+D})
constexpr int NREC = 10;        // per interface: 5 jumps, the sum of u_{1+D}, 4 flux sums
constexpr int LS = 36;          // line stride (floats) of the scalar planes: >= SEG*NSEG + 5 and a multiple of 4
constexpr int L4 = NP;          // line stride (float4) of the Roe-input and viscous planes (odd: no bank conflicts)
static_assert(SEG * (NSEG - 1) + 12 <= LS && LS % 4 == 0, "segment reads (three float4) stay in the line");
// shared-memory plan (bytes)
constexpr int OFF_Q = 0;                              // float  [NQ][W][LS]
constexpr int OFF_R4 = OFF_Q + NQ * W * LS * 4;       // float4 [W][L4]: sqrt(rho), u, v, w
constexpr int OFF_H = OFF_R4 + W * L4 * 16;           // float  [W][L4]: H
constexpr int OFF_V4 = OFF_H + ((W * L4 * 4 + 15) & ~15);  // float4 [W][L4]: viscous flux of this direction
constexpr int OFF_REC = OFF_V4 + W * L4 * 16;         // float  [NREC][W][NI]
constexpr int FS = 30;          // line stride (doubles) of the interface fluxes (no bank conflicts in y, z)
constexpr int OFF_F = OFF_REC + NREC * W * NI * 4;    // double [5][W][FS]: interface flux / dx
constexpr int OFF_P2 = OFF_F + 5 * W * FS * 8;         // double [TP*W][10]: epilogue operands U_n and acc / u
constexpr int BYTES = OFF_P2 + 10 * TP * W * 8;
static_assert(FS >= NI, "interface-flux line");
// epilogue operand k (5 doubles per point) prefetched into the scalar planes, dead after BC
static_assert(5 * TP * W * 8 <= NQ * W * LS * 4, "prefetch slots fit the scalar planes");
static_assert(BYTES + 1024 <= 233472 / 4, "four CTAs per SM");
static_assert(OFF_R4 % 16 == 0 && OFF_V4 % 16 == 0 && OFF_F % 8 == 0 && OFF_REC % 16 == 0, "alignment");
static_assert(TP * W <= THREADS && NI * W <= THREADS, "one point / interface per thread in D and E");

// FP64 -> FP32 by truncating the bit pattern (integer instructions only): sign and exponent
// exact for |x| in [2^-126, 2^128); smaller magnitudes give signed zero, larger ones, infinities
// and NaNs give +-inf (a non-finite state is then reported by the checks of phase A).
__device__ __forceinline__ float d2f_tz(double x) {
  const uint32_t h = (uint32_t)__double2hiint(x), l = (uint32_t)__double2loint(x);
  const uint32_t e11 = (h >> 20) & 0x7ffu;
  uint32_t b = __funnelshift_l(l, h, 3) + 0x40000000u;  // rebased exponent, top 23 mantissa bits
  b = (e11 <= 896u) ? 0u : b;
  b = (e11 >= 1151u) ? 0x7f800000u : b;
  return __uint_as_float(b | (h & 0x80000000u));
}

__device__ __forceinline__ float rcp_a(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_a(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Weighted WENO5 value written as an offset from the candidate c with the linear weight 6/10
// (Sec. 2.2: sum_k omega_k F_k = F_2 + omega_1 (F_1 - F_2) + omega_3 (F_3 - F_2)), the candidate
// differences being third differences of the data: with omega_k ~ c_k / B_k, c = (1, 6, 3)/10
// and B_k = (4 (eps + beta_k))^2, over the common denominator,
//   value = c + (B2 B3 d1 + 3 B1 B2 d3) / (B2 B3 + 6 B1 B3 + 3 B1 B2),
// d1 = F_1 - F_2, d3 = F_3 - F_2.  Unscaled products and an approximate reciprocal: valid while
// every B and product stays in the normal FP32 range (checked by the caller).
__device__ __forceinline__ float weno_fast(float B1, float B2, float B3, float c, float d1, float d3x3) {
  const float p23 = B2 * B3, p12 = B1 * B2;
  const float den = fmaf(6.0f * B1, B3, fmaf(3.0f, p12, p23));
  const float num = fmaf(p23, d1, p12 * d3x3);
  return fmaf(num, rcp_a(den), c);
}

// The same with the indicators rescaled by their common power of two and an IEEE division: any
// data whose indicators are finite.
__device__ __forceinline__ float weno_safe(float B1, float B2, float B3, float c, float d1, float d3x3) {
  const int E = max(exponent_of(B1), max(exponent_of(B2), exponent_of(B3)));
  const float sc = pow2f(max(-E, -126));
  B1 *= sc;
  B2 *= sc;
  B3 *= sc;
  const float p23 = B2 * B3, p12 = B1 * B2;
  const float den = fmaf(6.0f * B1, B3, fmaf(3.0f, p12, p23));
  const float num = fmaf(p23, d1, p12 * d3x3);
  return c + __fdiv_rn(num, den);
}

// Accumulation / RK epilogue with its operands from the prefetch slots: kp = k, ops = U_n then
// acc or the stage input; the arithmetic of dir_epilogue.
__device__ __forceinline__ void dir_epilogue_pre32(const DirArgs& a, long long p, const double cv[5], const double* kp,
                                                   const double* ops) {
  const long long N = a.g.N;
  switch (a.epi) {
    case EPI_ACC_WRITE:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] = cv[v];
      break;
    case EPI_ACC_ADD:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] = kp[v] + cv[v];
      break;
    case EPI_RHS_OUT:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.out[v * N + p] = kp[v] + cv[v];
      break;
    case EPI_RK4_FIRST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = kp[v] + cv[v];
        a.out[v * N + p] = fma(a.a, K, ops[v]);
        a.acc[v * N + p] = K;
      }
      break;
    case EPI_RK4_MID:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = kp[v] + cv[v];
        a.out[v * N + p] = fma(a.a, K, ops[v]);
        a.acc[v * N + p] = fma(2.0, K, ops[5 + v]);
      }
      break;
    case EPI_RK4_LAST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = kp[v] + cv[v];
        a.out[v * N + p] = fma(a.a, ops[5 + v] + K, ops[v]);
      }
      break;
    case EPI_SSP_1:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = kp[v] + cv[v];
        a.out[v * N + p] = fma(a.a, K, ops[v]);
      }
      break;
    case EPI_SSP_2:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = kp[v] + cv[v];
        a.out[v * N + p] = 0.75 * ops[v] + 0.25 * fma(a.a, K, ops[5 + v]);
      }
      break;
    case EPI_SSP_3:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = kp[v] + cv[v];
        a.out[v * N + p] = (1.0 / 3.0) * ops[v] + (2.0 / 3.0) * fma(a.a, K, ops[5 + v]);
      }
      break;
    default:
      break;
  }
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned), L2 only.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// dir_epilogue_pre32 for two x-adjacent points p and p + 1 (p even), their operands and results
// moved as 16-byte pairs: kp[v] = (k at p, k at p + 1), ops[j] likewise; the same arithmetic.
__device__ __forceinline__ void dir_epilogue_pre32x2(const DirArgs& a, long long p, const double c0[5],
                                                     const double c1[5], const double2* kp, const double2* ops) {
  const long long N = a.g.N;
  auto st = [&](double* base, int v, double x0, double x1) {
    *reinterpret_cast<double2*>(base + v * N + p) = make_double2(x0, x1);
  };
  switch (a.epi) {
    case EPI_ACC_WRITE:
#pragma unroll
      for (int v = 0; v < 5; ++v) st(a.k, v, c0[v], c1[v]);
      break;
    case EPI_ACC_ADD:
#pragma unroll
      for (int v = 0; v < 5; ++v) st(a.k, v, kp[v].x + c0[v], kp[v].y + c1[v]);
      break;
    case EPI_RHS_OUT:
#pragma unroll
      for (int v = 0; v < 5; ++v) st(a.out, v, kp[v].x + c0[v], kp[v].y + c1[v]);
      break;
    case EPI_RK4_FIRST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K0 = kp[v].x + c0[v], K1 = kp[v].y + c1[v];
        st(a.out, v, fma(a.a, K0, ops[v].x), fma(a.a, K1, ops[v].y));
        st(a.acc, v, K0, K1);
      }
      break;
    case EPI_RK4_MID:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K0 = kp[v].x + c0[v], K1 = kp[v].y + c1[v];
        st(a.out, v, fma(a.a, K0, ops[v].x), fma(a.a, K1, ops[v].y));
        st(a.acc, v, fma(2.0, K0, ops[5 + v].x), fma(2.0, K1, ops[5 + v].y));
      }
      break;
    case EPI_RK4_LAST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K0 = kp[v].x + c0[v], K1 = kp[v].y + c1[v];
        st(a.out, v, fma(a.a, ops[5 + v].x + K0, ops[v].x), fma(a.a, ops[5 + v].y + K1, ops[v].y));
      }
      break;
    case EPI_SSP_1:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K0 = kp[v].x + c0[v], K1 = kp[v].y + c1[v];
        st(a.out, v, fma(a.a, K0, ops[v].x), fma(a.a, K1, ops[v].y));
      }
      break;
    case EPI_SSP_2:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K0 = kp[v].x + c0[v], K1 = kp[v].y + c1[v];
        st(a.out, v, 0.75 * ops[v].x + 0.25 * fma(a.a, K0, ops[5 + v].x),
           0.75 * ops[v].y + 0.25 * fma(a.a, K1, ops[5 + v].y));
      }
      break;
    case EPI_SSP_3:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K0 = kp[v].x + c0[v], K1 = kp[v].y + c1[v];
        st(a.out, v, (1.0 / 3.0) * ops[v].x + (2.0 / 3.0) * fma(a.a, K0, ops[5 + v].x),
           (1.0 / 3.0) * ops[v].y + (2.0 / 3.0) * fma(a.a, K1, ops[5 + v].y));
      }
      break;
    default:
      break;
  }
}

template <int D>
__global__ void __launch_bounds__(THREADS, 4) k_dir32(const DirArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* Q = reinterpret_cast<float*>(smem + OFF_Q);
  float4* R4 = reinterpret_cast<float4*>(smem + OFF_R4);
  float* HS = reinterpret_cast<float*>(smem + OFF_H);
  float4* V4 = reinterpret_cast<float4*>(smem + OFF_V4);
  float* REC = reinterpret_cast<float*>(smem + OFF_REC);
  double* FD = reinterpret_cast<double*>(smem + OFF_F);
  double* PRE = reinterpret_cast<double*>(smem + OFF_Q);
  double* PRE2 = reinterpret_cast<double*>(smem + OFF_P2);

  constexpr int AX = (D == 0) ? 1 : 0;
  const int nD = a.g.n[D], na = a.g.n[AX];
  const long long N = a.g.N;
  const bool swap = (D == 2 && a.zorder);  // z pass with the line groups first (dir_zorder)
  const int s0 = (swap ? blockIdx.y : blockIdx.x) * TP;
  const int a0 = (swap ? blockIdx.x : blockIdx.y) * W;
  const int bz = blockIdx.z;
  const int tid = threadIdx.x;
  const float* fvf = reinterpret_cast<const float*>(a.fv);
  const long long fv_plane = (long long)(a.fv_dstride * D);
  // FP32 parameters rounded on the host (an FP64 -> FP32 conversion per thread would occupy the FP64 pipe)
  const float gm1 = a.gm1_hi;

  // ---- A: load, convert, primitive variables and point fluxes -------------------------
  int bad = 0;
  for (int it = tid; it < NP * W; it += THREADS) {
    int pos, line;
    if (D == 0) {
      line = it / NP;
      pos = it - line * NP;
    } else {
      pos = it / W;
      line = it - pos * W;
    }
    int c = s0 - 3 + pos;
    if (c < 0 || c >= nD) c = wrap_idx(c, nD);
    const int la = min(a0 + line, na - 1);
    const long long p = tile_flat<D>(a.g, c, la, bz);
    const float rho = d2f_tz(__ldg(a.u + p)), mx = d2f_tz(__ldg(a.u + N + p));
    const float my = d2f_tz(__ldg(a.u + 2 * N + p)), mz = d2f_tz(__ldg(a.u + 3 * N + p));
    const float e = d2f_tz(__ldg(a.u + 4 * N + p));
    float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (fvf != nullptr) {
      const float* fp = fvf + fv_plane * N + p;
      fv = make_float4(__ldg(fp), __ldg(fp + N), __ldg(fp + 2 * N), __ldg(fp + 3 * N));
    }
    const float ri = rcp_a(rho);
    const float vx = mx * ri, vy = my * ri, vz = mz * ri;
    const float ke2 = fmaf(mx, vx, fmaf(my, vy, mz * vz));
    const float pr = gm1 * fmaf(-0.5f, ke2, e);
    const float ep = e + pr;
    bad |= !(rho > 0.0f && rho < INFINITY && pr > 0.0f && pr < INFINITY);
    const float un = (D == 0) ? vx : (D == 1) ? vy : vz;
    float* q = Q + line * LS + pos;
    q[0 * W * LS] = rho;
    q[1 * W * LS] = mx;
    q[2 * W * LS] = my;
    q[3 * W * LS] = mz;
    q[4 * W * LS] = e;
    q[5 * W * LS] = (D == 0) ? fmaf(mx, un, pr) : mx * un;
    q[6 * W * LS] = (D == 1) ? fmaf(my, un, pr) : my * un;
    q[7 * W * LS] = (D == 2) ? fmaf(mz, un, pr) : mz * un;
    q[8 * W * LS] = ep * un;
    float sr;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sr) : "f"(rho));
    R4[line * L4 + pos] = make_float4(sr, vx, vy, vz);
    HS[line * L4 + pos] = ep * ri;
    V4[line * L4 + pos] = fv;
  }
  __syncthreads();

  // ---- BC: WENO5 left/right values, SEG interfaces of one scalar on one line per item -------
  // Items run over lines fastest, then segments, then scalars, so that the 8 threads of a
  // shared-memory phase read and write 8 different banks.
  {
    const float eps4 = a.eps4_hi;
    const bool eps_ok = eps4 >= 1e-9f && eps4 <= 1.0f;  // unscaled products stay in range (see below)
    for (int it = tid; it < NQ * W * NSEG; it += THREADS) {
      const int m = it / (W * NSEG);
      const int rem = it - m * (W * NSEG);
      const int seg = rem / W, line = rem - seg * W;
      const float* q = Q + (m * W + line) * LS + SEG * seg;
      const float4 qa = *reinterpret_cast<const float4*>(q);
      const float4 qb = *reinterpret_cast<const float4*>(q + 4);
      const float4 qc = *reinterpret_cast<const float4*>(q + 8);
      const float P[SEG + 5] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w, qc.x};
      // first, second and third differences; window w = points w, w+1, w+2
      float g[SEG + 4], sd[SEG + 3], T3[SEG + 2], T2[SEG + 2];
      float gmax = 0.0f;
#pragma unroll
      for (int k = 0; k < SEG + 4; ++k) {
        g[k] = P[k + 1] - P[k];
        gmax = fmaxf(gmax, fabsf(g[k]));
      }
#pragma unroll
      for (int w = 0; w < SEG + 3; ++w) sd[w] = g[w + 1] - g[w];
#pragma unroll
      for (int k = 0; k < SEG + 2; ++k) {
        const float T = sd[k + 1] - sd[k];
        T3[k] = (1.0f / 3.0f) * T;
        T2[k] = 0.5f * T;
      }
      // window indicators, roles 1..3 (first-derivative term at the window's right end, centre,
      // left end)
      float B[SEG + 3][3];
#pragma unroll
      for (int w = 0; w < SEG + 3; ++w) {
        const float gm = g[w], gp = g[w + 1];
        const float aa = fmaf((13.0f / 3.0f) * sd[w], sd[w], eps4);
        const float u1 = fmaf(3.0f, gp, -gm), u2 = gm + gp, u3 = fmaf(-3.0f, gm, gp);
        const float b1 = fmaf(u1, u1, aa), b2 = fmaf(u2, u2, aa), b3 = fmaf(u3, u3, aa);
        B[w][0] = b1 * b1;
        B[w][1] = b2 * b2;
        B[w][2] = b3 * b3;
      }
      // With every first difference <= 64 in magnitude and 1e-9 <= 4 eps <= 1, each B lies in
      // [(4 eps)^2, (34 * 64^2 + 1)^2] and the products and the numerator stay within the normal
      // FP32 range: the unscaled form is exact to FP32 rounding.
      const bool fast = eps_ok && gmax <= 64.0f;
      float vL[SEG], vR[SEG];
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        // interface j: left-biased from points j..j+4, right-biased from j+1..j+5; candidate-2
        // values eR (left) and eL (right); F_1 - F_2 = -T_j/3, F_3 - F_2 = -T_{j+1}/6 (left),
        // F_1 - F_2 = T_{j+2}/3, F_3 - F_2 = T_{j+1}/6 (right)
        const float eR = fmaf(1.0f / 3.0f, g[j + 2], fmaf(1.0f / 6.0f, g[j + 1], P[j + 2]));
        const float eL = fmaf(-1.0f / 6.0f, g[j + 3], fmaf(-1.0f / 3.0f, g[j + 2], P[j + 3]));
        if (fast) {
          vL[j] = weno_fast(B[j][0], B[j + 1][1], B[j + 2][2], eR, -T3[j], -T2[j + 1]);
          vR[j] = weno_fast(B[j + 3][2], B[j + 2][1], B[j + 1][0], eL, T3[j + 2], T2[j + 1]);
        } else {
          vL[j] = weno_safe(B[j][0], B[j + 1][1], B[j + 2][2], eR, -T3[j], -T2[j + 1]);
          vR[j] = weno_safe(B[j + 3][2], B[j + 2][1], B[j + 1][0], eL, T3[j + 2], T2[j + 1]);
        }
      }
      float* r = REC + line * NI + SEG * seg;
      if (m < 5) {
        *reinterpret_cast<float4*>(r + m * W * NI) =
            make_float4(vR[0] - vL[0], vR[1] - vL[1], vR[2] - vL[2], vR[3] - vL[3]);
        if (m == 1 + D)
          *reinterpret_cast<float4*>(r + 5 * W * NI) =
              make_float4(vL[0] + vR[0], vL[1] + vR[1], vL[2] + vR[2], vL[3] + vR[3]);
      } else {
        *reinterpret_cast<float4*>(r + (m + 1) * W * NI) =
            make_float4(vL[0] + vR[0], vL[1] + vR[1], vL[2] + vR[2], vL[3] + vR[3]);
      }
    }
  }
  __syncthreads();

  // ---- epilogue operand k: fetched asynchronously into the dead scalar planes while D runs;
  //      each thread later reads only its own point's slots
  auto point_of = [&](int it, int& pp, int& line) {
    if (D == 0) {
      line = it / TP;
      pp = it - line * TP;
    } else {
      pp = it / W;
      line = it - pp * W;
    }
  };
  const int nops = epilogue_operands(a.epi);  // k, then U_n, then acc or the stage input
  // y and z passes on grids with nx even: a thread owns two x-adjacent points (lines 2j, 2j+1 of
  // the tile; their flat index is even, so every operand pair is 16-byte aligned)
  const bool pairs = (D != 0) && ((a.g.n[0] & 1) == 0);
  const double* third = (a.epi == EPI_SSP_2 || a.epi == EPI_SSP_3) ? a.u : a.acc;
  if (pairs) {
    if (nops > 0 && tid < TP * W / 2) {
      const int pp = tid / (W / 2), l0 = 2 * (tid - pp * (W / 2));
      if (s0 + pp < nD && a0 + l0 < na) {  // na = nx is even: the second point exists too
        const long long p = tile_flat<D>(a.g, s0 + pp, a0 + l0, bz);
        double2* kp = reinterpret_cast<double2*>(PRE) + 5 * tid;
        double2* op = reinterpret_cast<double2*>(PRE2) + 10 * tid;
#pragma unroll
        for (int v = 0; v < 5; ++v) cp_async16(kp + v, a.k + v * N + p);
        if (nops >= 10) {
#pragma unroll
          for (int v = 0; v < 5; ++v) cp_async16(op + v, a.un + v * N + p);
        }
        if (nops == 15) {
#pragma unroll
          for (int v = 0; v < 5; ++v) cp_async16(op + 5 + v, third + v * N + p);
        }
      }
    }
  } else if (nops > 0 && tid < TP * W) {
    int pp, line;
    point_of(tid, pp, line);
    if (s0 + pp < nD && a0 + line < na) {
      const long long p = tile_flat<D>(a.g, s0 + pp, a0 + line, bz);
#pragma unroll
      for (int v = 0; v < 5; ++v) cp_async8(PRE + 5 * tid + v, a.k + v * N + p);
      if (nops >= 10) {
#pragma unroll
        for (int v = 0; v < 5; ++v) cp_async8(PRE2 + 10 * tid + v, a.un + v * N + p);
      }
      if (nops == 15) {
#pragma unroll
        for (int v = 0; v < 5; ++v) cp_async8(PRE2 + 10 * tid + 5 + v, third + v * N + p);
      }
    }
  }
  cp_async_commit();

  // ---- D: Roe flux + viscous interface flux, / dx, widened to FP64 ----------------------
  if (tid < NI * W) {
    int r, line;
    if (D == 0) {
      line = tid / NI;
      r = tid - line * NI;
    } else {
      r = tid / W;
      line = tid - r * W;
    }
    // interface r lies between the tile's points r - 1 and r, i.e. positions r + 2 and r + 3
    const float* rc_ = REC + line * NI + r;
    float du[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) du[v] = rc_[v * W * NI];
    const float S0 = rc_[5 * W * NI];
    const float S1 = rc_[6 * W * NI], S2 = rc_[7 * W * NI], S3 = rc_[8 * W * NI], S4 = rc_[9 * W * NI];
    const float4 qa = R4[line * L4 + r + 2], qb = R4[line * L4 + r + 3];
    const float Ha = HS[line * L4 + r + 2], Hb = HS[line * L4 + r + 3];
    const float rs = rcp_a(qa.x + qb.x);
    const float wa = qa.x * rs, wb = qb.x * rs;
    const float V0 = fmaf(wa, qa.y, wb * qb.y), V1 = fmaf(wa, qa.z, wb * qb.z), V2 = fmaf(wa, qa.w, wb * qb.w);
    const float H = fmaf(wa, Ha, wb * Hb);
    const float q2h = 0.5f * fmaf(V0, V0, fmaf(V1, V1, V2 * V2));
    const float c2 = gm1 * (H - q2h);
    bad |= !(c2 > 0.0f);
    const float rc = rsqrt_a(c2);
    const float c = c2 * rc;
    constexpr int T1 = (D == 0) ? 1 : 0;
    constexpr int T2 = (D == 2) ? 1 : 2;
    const float V[3] = {V0, V1, V2};
    const float un = V[D], vt1 = V[T1], vt2 = V[T2];
    const float b1 = gm1 * (rc * rc);
    const float vdm = fmaf(V0, du[1], fmaf(V1, du[2], V2 * du[3]));
    const float phi = b1 * (fmaf(q2h, du[0], du[4]) - vdm);
    const float a2 = du[0] - phi;
    const float a3 = fmaf(-vt1, du[0], du[1 + T1]);
    const float a4 = fmaf(-vt2, du[0], du[1 + T2]);
    const float ach = 0.5f * (fmaf(un, du[0], -du[1 + D]) * rc);
    const float ph = 0.5f * phi;
    const float a1 = ph + ach, a5 = ph - ach;
    float l1 = fabsf(un - c), l5 = fabsf(un + c);
    const float l2 = fabsf(un);
    const float hd = a.hd_hi;
    const float delta = hd * c;
    if (l1 < delta) l1 = fmaf(l1, l1, delta * delta) * __fdividef(0.5f, delta);
    if (l5 < delta) l5 = fmaf(l5, l5, delta * delta) * __fdividef(0.5f, delta);
    const float A1 = l1 * a1, A2 = l2 * a2, A3 = l2 * a3, A4 = l2 * a4, A5 = l5 * a5;
    const float S = A1 + A5;
    const float d0 = S + A2;
    const float cD = c * (A5 - A1);
    float diss[5];
    diss[0] = d0;
    diss[1 + D] = fmaf(d0, un, cD);
    diss[1 + T1] = fmaf(d0, vt1, A3);
    diss[1 + T2] = fmaf(d0, vt2, A4);
    diss[4] = fmaf(S, H, fmaf(cD, un, fmaf(A2, q2h, fmaf(A3, vt1, A4 * vt2))));
    // viscous interface flux: its difference over the two faces of a point is the 4th-order
    // central derivative (f_{i-2} - 8 f_{i-1} + 8 f_{i+1} - f_{i+2}) / 12 of the point values
    const float4 fm1 = V4[line * L4 + r + 1], f0 = V4[line * L4 + r + 2];
    const float4 f1 = V4[line * L4 + r + 3], f2 = V4[line * L4 + r + 4];
    const float G0 = fmaf(7.0f / 12.0f, f0.x + f1.x, (-1.0f / 12.0f) * (fm1.x + f2.x));
    const float G1 = fmaf(7.0f / 12.0f, f0.y + f1.y, (-1.0f / 12.0f) * (fm1.y + f2.y));
    const float G2 = fmaf(7.0f / 12.0f, f0.z + f1.z, (-1.0f / 12.0f) * (fm1.z + f2.z));
    const float G3 = fmaf(7.0f / 12.0f, f0.w + f1.w, (-1.0f / 12.0f) * (fm1.w + f2.w));
    const float rdx = a.g.rh_f[D];
    const float F0 = 0.5f * (S0 - diss[0]);
    const float F1 = fmaf(0.5f, S1 - diss[1], -G0);
    const float F2 = fmaf(0.5f, S2 - diss[2], -G1);
    const float F3 = fmaf(0.5f, S3 - diss[3], -G2);
    const float F4 = fmaf(0.5f, S4 - diss[4], -G3);
    double* fd = FD + line * FS + r;
    fd[0 * W * FS] = f2d_bits(F0 * rdx);
    fd[1 * W * FS] = f2d_bits(F1 * rdx);
    fd[2 * W * FS] = f2d_bits(F2 * rdx);
    fd[3 * W * FS] = f2d_bits(F3 * rdx);
    fd[4 * W * FS] = f2d_bits(F4 * rdx);
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(a.status, ST_NONPHYS);
  cp_async_wait_all();
  __syncthreads();

  // ---- E: FP64 conservative difference + epilogue ----------------------------------------
  if (pairs) {
    if (tid < TP * W / 2) {
      const int pp = tid / (W / 2), l0 = 2 * (tid - pp * (W / 2));
      if (s0 + pp < nD && a0 + l0 < na) {
        const double* f0 = FD + l0 * FS + pp;
        const double* f1 = f0 + FS;
        double c0[5], c1[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          c0[v] = f0[v * W * FS] - f0[v * W * FS + 1];
          c1[v] = f1[v * W * FS] - f1[v * W * FS + 1];
        }
        dir_epilogue_pre32x2(a, tile_flat<D>(a.g, s0 + pp, a0 + l0, bz), c0, c1,
                             reinterpret_cast<const double2*>(PRE) + 5 * tid,
                             reinterpret_cast<const double2*>(PRE2) + 10 * tid);
      }
    }
  } else if (tid < TP * W) {
    int pp, line;
    point_of(tid, pp, line);
    if (s0 + pp < nD && a0 + line < na) {
      const double* fd = FD + line * FS + pp;
      double cv[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) cv[v] = fd[v * W * FS] - fd[v * W * FS + 1];
      dir_epilogue_pre32(a, tile_flat<D>(a.g, s0 + pp, a0 + line, bz), cv, PRE + 5 * tid, PRE2 + 10 * tid);
    }
  }
}

template <int D>
cudaError_t launch32(const DirArgs& a, cudaStream_t s) {
  constexpr int AX = (D == 0) ? 1 : 0;
  constexpr int BX = (D == 2) ? 1 : 2;
  dim3 grid((a.g.n[D] + TP - 1) / TP, (a.g.n[AX] + W - 1) / W, a.g.n[BX]);
  if (D == 2 && a.zorder) {
    const unsigned t = grid.x;
    grid.x = grid.y;
    grid.y = t;
  }
  k_dir32<D><<<grid, THREADS, BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t attr32() {
  cudaError_t e = cudaFuncSetAttribute(k_dir32<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dir32<D>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

}  // namespace

cudaError_t prepare_dir32_kernels() {
  cudaError_t e = attr32<0>();
  if (e == cudaSuccess) e = attr32<1>();
  if (e == cudaSuccess) e = attr32<2>();
  return e;
}

// One tile shape (27 x 8) for every pass; the tile variants of the FP64 modes do not apply.
cudaError_t launch_dir32(int d, const DirArgs& a, cudaStream_t s) {
  if (d == 0) return launch32<0>(a, s);
  if (d == 1) return launch32<1>(a, s);
  return launch32<2>(a, s);
}

}  // namespace ns3d
