// FP32-bulk direction pass (precision NS3D_FP32_BULK): the same fused WENO5 +
// Roe + conservative difference + viscous divergence as k_dir.cu, with the
// point fluxes, smoothness indicators, weights, interface values and the Roe
// flux in FP32 (arXiv 2211.16718, Sec. 2.2 arithmetic unchanged, precision
// reduced).  The interface fluxes are widened to FP64 before the conservative
// difference, so the sum over the grid still telescopes exactly; the viscous
// divergence, the accumulation / RK stage update and the state stay in FP64.
// FP64 <-> FP32 conversions use integer bit manipulation (round to nearest), so
// the FP64 pipe only carries the difference, the viscous divergence and the
// epilogue.
#include <math.h>

#include "df.cuh"
#include "k_dir_common.cuh"
#include "ns3d_internal.cuh"

namespace ns3d {

namespace {

constexpr int NQ = 9;
constexpr int THREADS = 256;  // 8 warps per tile: latency hiding for the FP32 chains

// Tile plan: TP points along the pencil x W lines.  The y and z passes can run 32 x 4 or
// 16 x 8 tiles (W consecutive x-lines per row of loads).  Every shape computes the same bits
// (the per-interface arithmetic does not depend on the tiling).
template <int TP_, int W_>
struct P32 {
  static constexpr int TP = TP_, W = W_;
  static constexpr int NP = TP + 6, NW = TP + 4, NI = TP + 1;
  // shared-memory plan (4-byte words)
  static constexpr int OFF_Q = 0;                          // float [NQ][NP*W]
  static constexpr int OFF_ROE = OFF_Q + NQ * NP * W;      // float [5][NP*W]
  static constexpr int OFF_B = OFF_ROE + 5 * NP * W;       // float [NQ][3][NW*W]
  static constexpr int OFF_R = OFF_B + NQ * 3 * NW * W;    // float [18][NI*W]
  static constexpr int OFF_FV = (OFF_R + 18 * NI * W + 1) & ~1;  // double [4][NP*W]
  static constexpr int OFF_F = OFF_FV + 2 * 4 * NP * W;    // double [5][NI*W]
  static constexpr int WORDS = OFF_F + 2 * 5 * NI * W;
  static constexpr int BYTES = WORDS * 4;
};

__device__ __forceinline__ float weno_combine32(float B1, float B2, float B3, float F1, float F2, float F3) {
  // common power-of-two scaling keeps the products in range (omega is scale-free)
  const int E = max(exponent_of(B1), max(exponent_of(B2), exponent_of(B3)));
  const float sc = pow2f(-E);
  B1 *= sc;
  B2 *= sc;
  B3 *= sc;
  const float p23 = B2 * B3;
  const float t13 = 6.0f * (B1 * B3);
  const float t12 = 3.0f * (B1 * B2);
  const float num = fmaf(p23, F1, fmaf(t13, F2, t12 * F3));
  const float den = p23 + t13 + t12;
  return __fdiv_rn(num, den);
}

template <int D, int TP_, int W_>
__global__ void __launch_bounds__(THREADS) k_dir32(const DirArgs a) {
  using PL = P32<TP_, W_>;
  constexpr int TP = PL::TP, W = PL::W, NP = PL::NP, NW = PL::NW, NI = PL::NI;
  constexpr int OFF_Q = PL::OFF_Q, OFF_ROE = PL::OFF_ROE, OFF_B = PL::OFF_B, OFF_R = PL::OFF_R;
  constexpr int OFF_FV = PL::OFF_FV, OFF_F = PL::OFF_F;
  extern __shared__ float smf[];
  double* smd = reinterpret_cast<double*>(smf);
  const int nD = a.g.n[D];
  constexpr int AX = (D == 0) ? 1 : 0;
  const int na = a.g.n[AX];
  const long long N = a.g.N;
  const bool swap = (D == 2 && a.zorder);  // z pass with the line groups first (dir_zorder)
  const int s0 = (swap ? blockIdx.y : blockIdx.x) * TP;
  const int a0 = (swap ? blockIdx.x : blockIdx.y) * W;
  const int bz = blockIdx.z;
  const int tid = threadIdx.x;

  // ---- A: load, convert, point fluxes in FP32 ---------------------------------
  for (int item = tid; item < NP * W; item += THREADS) {
    int pos, line;
    tile_split<D, W>(item, NP, pos, line);
    const int c = wrap_idx(s0 - 3 + pos, nD);
    const int la = min(a0 + line, na - 1);
    const long long p = tile_flat<D>(a.g, c, la, bz);
    float U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = d2f_rn(__ldg(a.u + v * N + p));
    const float vx = d2f_rn(__ldg(a.pm + PM_U * N + p)), vy = d2f_rn(__ldg(a.pm + PM_V * N + p));
    const float vz = d2f_rn(__ldg(a.pm + PM_W * N + p)), pr = d2f_rn(__ldg(a.pm + PM_P * N + p));
    const float un = (D == 0) ? vx : (D == 1) ? vy : vz;
    const int s = tile_idx<D, W>(pos, line, NP);
    float* q = smf + OFF_Q;
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v * NP * W + s] = U[v];
    q[5 * NP * W + s] = (D == 0) ? fmaf(U[1], un, pr) : U[1] * un;
    q[6 * NP * W + s] = (D == 1) ? fmaf(U[2], un, pr) : U[2] * un;
    q[7 * NP * W + s] = (D == 2) ? fmaf(U[3], un, pr) : U[3] * un;
    q[8 * NP * W + s] = (U[4] + pr) * un;
    float* r = smf + OFF_ROE;
    r[0 * NP * W + s] = d2f_rn(__ldg(a.pm + PM_SR * N + p));
    r[1 * NP * W + s] = vx;
    r[2 * NP * W + s] = vy;
    r[3 * NP * W + s] = vz;
    r[4 * NP * W + s] = d2f_rn(__ldg(a.pm + PM_H * N + p));
    if (a.fv != nullptr) {  // FP64 as stored, first read in phase E: copied asynchronously
      double* f = smd + OFF_FV / 2;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) cp_async8(f + cc * NP * W + s, a.fv + (long long)(a.fv_dstride * D + cc) * N + p);
    }
  }
  cp_async_commit();
  __syncthreads();

  // ---- B: squared scaled smoothness indicators (FP32) --------------------------
  {
    const float* q = smf + OFF_Q;
    float* bw = smf + OFF_B;
    const float eps4 = (float)a.eps4;
    for (int item = tid; item < NQ * NW * W; item += THREADS) {
      const int m = item / (NW * W);
      int w, line;
      tile_split<D, W>(item - m * NW * W, NW, w, line);
      const float* qm = q + m * NP * W;
      const float x = qm[tile_idx<D, W>(w, line, NP)];
      const float y = qm[tile_idx<D, W>(w + 1, line, NP)];
      const float z = qm[tile_idx<D, W>(w + 2, line, NP)];
      const float gm = y - x, gp = z - y, sd = gp - gm;
      const float aa = fmaf((13.0f / 3.0f) * sd, sd, eps4);
      const float u1 = fmaf(3.0f, gp, -gm), u2 = gm + gp, u3 = fmaf(-3.0f, gm, gp);
      const float b1 = fmaf(u1, u1, aa), b2 = fmaf(u2, u2, aa), b3 = fmaf(u3, u3, aa);
      const int o = tile_idx<D, W>(w, line, NW);
      bw[(m * 3 + 0) * NW * W + o] = b1 * b1;
      bw[(m * 3 + 1) * NW * W + o] = b2 * b2;
      bw[(m * 3 + 2) * NW * W + o] = b3 * b3;
    }
  }
  __syncthreads();

  // ---- C: left/right WENO5 values (FP32) -------------------------------------------
  {
    const float* q = smf + OFF_Q;
    const float* bw = smf + OFF_B;
    float* rec = smf + OFF_R;
    for (int item = tid; item < NQ * NI * W; item += THREADS) {
      const int m = item / (NI * W);
      int f, line;
      tile_split<D, W>(item - m * NI * W, NI, f, line);
      const float* qm = q + m * NP * W;
      const float P0 = qm[tile_idx<D, W>(f, line, NP)], P1 = qm[tile_idx<D, W>(f + 1, line, NP)];
      const float P2 = qm[tile_idx<D, W>(f + 2, line, NP)], P3 = qm[tile_idx<D, W>(f + 3, line, NP)];
      const float P4 = qm[tile_idx<D, W>(f + 4, line, NP)], P5 = qm[tile_idx<D, W>(f + 5, line, NP)];
      const float xR = fmaf(11.0f / 6.0f, P2, fmaf(-7.0f / 6.0f, P1, (1.0f / 3.0f) * P0));
      const float eR = fmaf(1.0f / 3.0f, P3, fmaf(5.0f / 6.0f, P2, (-1.0f / 6.0f) * P1));
      const float eL = fmaf(-1.0f / 6.0f, P4, fmaf(5.0f / 6.0f, P3, (1.0f / 3.0f) * P2));
      const float xL = fmaf(1.0f / 3.0f, P5, fmaf(-7.0f / 6.0f, P4, (11.0f / 6.0f) * P3));
      const float* b = bw + m * 3 * NW * W;
      const float vL = weno_combine32(b[0 * NW * W + tile_idx<D, W>(f, line, NW)], b[1 * NW * W + tile_idx<D, W>(f + 1, line, NW)],
                                      b[2 * NW * W + tile_idx<D, W>(f + 2, line, NW)], xR, eR, eL);
      const float vR = weno_combine32(b[2 * NW * W + tile_idx<D, W>(f + 3, line, NW)], b[1 * NW * W + tile_idx<D, W>(f + 2, line, NW)],
                                      b[0 * NW * W + tile_idx<D, W>(f + 1, line, NW)], xL, eL, eR);
      const int o = tile_idx<D, W>(f, line, NI);
      rec[(2 * m) * NI * W + o] = vL;
      rec[(2 * m + 1) * NI * W + o] = vR;
    }
  }
  cp_async_wait_all();  // this thread's viscous-flux copies; the barrier publishes them
  __syncthreads();

  // ---- epilogue operands: fetched asynchronously into the (now unused) indicator space
  //      while phase D runs; each thread later reads only its own point's slots
  static_assert(TP * W <= THREADS, "one epilogue point per thread");
  static_assert(30 * TP * W <= NQ * 3 * NW * W && OFF_B % 2 == 0, "prefetch slots fit the indicator space");
  double* pre = smd + OFF_B / 2 + 15 * tid;
  if (tid < TP * W) {
    int pp, line;
    tile_split<D, W>(tid, TP, pp, line);
    if (s0 + pp < nD && a0 + line < na) epilogue_prefetch(a, tile_flat<D>(a.g, s0 + pp, a0 + line, bz), pre);
  }
  cp_async_commit();

  // ---- D: Roe flux (FP32), widened to FP64 -----------------------------------------
  {
    const float gm1 = (float)(a.gamma - 1.0);
    const float hdelta = (float)a.hdelta;
    const float* r = smf + OFF_ROE;
    const float* rec = smf + OFF_R;
    double* F = smd + OFF_F / 2;
    int bad = 0;
    for (int item = tid; item < NI * W; item += THREADS) {
      int f, line;
      tile_split<D, W>(item, NI, f, line);
      const int o = tile_idx<D, W>(f, line, NI);
      float uL[5], uR[5], fL[5], fR[5];
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
      const int sa = tile_idx<D, W>(f + 2, line, NP), sb = tile_idx<D, W>(f + 3, line, NP);
      const float ra = r[sa], rb = r[sb];
      const float rs = __frcp_rn(ra + rb);
      const float wa = ra * rs, wb = rb * rs;
      float V[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) V[m] = fmaf(wa, r[(1 + m) * NP * W + sa], wb * r[(1 + m) * NP * W + sb]);
      const float H = fmaf(wa, r[4 * NP * W + sa], wb * r[4 * NP * W + sb]);
      const float q2h = 0.5f * fmaf(V[0], V[0], fmaf(V[1], V[1], V[2] * V[2]));
      const float c2 = gm1 * (H - q2h);
      bad |= !(c2 > 0.0f);
      const float c = __fsqrt_rn(c2);
      const float rc = __frcp_rn(c);
      float du[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) du[v] = uR[v] - uL[v];
      constexpr int T1 = (D == 0) ? 1 : 0;
      constexpr int T2 = (D == 2) ? 1 : 2;
      const float un = V[D], vt1 = V[T1], vt2 = V[T2];
      const float b1 = gm1 * (rc * rc);
      const float vdm = fmaf(V[0], du[1], fmaf(V[1], du[2], V[2] * du[3]));
      const float phi = b1 * (fmaf(q2h, du[0], du[4]) - vdm);
      const float a2 = du[0] - phi;
      const float a3 = fmaf(-vt1, du[0], du[1 + T1]);
      const float a4 = fmaf(-vt2, du[0], du[1 + T2]);
      const float ach = 0.5f * (fmaf(un, du[0], -du[1 + D]) * rc);
      const float ph = 0.5f * phi;
      const float a1 = ph + ach, a5 = ph - ach;
      float l1 = fabsf(un - c), l5 = fabsf(un + c);
      const float l2 = fabsf(un);
      const float delta = hdelta * c;
      if (l1 < delta) l1 = (l1 * l1 + delta * delta) / (2.0f * delta);
      if (l5 < delta) l5 = (l5 * l5 + delta * delta) / (2.0f * delta);
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
#pragma unroll
      for (int v = 0; v < 5; ++v) F[v * NI * W + o] = f2d_bits(0.5f * (fL[v] + fR[v] - diss[v]));
    }
    if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(a.status, ST_NONPHYS);
  }
  __syncthreads();

  // ---- E: FP64 conservative difference + viscous divergence + epilogue -------------
  cp_async_wait_all();
  {
    const double rdx = a.g.rh[D];
    const double r12 = a.g.r12h[D];
    const double* F = smd + OFF_F / 2;
    const double* fvs = smd + OFF_FV / 2;
    for (int item = tid; item < TP * W; item += THREADS) {
      int pp, line;
      tile_split<D, W>(item, TP, pp, line);
      if (s0 + pp >= nD || a0 + line >= na) continue;
      double cv[5];
      const int op = tile_idx<D, W>(pp + 1, line, NI), om = tile_idx<D, W>(pp, line, NI);
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
      dir_epilogue_pre(a, tile_flat<D>(a.g, s0 + pp, a0 + line, bz), cv, pre);
    }
  }
}

template <int D, int TP, int W>
cudaError_t launch32(const DirArgs& a, cudaStream_t s) {
  constexpr int AX = (D == 0) ? 1 : 0;
  constexpr int BX = (D == 2) ? 1 : 2;
  dim3 grid((a.g.n[D] + TP - 1) / TP, (a.g.n[AX] + W - 1) / W, a.g.n[BX]);
  if (D == 2 && a.zorder) {
    const unsigned t = grid.x;
    grid.x = grid.y;
    grid.y = t;
  }
  k_dir32<D, TP, W><<<grid, THREADS, P32<TP, W>::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int D, int TP, int W>
cudaError_t attr32() {
  return cudaFuncSetAttribute(k_dir32<D, TP, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, P32<TP, W>::BYTES);
}

}  // namespace

cudaError_t prepare_dir32_kernels() {
  cudaError_t e = attr32<0, 32, 4>();
  if (e == cudaSuccess) e = attr32<1, 16, 8>();
  if (e == cudaSuccess) e = attr32<2, 16, 8>();
  if (e == cudaSuccess) e = attr32<1, 32, 4>();
  if (e == cudaSuccess) e = attr32<2, 32, 4>();
  return e;
}

// x pass: 32 x 4.  y and z passes by the context's variant: 0 -> y 32 x 4, z 16 x 8 (the fastest
// measured on GB300 at 256^3 with the epilogue prefetch); 1 -> y and z 32 x 4; 2 -> y and z 16 x 8.
cudaError_t launch_dir32(int d, const DirArgs& a, cudaStream_t s) {
  if (d == 0) return launch32<0, 32, 4>(a, s);
  if (d == 1) return (a.variant == 2) ? launch32<1, 16, 8>(a, s) : launch32<1, 32, 4>(a, s);
  return (a.variant == 1) ? launch32<2, 32, 4>(a, s) : launch32<2, 16, 8>(a, s);
}

}  // namespace ns3d
