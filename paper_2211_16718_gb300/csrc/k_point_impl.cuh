// Per-point bodies of the primitive-variable and viscous-flux passes (FP64),
// shared by the standalone kernels (k_pointwise.cu) and the batched / persistent
// ensemble kernels (ns3d_batch.cu).
#pragma once

#include <math.h>

#include "df.cuh"
#include "ns3d_internal.cuh"

namespace ns3d {

// Global load through the read-only cache (NC) or a plain coherent load.
template <bool NC>
__device__ __forceinline__ double ldx(const double* p) {
  if (NC) return __ldg(p);
  return *p;
}

// Positive and finite, from the bit pattern (integer compare, no FP64 instruction).
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool is_finite_bits(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
}

// A double-float value stored in an 8-byte plane slot (hi, lo as two floats).
__device__ __forceinline__ void store_df(double* slot, df v) { *reinterpret_cast<float2*>(slot) = make_float2(v.hi, v.lo); }
__device__ __forceinline__ df load_df(const double* slot) {
  const float2 v = *reinterpret_cast<const float2*>(slot);
  return df{v.x, v.y};
}

// Primitive variables of point p (Sec. 2.1 equation of state): u, v, w, p,
// T = gamma p / rho, H = (e + p)/rho, sqrt(rho).  Returns 1 if non-physical.
// DF (the NS3D_FP64 layout): u, v, w, p in FP64; T, H and sqrt(rho), which are only
// consumed as double-float (Roe average, viscous and statistics kernels), stored as
// double-float pairs and computed on the FP32 pipe; 1/rho from a double-float seed and
// one FP64 Newton step (FP64-accurate: the seed's error squared is ~2^-92).  FP64 work
// per point: 11 instructions instead of ~32 with the IEEE division and square root.
template <bool DF = false>
__device__ __forceinline__ int prim_point(const double* __restrict__ u, double* __restrict__ pm, long long N,
                                          long long p, double gamma) {
  const double rho = u[p], mx = u[N + p], my = u[2 * N + p], mz = u[3 * N + p], e = u[4 * N + p];
  if (DF) {
    const df rd = d2df_bits(rho);
    const df rr = df_div(df{1.0f, 0.0f}, rd);
    double ri = f2d_bits(rr.hi) + f2d_bits(rr.lo);
    ri = fma(ri, fma(-rho, ri, 1.0), ri);
    const double vx = mx * ri, vy = my * ri, vz = mz * ri;
    const double ke2 = fma(mx, vx, fma(my, vy, mz * vz));
    const double pr = (gamma - 1.0) * fma(-0.5, ke2, e);  // = (gamma-1)(e - ke2/2), one rounding as e - ke
    pm[PM_U * N + p] = vx;
    pm[PM_V * N + p] = vy;
    pm[PM_W * N + p] = vz;
    pm[PM_P * N + p] = pr;
    const df dp = d2df_bits(pr);
    store_df(pm + PM_T * N + p, df_mul(df_mul_u(d2df_bits(gamma), dp), rr));
    store_df(pm + PM_H * N + p, df_mul(df_add_fast(d2df_bits(e), dp), rr));
    store_df(pm + PM_SR * N + p, df_sqrt(rd));
    return !pos_finite(rho) | !pos_finite(pr) | !is_finite_bits(e) | !is_finite_bits(mx) | !is_finite_bits(my) |
           !is_finite_bits(mz);
  }
  const double ri = 1.0 / rho;
  const double vx = mx * ri, vy = my * ri, vz = mz * ri;
  const double ke = 0.5 * fma(mx, vx, fma(my, vy, mz * vz));  // explicit: the same bits in every kernel
  const double pr = (gamma - 1.0) * (e - ke);
  pm[PM_U * N + p] = vx;
  pm[PM_V * N + p] = vy;
  pm[PM_W * N + p] = vz;
  pm[PM_P * N + p] = pr;
  pm[PM_T * N + p] = gamma * pr * ri;
  pm[PM_H * N + p] = (e + pr) * ri;
  pm[PM_SR * N + p] = sqrt(rho);
  return !(rho > 0.0) | !isfinite(rho) | !(pr > 0.0) | !isfinite(e) | !isfinite(mx + my + mz);
}

__device__ __forceinline__ long long flat3(int i, int j, int k, int nx, int ny) {
  return ((long long)k * ny + j) * nx + i;
}

// Periodic wrap of c + off for |off| <= 2: two compares instead of a division (any n >= 2),
// the modulo only for a one-point dimension.
__device__ __forceinline__ int wrap_near(int c, int off, int n) {
  if (n < 2) return wrap_idx(c + off, n);
  int r = c + off;
  r = (r < 0) ? r + n : r;
  return (r >= n) ? r - n : r;
}

// 4th-order central first derivative, difference form, times 1/(12 h).  The final product is
// rounded on its own (__dmul_rn) so that no call site can fuse it into a following addition:
// every kernel that evaluates a gradient then produces the same bits.
__device__ __forceinline__ double d4(double qm2, double qm1, double qp1, double qp2, double r12h) {
  return __dmul_rn(fma(8.0, qp1 - qm1, -(qp2 - qm2)), r12h);
}

// d4 in double-float from the four stencil values, already double-float (d2df_bits of
// the FP64 values): the NS3D_FP64 form of the viscous and statistics kernels.
__device__ __forceinline__ df d4_dfv(df qm2, df qm1, df qp1, df qp2, df r12h) {
  const df d1 = df_add_fast(qp1, df_neg(qm1));
  const df d2 = df_add_fast(qp2, df_neg(qm2));
  return df_mul_u(df_add_fast(df_mul_f_u(d1, 8.0f), df_neg(d2)), r12h);
}
__device__ __forceinline__ df d4_df(double qm2, double qm1, double qp1, double qp2, df r12h) {
  return d4_dfv(d2df_bits(qm2), d2df_bits(qm1), d2df_bits(qp1), d2df_bits(qp2), r12h);
}

// Viscous flux vectors at point p from the double-float gradients G[q][d] = d(u,v,w,T)_q/dx_d
// and velocity (Sec. 2.1 stresses with the symmetric strain rate, heat flux q = -kappa grad T),
// stored as double-float pairs (the direction pass of NS3D_FP64 takes their divergence in
// double-float); plane layout as visc_point_ijk.
__device__ __forceinline__ void visc_fluxes_df(const df G[4][3], const df vel[3], double mu, double kappa,
                                               double* __restrict__ fv, long long N, long long p, int only_d) {
  const df dmu = d2df_bits(mu), dkap = d2df_bits(kappa);
  const double two3 = 2.0 / 3.0;
  const df c23{(float)two3, (float)(two3 - (double)(float)two3)};
  const df tdiv = df_mul_u(df_add_fast(G[0][0], df_add_fast(G[1][1], G[2][2])), c23);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (only_d >= 0 && d != only_d) continue;
    const int b = (only_d >= 0) ? 0 : 4 * d;
    df tau[3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
      tau[m] = (m == d) ? df_mul(dmu, df_add_fast(df_twice(G[d][d]), df_neg(tdiv)))
                        : df_mul(dmu, df_add_fast(G[m][d], G[d][m]));
    const df en = df_add_fast(df_add_fast(df_mul_u(vel[0], tau[0]), df_mul_u(vel[1], tau[1])),
                              df_add_fast(df_mul_u(vel[2], tau[2]), df_mul_u(dkap, G[3][d])));
    store_df(fv + (long long)(b + 0) * N + p, tau[0]);
    store_df(fv + (long long)(b + 1) * N + p, tau[1]);
    store_df(fv + (long long)(b + 2) * N + p, tau[2]);
    store_df(fv + (long long)(b + 3) * N + p, en);
  }
}

// Gradients of (u, v, w, T) at point p, then the three viscous flux vectors
// f^v, g^v, h^v (Sec. 2.1 stresses with the symmetric strain rate, heat flux
// q = -kappa grad T), written to fv[(4 d + c) N + p]; with only_d >= 0 just the
// flux along only_d, written to fv[c N + p] (same arithmetic, so the same bits).
template <bool NC = true>
__device__ __forceinline__ void visc_point_ijk(const double* __restrict__ pm, double* __restrict__ fv, int nx, int ny,
                                               int nz, int i, int j, int k, const double r12[3], double mu,
                                               double kappa, int only_d = -1) {
  const long long N = (long long)nx * ny * nz;
  const long long p = flat3(i, j, k, nx, ny);
  double G[4][3];
  const int n3[3] = {nx, ny, nz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long nb[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int off = (o < 2) ? (o - 2) : (o - 1);  // -2, -1, +1, +2
      int c[3] = {i, j, k};
      c[d] = wrap_near(c[d], off, n3[d]);
      nb[o] = flat3(c[0], c[1], c[2], nx, ny);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int plane = (q < 3) ? q : PM_T;
      const double* A = pm + (long long)plane * N;
      G[q][d] = d4(ldx<NC>(A + nb[0]), ldx<NC>(A + nb[1]), ldx<NC>(A + nb[2]), ldx<NC>(A + nb[3]), r12[d]);
    }
  }
  const double vel[3] = {pm[PM_U * N + p], pm[PM_V * N + p], pm[PM_W * N + p]};
  const double tdiv = (2.0 / 3.0) * (G[0][0] + G[1][1] + G[2][2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (only_d >= 0 && d != only_d) continue;
    const int b = (only_d >= 0) ? 0 : 4 * d;
    double tau[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) tau[m] = (m == d) ? mu * fma(2.0, G[d][d], -tdiv) : mu * (G[m][d] + G[d][m]);
    const double en = fma(vel[0], tau[0], fma(vel[1], tau[1], fma(vel[2], tau[2], kappa * G[3][d])));
    fv[(long long)(b + 0) * N + p] = tau[0];
    fv[(long long)(b + 1) * N + p] = tau[1];
    fv[(long long)(b + 2) * N + p] = tau[2];
    fv[(long long)(b + 3) * N + p] = en;
  }
}

// visc_point in the NS3D_FP64 form (primitives in the layout of prim_point<true>: the
// temperature plane holds double-float pairs): the stencil values converted to double-float and
// everything from the differences on (gradients, stresses, heat flux, work term) in
// double-float on the FP32 pipe, with one FP64 addition per output (hi + lo).  The
// viscous fluxes are ~mu |grad u| in size: the double-float rounding of the stencil
// values (2^-48 |u|) gives an error ~mu 2^-48 |u| / dx^2 in the right-hand side, far below
// the FP64 rounding of the convective terms it is added to.
template <bool NC = true>
__device__ __forceinline__ void visc_point_df_ijk(const double* __restrict__ pm, double* __restrict__ fv, int nx,
                                                  int ny, int nz, int i, int j, int k, const double r12[3], double mu,
                                                  double kappa, int only_d = -1) {
  const long long N = (long long)nx * ny * nz;
  const long long p = flat3(i, j, k, nx, ny);
  df G[4][3];
  const int n3[3] = {nx, ny, nz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long nb[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      const int off = (o < 2) ? (o - 2) : (o - 1);  // -2, -1, +1, +2
      int c[3] = {i, j, k};
      c[d] = wrap_near(c[d], off, n3[d]);
      nb[o] = flat3(c[0], c[1], c[2], nx, ny);
    }
    const df r = d2df_bits(r12[d]);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double* A = pm + (long long)q * N;
      G[q][d] = d4_df(ldx<NC>(A + nb[0]), ldx<NC>(A + nb[1]), ldx<NC>(A + nb[2]), ldx<NC>(A + nb[3]), r);
    }
    {  // T: a double-float plane in the NS3D_FP64 layout (prim_point<true>)
      const double* A = pm + (long long)PM_T * N;
      auto t = [&](long long q) {
        const double v = ldx<NC>(A + q);
        return df{__int_as_float(__double2loint(v)), __int_as_float(__double2hiint(v))};
      };
      G[3][d] = d4_dfv(t(nb[0]), t(nb[1]), t(nb[2]), t(nb[3]), r);
    }
  }
  const df vel[3] = {d2df_bits(pm[PM_U * N + p]), d2df_bits(pm[PM_V * N + p]), d2df_bits(pm[PM_W * N + p])};
  visc_fluxes_df(G, vel, mu, kappa, fv, N, p, only_d);
}

// The per-point forms above, addressed by the flat point index p (batched kernels).
template <bool NC = true>
__device__ __forceinline__ void visc_point(const double* __restrict__ pm, double* __restrict__ fv, int nx, int ny,
                                           int nz, long long p, const double r12[3], double mu, double kappa,
                                           int only_d = -1) {
  visc_point_ijk<NC>(pm, fv, nx, ny, nz, (int)(p % nx), (int)((p / nx) % ny), (int)(p / ((long long)nx * ny)), r12,
                     mu, kappa, only_d);
}
template <bool NC = true>
__device__ __forceinline__ void visc_point_df(const double* __restrict__ pm, double* __restrict__ fv, int nx, int ny,
                                              int nz, long long p, const double r12[3], double mu, double kappa,
                                              int only_d = -1) {
  visc_point_df_ijk<NC>(pm, fv, nx, ny, nz, (int)(p % nx), (int)((p / nx) % ny), (int)(p / ((long long)nx * ny)),
                        r12, mu, kappa, only_d);
}

}  // namespace ns3d
