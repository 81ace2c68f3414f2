// Pointwise and stencil-reduction kernels of libns3d.so:
//  - primitive variables (Sec. 2.1 equation of state),
//  - velocity/temperature gradients -> viscous flux vectors f^v, g^v, h^v
//    (Sec. 2.1 stresses and heat flux, 4th-order central differences),
//  - statistics (conservation sums, kinetic energy, enstrophy, extrema, CFL)
//    with a deterministic two-level FP64 reduction (warp shuffles + fixed-order
//    partials).
#include <math.h>

#include "df.cuh"
#include "df2.cuh"
#include "k_point_impl.cuh"
#include "ns3d_internal.cuh"

namespace ns3d {

namespace {

constexpr int PW_THREADS = 256;

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = 152LL * 16;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// Primitive variables of every point (body: prim_point; DF: the NS3D_FP64 layout).
template <bool DF>
__global__ void __launch_bounds__(PW_THREADS) k_prim(const double* __restrict__ u, double* __restrict__ pm,
                                                     long long N, long long p0, long long p1, double gamma,
                                                     int* __restrict__ status) {
  int bad = 0;
  for (long long p = p0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; p < p1; p += (long long)gridDim.x * blockDim.x)
    bad |= prim_point<DF>(u, pm, N, p, gamma);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONPHYS);
}

// Gradients of (u, v, w, T) at every point, then the three viscous flux vectors, all FP64
// (NS3D_FP64_STRICT; body: visc_point_ijk).  The NS3D_FP64 form is k_visc_tiled below.
__global__ void __launch_bounds__(PW_THREADS) k_visc(const double* __restrict__ pm, double* __restrict__ fv,
                                                     int nx, int ny, int nz, double r12hx, double r12hy,
                                                     double r12hz, double mu, double kappa, int only_d, int z0) {
  // one thread per point of a 32 x 8 block of an x-y plane; blockIdx.z = the plane (from z0)
  const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = z0 + blockIdx.z;
  if (i >= nx || j >= ny) return;
  const double r12[3] = {r12hx, r12hy, r12hz};
  visc_point_ijk(pm, fv, nx, ny, nz, i, j, k, r12, mu, kappa, only_d);
}

// Tiled NS3D_FP64 viscous-flux kernel (primitives in the layout of prim_point<true>).  A CTA
// owns a 32 x 8 block of x-y columns and marches along z through VT_CZ planes.  Each plane of
// (u, v, w, T), with a 2-point x-y halo, is converted to double-float once into a ring of 5
// planes (z-2 .. z+2) in shared memory, so every stencil value is converted once rather than
// once per stencil that uses it (12 times).  The ring holds the fields in pairs, (u, v) and
// (w, T), each position a 16-byte record (hi, hi, lo, lo): the 12 gradient stencils run as 6
// two-lane double-float stencils on the packed FP32 instructions (df2.cuh; each lane the
// operations of d4_dfv), the flux assembly reads the lanes as scalars.  The per-point
// arithmetic is that of visc_point_df_ijk: the same conversions, the same gradient and flux
// operations, so the same bits.
constexpr int VT_X = 32, VT_Y = 8, VT_HX = VT_X + 4, VT_HY = VT_Y + 4, VT_PLANE = VT_HX * VT_HY;
constexpr int VT_RING = 5, VT_CZ = VISC_ZCHUNK;
constexpr int VT_SMEM = VT_RING * 2 * VT_PLANE * (int)sizeof(float4);  // 69,120 bytes

// d4_dfv on two lanes.
__device__ __forceinline__ df2 d4_dfv2(df2 qm2, df2 qm1, df2 qp1, df2 qp2, df2 r12h) {
  const df2 d1 = df2_add_fast(qp1, df2_neg(qm1));
  const df2 d2 = df2_add_fast(qp2, df2_neg(qm2));
  return df2_mul_u(df2_add_fast(df2_mul_f_u(d1, 8.0f), df2_neg(d2)), r12h);
}

__global__ void __launch_bounds__(VT_X * VT_Y, 3) k_visc_tiled(const double* __restrict__ pm, double* __restrict__ fv,
                                                                const Grid g, double mu, double kappa, int only_d,
                                                                int zc0) {
  extern __shared__ float4 ring4[];  // [VT_RING][2][VT_HY][VT_HX]: (u, v) and (w, T)
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long N = g.N;
  const int x0 = blockIdx.x * VT_X, y0 = blockIdx.y * VT_Y, z0 = (zc0 + blockIdx.z) * VT_CZ;
  const int z1 = min(z0 + VT_CZ, nz);
  const int tid = threadIdx.x, tx = tid % VT_X, ty = tid / VT_X;
  const df2 r12[3] = {df2_splat(d2df_bits(g.r12h[0])), df2_splat(d2df_bits(g.r12h[1])),
                      df2_splat(d2df_bits(g.r12h[2]))};
  auto slot = [&](int zz) { return ring4 + ((zz - z0 + 2) % VT_RING) * 2 * VT_PLANE; };
  // in-plane offsets of this thread's halo-tile positions (the same for every plane)
  constexpr int NPOS = (VT_PLANE + VT_X * VT_Y - 1) / (VT_X * VT_Y);
  int xy[NPOS];
#pragma unroll
  for (int k = 0; k < NPOS; ++k) {
    const int pos = tid + k * VT_X * VT_Y;
    const int hy = pos / VT_HX, hx = pos - hy * VT_HX;
    xy[k] = wrap_idx(y0 - 2 + hy, ny) * nx + wrap_idx(x0 - 2 + hx, nx);
  }
  const long long plane_n = (long long)nx * ny;
  auto load_plane = [&](int zz) {  // plane zz (periodic) of the four fields, with halo
    const long long zoff = (long long)wrap_idx(zz, nz) * plane_n;
    float4* R = slot(zz);
#pragma unroll
    for (int k = 0; k < NPOS; ++k) {
      const int pos = tid + k * VT_X * VT_Y;
      if (pos >= VT_PLANE) break;
      const long long p = zoff + xy[k];
      const df vu = d2df_bits(__ldg(pm + (long long)PM_U * N + p));
      const df vv = d2df_bits(__ldg(pm + (long long)PM_V * N + p));
      const df vw = d2df_bits(__ldg(pm + (long long)PM_W * N + p));
      const float2 vT = __ldg(reinterpret_cast<const float2*>(pm + (long long)PM_T * N + p));  // double-float plane
      R[pos] = make_float4(vu.hi, vv.hi, vu.lo, vv.lo);
      R[VT_PLANE + pos] = make_float4(vw.hi, vT.x, vw.lo, vT.y);
    }
  };
  auto ld = [](const float4* P, int i) { return df2_from4(P[i]); };
  for (int zz = z0 - 2; zz < z0 + 2; ++zz) load_plane(zz);
  for (int z = z0; z < z1; ++z) {
    load_plane(z + 2);
    __syncthreads();
    if (x0 + tx < nx && y0 + ty < ny) {
      const int c = (ty + 2) * VT_HX + (tx + 2);
      const float4 *Zm2 = slot(z - 2), *Zm1 = slot(z - 1), *Z0 = slot(z), *Zp1 = slot(z + 1), *Zp2 = slot(z + 2);
      // the flux along only_d (lean storage) needs 8 of the 12 gradients: d(u, v, w, T)/dx_d, the
      // derivatives of the velocity component along only_d, and the diagonal (divergence)
      auto need = [&](int q, int e) { return only_d < 0 || e == only_d || (q < 3 && (q == only_d || q == e)); };
      df G[4][3];
#pragma unroll
      for (int k = 0; k < 2; ++k) {  // field pair k: (u, v) or (w, T)
        const float4* P = Z0 + k * VT_PLANE;
        const int o = k * VT_PLANE + c;
        df2 Gk[3];
        const df2 zero{f2splat(0.0f), f2splat(0.0f)};
        Gk[0] = (need(2 * k, 0) || need(2 * k + 1, 0))
                    ? d4_dfv2(ld(P, c - 2), ld(P, c - 1), ld(P, c + 1), ld(P, c + 2), r12[0]) : zero;
        Gk[1] = (need(2 * k, 1) || need(2 * k + 1, 1))
                    ? d4_dfv2(ld(P, c - 2 * VT_HX), ld(P, c - VT_HX), ld(P, c + VT_HX), ld(P, c + 2 * VT_HX), r12[1])
                    : zero;
        Gk[2] = (need(2 * k, 2) || need(2 * k + 1, 2)) ? d4_dfv2(ld(Zm2, o), ld(Zm1, o), ld(Zp1, o), ld(Zp2, o), r12[2])
                                                      : zero;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const df dz{0.0f, 0.0f};
          G[2 * k][e] = need(2 * k, e) ? df2_lane0(Gk[e]) : dz;
          G[2 * k + 1][e] = need(2 * k + 1, e) ? df2_lane1(Gk[e]) : dz;
        }
      }
      const df2 uv = ld(Z0, c), wT = ld(Z0 + VT_PLANE, c);
      const df vel[3] = {df2_lane0(uv), df2_lane1(uv), df2_lane0(wT)};
      visc_fluxes_df(G, vel, mu, kappa, fv, N, flat3(x0 + tx, y0 + ty, z, nx, ny), only_d);
    }
    __syncthreads();  // the slot of plane z - 2 takes plane z + 3 next
  }
}

// Launch geometry of the stencil point kernels: 32 x 8 x 1 blocks over (x, y, z).
inline dim3 plane_grid(const Grid& g) { return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.n[2]); }

// ---- FP32-bulk viscous fluxes (NS3D_FP32_BULK) ---------------------------------------
// The tiled form of k_visc_tiled in FP32, straight from the conserved state: a CTA owns a
// 32 x 8 block of x-y columns and marches along z through VT_CZ planes; every plane of
// (u, v, w, T), with a 2-point x-y halo, is formed once from the state (converted to FP32 by
// bit manipulation) into a ring of 5 planes (z-2 .. z+2) of float4 in shared memory.  Each
// point then takes the 12 gradients with the 4th-order central difference and writes the
// viscous flux vectors as FP32 planes fv[4 d + c][N] (only_d = d: fv[c][N]), which the FP32-bulk
// direction passes read.
__device__ __forceinline__ float d2f_trunc_fast(double x) {
  const uint32_t h = (uint32_t)__double2hiint(x), l = (uint32_t)__double2loint(x);
  const uint32_t e11 = (h >> 20) & 0x7ffu;
  uint32_t b = __funnelshift_l(l, h, 3) + 0x40000000u;
  b = (e11 <= 896u) ? 0u : b;
  b = (e11 >= 1151u) ? 0x7f800000u : b;
  return __uint_as_float(b | (h & 0x80000000u));
}

constexpr int V32_SMEM = VT_RING * VT_PLANE * (int)sizeof(float4);  // 34,560 bytes

__global__ void __launch_bounds__(VT_X * VT_Y, 4) k_visc32t(const double* __restrict__ u, float* __restrict__ fv,
                                                             const Grid g, float gamma, float mu, float kappa,
                                                             int only_d) {
  extern __shared__ float4 ring4[];  // [VT_RING][VT_HY][VT_HX]: u, v, w, T
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long N = g.N;
  const int x0 = blockIdx.x * VT_X, y0 = blockIdx.y * VT_Y, z0 = blockIdx.z * VT_CZ;
  const int z1 = min(z0 + VT_CZ, nz);
  const int tid = threadIdx.x, tx = tid % VT_X, ty = tid / VT_X;
  const float r12[3] = {(float)g.r12h[0], (float)g.r12h[1], (float)g.r12h[2]};
  const float gm1 = gamma - 1.0f;
  auto slot = [&](int zz) { return ring4 + ((zz - z0 + 2) % VT_RING) * VT_PLANE; };
  constexpr int NPOS = (VT_PLANE + VT_X * VT_Y - 1) / (VT_X * VT_Y);
  int xy[NPOS];
#pragma unroll
  for (int k = 0; k < NPOS; ++k) {
    const int pos = tid + k * VT_X * VT_Y;
    const int hy = pos / VT_HX, hx = pos - hy * VT_HX;
    xy[k] = wrap_idx(y0 - 2 + hy, ny) * nx + wrap_idx(x0 - 2 + hx, nx);
  }
  const long long plane_n = (long long)nx * ny;
  auto load_plane = [&](int zz) {
    const long long zoff = (long long)wrap_idx(zz, nz) * plane_n;
    float4* R = slot(zz);
#pragma unroll
    for (int k = 0; k < NPOS; ++k) {
      const int pos = tid + k * VT_X * VT_Y;
      if (pos >= VT_PLANE) break;
      const long long p = zoff + xy[k];
      const float rho = d2f_trunc_fast(__ldg(u + p)), mx = d2f_trunc_fast(__ldg(u + N + p));
      const float my = d2f_trunc_fast(__ldg(u + 2 * N + p)), mz = d2f_trunc_fast(__ldg(u + 3 * N + p));
      const float e = d2f_trunc_fast(__ldg(u + 4 * N + p));
      const float ri = __fdividef(1.0f, rho);
      const float vx = mx * ri, vy = my * ri, vz = mz * ri;
      const float pr = gm1 * fmaf(-0.5f, fmaf(mx, vx, fmaf(my, vy, mz * vz)), e);
      R[pos] = make_float4(vx, vy, vz, gamma * pr * ri);
    }
  };
  for (int zz = z0 - 2; zz < z0 + 2; ++zz) load_plane(zz);
  for (int z = z0; z < z1; ++z) {
    load_plane(z + 2);
    __syncthreads();
    if (x0 + tx < nx && y0 + ty < ny) {
      const int c = (ty + 2) * VT_HX + (tx + 2);
      const float4 *Zm2 = slot(z - 2), *Zm1 = slot(z - 1), *Z0 = slot(z), *Zp1 = slot(z + 1), *Zp2 = slot(z + 2);
      auto d4v = [](float4 m2, float4 m1, float4 p1, float4 p2, float r) {
        return make_float4(fmaf(8.0f, p1.x - m1.x, -(p2.x - m2.x)) * r, fmaf(8.0f, p1.y - m1.y, -(p2.y - m2.y)) * r,
                           fmaf(8.0f, p1.z - m1.z, -(p2.z - m2.z)) * r, fmaf(8.0f, p1.w - m1.w, -(p2.w - m2.w)) * r);
      };
      // G[d] = d(u, v, w, T)/dx_d
      const float4 Gd[3] = {d4v(Z0[c - 2], Z0[c - 1], Z0[c + 1], Z0[c + 2], r12[0]),
                            d4v(Z0[c - 2 * VT_HX], Z0[c - VT_HX], Z0[c + VT_HX], Z0[c + 2 * VT_HX], r12[1]),
                            d4v(Zm2[c], Zm1[c], Zp1[c], Zp2[c], r12[2])};
      float G[4][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        G[0][d] = Gd[d].x;
        G[1][d] = Gd[d].y;
        G[2][d] = Gd[d].z;
        G[3][d] = Gd[d].w;
      }
      const float4 v0 = Z0[c];
      const float vel[3] = {v0.x, v0.y, v0.z};
      const float tdiv = (2.0f / 3.0f) * (G[0][0] + G[1][1] + G[2][2]);
      const long long p = flat3(x0 + tx, y0 + ty, z, nx, ny);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (only_d >= 0 && d != only_d) continue;
        const int b = (only_d >= 0) ? 0 : 4 * d;
        float tau[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) tau[m] = (m == d) ? mu * fmaf(2.0f, G[d][d], -tdiv) : mu * (G[m][d] + G[d][m]);
        const float en = fmaf(vel[0], tau[0], fmaf(vel[1], tau[1], fmaf(vel[2], tau[2], kappa * G[3][d])));
        fv[(long long)(b + 0) * N + p] = tau[0];
        fv[(long long)(b + 1) * N + p] = tau[1];
        fv[(long long)(b + 2) * N + p] = tau[2];
        fv[(long long)(b + 3) * N + p] = en;
      }
    }
    __syncthreads();  // the slot of plane z - 2 takes plane z + 3 next
  }
}

// ---- statistics ------------------------------------------------------------
constexpr int ST_THREADS = 256;
constexpr int ST_MAX_BLOCKS = 4096;
constexpr int NSUM = 7;   // mass, 3 momenta, energy, ke, enstrophy
constexpr int NRED = 10;  // + rho_min, p_min, max wavespeed/dx

struct Red {
  double s[NSUM];
  double rmin, pmin, wmax;
};

__device__ __forceinline__ void red_combine(Red& a, const Red& b) {
#pragma unroll
  for (int m = 0; m < NSUM; ++m) a.s[m] += b.s[m];
  a.rmin = fmin(a.rmin, b.rmin);
  a.pmin = fmin(a.pmin, b.pmin);
  a.wmax = fmax(a.wmax, b.wmax);
}

__device__ __forceinline__ Red warp_reduce(Red r) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Red o;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) o.s[m] = __shfl_down_sync(0xffffffffu, r.s[m], off);
    o.rmin = __shfl_down_sync(0xffffffffu, r.rmin, off);
    o.pmin = __shfl_down_sync(0xffffffffu, r.pmin, off);
    o.wmax = __shfl_down_sync(0xffffffffu, r.wmax, off);
    red_combine(r, o);
  }
  return r;
}

// Fixed-shape block reduction: lane order, then warp order.  Result valid in thread 0.
__device__ Red block_reduce(Red r) {
  __shared__ double sh[ST_THREADS / 32][NRED];
  r = warp_reduce(r);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NSUM; ++m) sh[wid][m] = r.s[m];
    sh[wid][7] = r.rmin;
    sh[wid][8] = r.pmin;
    sh[wid][9] = r.wmax;
  }
  __syncthreads();
  if (wid == 0) {
    Red t;
    if (lane < ST_THREADS / 32) {
#pragma unroll
      for (int m = 0; m < NSUM; ++m) t.s[m] = sh[lane][m];
      t.rmin = sh[lane][7];
      t.pmin = sh[lane][8];
      t.wmax = sh[lane][9];
    } else {
#pragma unroll
      for (int m = 0; m < NSUM; ++m) t.s[m] = 0.0;
      t.rmin = INFINITY;
      t.pmin = INFINITY;
      t.wmax = 0.0;
    }
    r = warp_reduce(t);
  }
  return r;
}

// Statistics: a block walks its tiles of
// 32 x 8 x-y columns times VT_CZ planes in a fixed order; the velocity planes, with a 2-point
// x-y halo, are converted to double-float once into a 5-plane ring (z-2 .. z+2) for the
// vorticity stencils.  The accumulation order is fixed by the grid shape, so the result is
// deterministic.  Sums, minima and counts in FP64; kinetic energy, vorticity, enstrophy and
// wave speed in double-float on the FP32 pipe.  DFT: the temperature plane holds
// double-float pairs (prim_point<true>).
constexpr int SR_SMEM = VT_RING * 3 * VT_PLANE * (int)sizeof(float2);  // 51,840 bytes

template <bool DFT>
__global__ void __launch_bounds__(ST_THREADS, 4) k_stats_tiled(const double* __restrict__ u, const double* __restrict__ pm,
                                                                const Grid g, double* __restrict__ partials, int ntx,
                                                                int nty, long long ntiles) {
  extern __shared__ float2 ring[];  // [VT_RING][3][VT_HY][VT_HX]
  static_assert(VT_X * VT_Y == ST_THREADS, "one point per thread and plane");
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const long long N = g.N;
  const long long plane_n = (long long)nx * ny;
  const df r12d[3] = {d2df_bits(g.r12h[0]), d2df_bits(g.r12h[1]), d2df_bits(g.r12h[2])};
  const df rhd[3] = {d2df_bits(g.rh[0]), d2df_bits(g.rh[1]), d2df_bits(g.rh[2])};
  const int tid = threadIdx.x, tx = tid % VT_X, ty = tid / VT_X;
  constexpr int NPOS = (VT_PLANE + ST_THREADS - 1) / ST_THREADS;
  df wmax{0.0f, 0.0f};
  Red r;
#pragma unroll
  for (int m = 0; m < NSUM; ++m) r.s[m] = 0.0;
  r.rmin = INFINITY;
  r.pmin = INFINITY;
  r.wmax = 0.0;
  auto ld = [](const float2* P, int i) { const float2 v = P[i]; return df{v.x, v.y}; };
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int x0 = (int)(t % ntx) * VT_X;
    const long long rest = t / ntx;
    const int y0 = (int)(rest % nty) * VT_Y, z0 = (int)(rest / nty) * VT_CZ;
    const int z1 = min(z0 + VT_CZ, nz);
    auto slot = [&](int zz) { return ring + ((zz - z0 + 2) % VT_RING) * 3 * VT_PLANE; };
    int xy[NPOS];
#pragma unroll
    for (int k = 0; k < NPOS; ++k) {
      const int pos = tid + k * ST_THREADS;
      const int hy = pos / VT_HX, hx = pos - hy * VT_HX;
      xy[k] = wrap_idx(y0 - 2 + hy, ny) * nx + wrap_idx(x0 - 2 + hx, nx);
    }
    auto load_plane = [&](int zz) {
      const long long zoff = (long long)wrap_idx(zz, nz) * plane_n;
      float2* R = slot(zz);
#pragma unroll
      for (int k = 0; k < NPOS; ++k) {
        const int pos = tid + k * ST_THREADS;
        if (pos >= VT_PLANE) break;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const df v = d2df_bits(__ldg(pm + (long long)q * N + zoff + xy[k]));
          R[q * VT_PLANE + pos] = make_float2(v.hi, v.lo);
        }
      }
    };
    __syncthreads();  // the previous tile's last reads of the ring
    for (int zz = z0 - 2; zz < z0 + 2; ++zz) load_plane(zz);
    for (int z = z0; z < z1; ++z) {
      load_plane(z + 2);
      __syncthreads();
      if (x0 + tx < nx && y0 + ty < ny) {
        const long long p = (long long)z * plane_n + (long long)(y0 + ty) * nx + (x0 + tx);
        const int c = (ty + 2) * VT_HX + (tx + 2);
        const float2 *Zm2 = slot(z - 2), *Zm1 = slot(z - 1), *Z0 = slot(z), *Zp1 = slot(z + 1), *Zp2 = slot(z + 2);
        const double rho = __ldg(u + p);
        const double pr = __ldg(pm + PM_P * N + p);
        r.s[0] += rho;
        r.s[1] += __ldg(u + N + p);
        r.s[2] += __ldg(u + 2 * N + p);
        r.s[3] += __ldg(u + 3 * N + p);
        r.s[4] += __ldg(u + 4 * N + p);
        const df rd = d2df_bits(rho);
        const df rh2{0.5f * rd.hi, 0.5f * rd.lo};  // rho / 2, exact
        const df vd[3] = {ld(Z0, c), ld(Z0 + VT_PLANE, c), ld(Z0 + 2 * VT_PLANE, c)};
        const df ke = df_mul_u(rh2, df_add_pos_u(df_sqr_u(vd[0]), df_add_pos_u(df_sqr_u(vd[1]), df_sqr_u(vd[2]))));
        r.s[5] = (r.s[5] + f2d_bits(ke.hi)) + f2d_bits(ke.lo);
        // vorticity: dv_m/dx_d for m != d
        auto gx = [&](int m) {
          const float2* P = Z0 + m * VT_PLANE;
          return d4_dfv(ld(P, c - 2), ld(P, c - 1), ld(P, c + 1), ld(P, c + 2), r12d[0]);
        };
        auto gy = [&](int m) {
          const float2* P = Z0 + m * VT_PLANE;
          return d4_dfv(ld(P, c - 2 * VT_HX), ld(P, c - VT_HX), ld(P, c + VT_HX), ld(P, c + 2 * VT_HX), r12d[1]);
        };
        auto gz = [&](int m) {
          const int o = m * VT_PLANE + c;
          return d4_dfv(ld(Zm2, o), ld(Zm1, o), ld(Zp1, o), ld(Zp2, o), r12d[2]);
        };
        const df wx = df_add_fast(gy(2), df_neg(gz(1)));
        const df wy = df_add_fast(gz(0), df_neg(gx(2)));
        const df wz = df_add_fast(gx(1), df_neg(gy(0)));
        const df en = df_mul_u(rh2, df_add_pos_u(df_sqr_u(wx), df_add_pos_u(df_sqr_u(wy), df_sqr_u(wz))));
        r.s[6] = (r.s[6] + f2d_bits(en.hi)) + f2d_bits(en.lo);
        r.rmin = fmin(r.rmin, rho);
        r.pmin = fmin(r.pmin, pr);
        const df cs = df_sqrt(DFT ? load_df(pm + PM_T * N + p) : d2df_bits(__ldg(pm + PM_T * N + p)));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const df w = df_mul(df_add_pos(df_abs(vd[d]), cs), rhd[d]);
          if (df_lt(wmax, w)) wmax = w;
        }
      }
      __syncthreads();  // the slot of plane z - 2 takes plane z + 3 next
    }
  }
  r.wmax = f2d_bits(wmax.hi) + f2d_bits(wmax.lo);
  r = block_reduce(r);
  if (threadIdx.x == 0) {
    double* o = partials + (long long)blockIdx.x * NRED;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) o[m] = r.s[m];
    o[7] = r.rmin;
    o[8] = r.pmin;
    o[9] = r.wmax;
  }
}

__global__ void __launch_bounds__(ST_THREADS) k_stats_final(const double* __restrict__ partials, int nblocks,
                                                            const int* __restrict__ status, double vol,
                                                            double inv_n, double* __restrict__ out) {
  Red r;
#pragma unroll
  for (int m = 0; m < NSUM; ++m) r.s[m] = 0.0;
  r.rmin = INFINITY;
  r.pmin = INFINITY;
  r.wmax = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double* q = partials + (long long)b * NRED;
    Red t;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) t.s[m] = q[m];
    t.rmin = q[7];
    t.pmin = q[8];
    t.wmax = q[9];
    red_combine(r, t);
  }
  r = block_reduce(r);
  if (threadIdx.x == 0) {
    for (int m = 0; m < 5; ++m) out[m] = r.s[m] * vol;
    out[5] = r.s[5] * inv_n;
    out[6] = r.s[6] * inv_n;
    out[7] = r.rmin;
    out[8] = r.pmin;
    out[9] = r.wmax;
    out[10] = (double)(*status);
    out[11] = 0.0;
  }
}

}  // namespace

cudaError_t launch_prim(const Grid& g, const double* u, double* pm, double gamma, int* status, cudaStream_t s,
                        int df, long long p0, long long p1) {
  if (p1 < 0) p1 = g.N;
  if (p0 < 0 || p1 > g.N || p0 >= p1) return p0 == p1 ? cudaSuccess : cudaErrorInvalidValue;
  const int grid = grid_for(p1 - p0, PW_THREADS);
  if (df)
    k_prim<true><<<grid, PW_THREADS, 0, s>>>(u, pm, g.N, p0, p1, gamma, status);
  else
    k_prim<false><<<grid, PW_THREADS, 0, s>>>(u, pm, g.N, p0, p1, gamma, status);
  return cudaGetLastError();
}

cudaError_t launch_visc(const Grid& g, const double* pm, double* fv, double mu, double kappa, cudaStream_t s,
                        int only_d, int df, int z0, int z1) {
  const double rx = g.r12h[0], ry = g.r12h[1], rz = g.r12h[2];
  const int nz = g.n[2];
  if (z1 < 0) z1 = nz;
  if (z0 < 0 || z1 > nz || z0 > z1) return cudaErrorInvalidValue;
  if (z0 == z1) return cudaSuccess;
  if (df) {
    if (z0 % VT_CZ != 0 || (z1 % VT_CZ != 0 && z1 != nz)) return cudaErrorInvalidValue;
    const int zc0 = z0 / VT_CZ, zc1 = (z1 + VT_CZ - 1) / VT_CZ;
    const dim3 grid((g.n[0] + VT_X - 1) / VT_X, (g.n[1] + VT_Y - 1) / VT_Y, zc1 - zc0);
    k_visc_tiled<<<grid, VT_X * VT_Y, VT_SMEM, s>>>(pm, fv, g, mu, kappa, only_d, zc0);
  } else {
    dim3 grid = plane_grid(g);
    grid.z = z1 - z0;
    k_visc<<<grid, PW_THREADS, 0, s>>>(pm, fv, g.n[0], g.n[1], nz, rx, ry, rz, mu, kappa, only_d, z0);
  }
  return cudaGetLastError();
}

cudaError_t prepare_visc_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_visc_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, VT_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stats_tiled<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SR_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stats_tiled<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SR_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_visc32t, cudaFuncAttributeMaxDynamicSharedMemorySize, V32_SMEM);
  return e;
}

cudaError_t launch_visc32(const Grid& g, const double* u, float* fv, double gamma, double mu, double kappa,
                          cudaStream_t s, int only_d) {
  const dim3 grid((g.n[0] + VT_X - 1) / VT_X, (g.n[1] + VT_Y - 1) / VT_Y, (g.n[2] + VT_CZ - 1) / VT_CZ);
  k_visc32t<<<grid, VT_X * VT_Y, V32_SMEM, s>>>(u, fv, g, (float)gamma, (float)mu, (float)kappa, only_d);
  return cudaGetLastError();
}

int stats_num_blocks(const Grid& g) {
  long long b = (g.N + ST_THREADS - 1) / ST_THREADS;
  return (int)(b < ST_MAX_BLOCKS ? (b > 0 ? b : 1) : ST_MAX_BLOCKS);
}

cudaError_t launch_stats(const Grid& g, const double* u, const double* pm, double gamma, double* partials,
                         cudaStream_t s, int df) {
  (void)gamma;
  const int ntx = (g.n[0] + VT_X - 1) / VT_X, nty = (g.n[1] + VT_Y - 1) / VT_Y, ntz = (g.n[2] + VT_CZ - 1) / VT_CZ;
  const long long ntiles = (long long)ntx * nty * ntz;
  // exactly stats_num_blocks(g) blocks: the partials k_stats_final reduces (blocks without a
  // tile write neutral partials)
  if (df)
    k_stats_tiled<true><<<stats_num_blocks(g), ST_THREADS, SR_SMEM, s>>>(u, pm, g, partials, ntx, nty, ntiles);
  else
    k_stats_tiled<false><<<stats_num_blocks(g), ST_THREADS, SR_SMEM, s>>>(u, pm, g, partials, ntx, nty, ntiles);
  return cudaGetLastError();
}

cudaError_t launch_stats_final(const Grid& g, const double* partials, int nblocks, const int* status, double* out,
                               cudaStream_t s) {
  k_stats_final<<<1, ST_THREADS, 0, s>>>(partials, nblocks, status, g.h[0] * g.h[1] * g.h[2], 1.0 / (double)g.N,
                                         out);
  return cudaGetLastError();
}

}  // namespace ns3d
