// Statistics of a caller-owned state without any device allocation.
//
// Some callers cannot let a library allocate device memory: a host code that
// owns all GPU memory through its own pool and budget (cudaMalloc/cudaFree
// would bypass that pool, can fail under memory pressure and synchronise the
// whole device), or an in-situ monitoring hook that runs inside another
// solver's time loop and must not perturb its memory footprint or timing.
// ns3d_stats needs a context, and creating one allocates tens of doubles per
// grid point of scratch.  ns3d_stats_noalloc gives those callers the same
// statistics from a fused variant of the statistics kernels whose only scratch
// (the per-block partial sums) lives in a fixed-size file-scope __device__
// array, loaded with the library and held by every GPU that loads it until the
// process exits.
#include <math.h>

#include <mutex>

#include "ns3d_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;   // partial-sum slots: 1024 x 12 doubles = 96 KB per device
constexpr int NA_SLOT = 12;           // 7 sums, rho_min, p_min, max wave speed/dx, status, unused
constexpr int NA_MAX_DEVICES = 64;
constexpr int NSUM = 7;

// Partial reductions of the most recent call on this device.  Every block of a
// call overwrites its own slot before the final kernel reads it, so nothing has
// to start at zero; concurrent calls on one device race on these slots.
static __device__ __align__(256) double g_stats_partials[NA_MAX_BLOCKS * NA_SLOT];

std::mutex g_setup_mutex;
double* g_partials_addr[NA_MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double d4na(double qm2, double qm1, double qp1, double qp2, double r12h) {
  return fma(8.0, qp1 - qm1, -(qp2 - qm2)) * r12h;
}

// Velocity component m (0..2) at flat point q, from the conserved state.
__device__ __forceinline__ double vel_at(const double* __restrict__ u, long long N, long long q, int m) {
  const double ri = 1.0 / __ldg(u + q);
  return __ldg(u + (long long)(1 + m) * N + q) * ri;
}

struct RedNA {
  double s[NSUM];
  double rmin, pmin, wmax, bad;
};

__device__ __forceinline__ void na_combine(RedNA& a, const RedNA& b) {
#pragma unroll
  for (int m = 0; m < NSUM; ++m) a.s[m] += b.s[m];
  a.rmin = fmin(a.rmin, b.rmin);
  a.pmin = fmin(a.pmin, b.pmin);
  a.wmax = fmax(a.wmax, b.wmax);
  a.bad = fmax(a.bad, b.bad);
}

__device__ __forceinline__ RedNA na_warp(RedNA r) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    RedNA o;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) o.s[m] = __shfl_down_sync(0xffffffffu, r.s[m], off);
    o.rmin = __shfl_down_sync(0xffffffffu, r.rmin, off);
    o.pmin = __shfl_down_sync(0xffffffffu, r.pmin, off);
    o.wmax = __shfl_down_sync(0xffffffffu, r.wmax, off);
    o.bad = __shfl_down_sync(0xffffffffu, r.bad, off);
    na_combine(r, o);
  }
  return r;
}

__device__ RedNA na_block(RedNA r) {
  __shared__ double sh[NA_THREADS / 32][NA_SLOT];
  r = na_warp(r);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NSUM; ++m) sh[wid][m] = r.s[m];
    sh[wid][7] = r.rmin;
    sh[wid][8] = r.pmin;
    sh[wid][9] = r.wmax;
    sh[wid][10] = r.bad;
  }
  __syncthreads();
  if (wid == 0) {
    RedNA t;
    if (lane < NA_THREADS / 32) {
#pragma unroll
      for (int m = 0; m < NSUM; ++m) t.s[m] = sh[lane][m];
      t.rmin = sh[lane][7];
      t.pmin = sh[lane][8];
      t.wmax = sh[lane][9];
      t.bad = sh[lane][10];
    } else {
#pragma unroll
      for (int m = 0; m < NSUM; ++m) t.s[m] = 0.0;
      t.rmin = INFINITY;
      t.pmin = INFINITY;
      t.wmax = 0.0;
      t.bad = 0.0;
    }
    r = na_warp(t);
  }
  return r;
}

__device__ __forceinline__ RedNA na_identity() {
  RedNA r;
#pragma unroll
  for (int m = 0; m < NSUM; ++m) r.s[m] = 0.0;
  r.rmin = INFINITY;
  r.pmin = INFINITY;
  r.wmax = 0.0;
  r.bad = 0.0;
  return r;
}

// Fused variant of the primitive + statistics kernels: primitives are computed on
// the fly from the conserved state (also at the vorticity stencil neighbours).
__global__ void __launch_bounds__(NA_THREADS) k_stats_noalloc(const double* __restrict__ u, int nx, int ny, int nz,
                                                              double hx, double hy, double hz, double gamma,
                                                              double* __restrict__ partials) {
  const long long N = (long long)nx * ny * nz;
  const int n3[3] = {nx, ny, nz};
  const double r12[3] = {1.0 / (12.0 * hx), 1.0 / (12.0 * hy), 1.0 / (12.0 * hz)};
  const double rh[3] = {1.0 / hx, 1.0 / hy, 1.0 / hz};
  RedNA r = na_identity();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / ((long long)nx * ny));
    const double rho = u[p], mx = u[N + p], my = u[2 * N + p], mz = u[3 * N + p], e = u[4 * N + p];
    const double ri = 1.0 / rho;
    const double vel[3] = {mx * ri, my * ri, mz * ri};
    const double pr = (gamma - 1.0) * (e - 0.5 * (mx * vel[0] + my * vel[1] + mz * vel[2]));
    r.s[0] += rho;
    r.s[1] += mx;
    r.s[2] += my;
    r.s[3] += mz;
    r.s[4] += e;
    r.s[5] += 0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    double G[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      long long nb[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int off = (o < 2) ? (o - 2) : (o - 1);
        int c[3] = {i, j, k};
        c[d] = ns3d::wrap_idx(c[d] + off, n3[d]);
        nb[o] = ((long long)c[2] * ny + c[1]) * nx + c[0];
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (m == d) continue;
        G[m][d] = d4na(vel_at(u, N, nb[0], m), vel_at(u, N, nb[1], m), vel_at(u, N, nb[2], m),
                       vel_at(u, N, nb[3], m), r12[d]);
      }
    }
    const double wx = G[2][1] - G[1][2], wy = G[0][2] - G[2][0], wz = G[1][0] - G[0][1];
    r.s[6] += 0.5 * rho * (wx * wx + wy * wy + wz * wz);
    r.rmin = fmin(r.rmin, rho);
    r.pmin = fmin(r.pmin, pr);
    const double c = sqrt(gamma * pr * ri);
#pragma unroll
    for (int d = 0; d < 3; ++d) r.wmax = fmax(r.wmax, (fabs(vel[d]) + c) * rh[d]);
    if (!(rho > 0.0) || !isfinite(rho) || !(pr > 0.0) || !isfinite(e) || !isfinite(mx + my + mz)) r.bad = 1.0;
  }
  r = na_block(r);
  if (threadIdx.x == 0) {
    double* o = partials + (long long)blockIdx.x * NA_SLOT;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) o[m] = r.s[m];
    o[7] = r.rmin;
    o[8] = r.pmin;
    o[9] = r.wmax;
    o[10] = r.bad;
    o[11] = 0.0;
  }
}

__global__ void __launch_bounds__(NA_THREADS) k_stats_noalloc_final(const double* __restrict__ partials, int nblocks,
                                                                    double vol, double inv_n,
                                                                    double* __restrict__ out) {
  RedNA r = na_identity();
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double* q = partials + (long long)b * NA_SLOT;
    RedNA t;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) t.s[m] = q[m];
    t.rmin = q[7];
    t.pmin = q[8];
    t.wmax = q[9];
    t.bad = q[10];
    na_combine(r, t);
  }
  r = na_block(r);
  if (threadIdx.x == 0) {
    for (int m = 0; m < 5; ++m) out[m] = r.s[m] * vol;
    out[5] = r.s[5] * inv_n;
    out[6] = r.s[6] * inv_n;
    out[7] = r.rmin;
    out[8] = r.pmin;
    out[9] = r.wmax;
    out[10] = r.bad;
    out[11] = 0.0;
  }
}

// Device address of the partials array for the current device, looked up once
// per device (with that device current) and cached.
int partials_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NS3D_ECUDA;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return NS3D_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_partials_addr[dev] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_stats_partials);
    if (e != cudaSuccess || ptr == nullptr) return NS3D_ECUDA;
    g_partials_addr[dev] = (double*)ptr;
  }
  *out = g_partials_addr[dev];
  return NS3D_OK;
}

}  // namespace

extern "C" int ns3d_stats_noalloc(const ns3d_params* p, const double* u_dev, double* out_dev, void* cuda_stream) {
  if (!p || !u_dev || !out_dev) return NS3D_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NS3D_EINVAL;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (1LL << 32)) return NS3D_EINVAL;  // beyond the largest grid this call supports
  if (!(p->lx > 0) || !(p->ly > 0) || !(p->lz > 0) || !isfinite(p->lx) || !isfinite(p->ly) || !isfinite(p->lz))
    return NS3D_EINVAL;
  if (!(p->gamma > 1.0) || !isfinite(p->gamma)) return NS3D_EINVAL;
  long long nb = (N + NA_THREADS - 1) / NA_THREADS;
  const int nblocks = (int)(nb < NA_MAX_BLOCKS ? nb : NA_MAX_BLOCKS);  // grid-stride beyond the slot count
  if (nblocks > NA_MAX_BLOCKS) return NS3D_EINVAL;
  double* partials = nullptr;
  int rc = partials_address(&partials);
  if (rc != NS3D_OK) return rc;
  const double hx = p->lx / p->nx, hy = p->ly / p->ny, hz = p->lz / p->nz;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_stats_noalloc<<<nblocks, NA_THREADS, 0, s>>>(u_dev, p->nx, p->ny, p->nz, hx, hy, hz, p->gamma, partials);
  if (cudaGetLastError() != cudaSuccess) return NS3D_ECUDA;
  k_stats_noalloc_final<<<1, NA_THREADS, 0, s>>>(partials, nblocks, hx * hy * hz, 1.0 / (double)N, out_dev);
  if (cudaGetLastError() != cudaSuccess) return NS3D_ECUDA;
  return NS3D_OK;
}
