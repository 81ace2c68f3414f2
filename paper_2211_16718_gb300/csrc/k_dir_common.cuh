// Pieces shared by the direction passes (k_dir.cu: FP64 modes, k_dir32.cu:
// FP32-bulk mode): tile indexing and the accumulation / Runge-Kutta epilogue.
#pragma once

#include "ns3d_internal.cuh"

namespace ns3d {

// Shared-memory index of (position along the pencil, line) in a tile of W lines:
// position-major for y/z lines (consecutive threads = consecutive x lines),
// line-major for x lines (consecutive threads = consecutive x points).
template <int D, int W>
__device__ __forceinline__ int tile_idx(int pos, int line, int npos) {
  return D == 0 ? line * npos + pos : pos * W + line;
}
template <int D, int W>
__device__ __forceinline__ void tile_split(int item, int npos, int& pos, int& line) {
  if (D == 0) {
    pos = item % npos;
    line = item / npos;
  } else {
    line = item % W;
    pos = item / W;
  }
}

// Flat grid index of pencil coordinate c on line la of the tile row bz.
template <int D>
__device__ __forceinline__ long long tile_flat(const Grid& g, int c, int la, int bz) {
  constexpr int AX = (D == 0) ? 1 : 0;
  constexpr int BX = (D == 2) ? 1 : 2;
  int idx[3];
  idx[D] = c;
  idx[AX] = la;
  idx[BX] = bz;
  return ((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0];
}

// Accumulate this direction's contribution cv[5] at point p, or finish the RHS /
// RK stage (last direction), according to a.epi.
__device__ __forceinline__ void dir_epilogue(const DirArgs& a, long long p, const double cv[5]) {
  const long long N = a.g.N;
  switch (a.epi) {
    case EPI_ACC_WRITE:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] = cv[v];
      break;
    case EPI_ACC_ADD:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] += cv[v];
      break;
    case EPI_RHS_OUT:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.out[v * N + p] = a.k[v * N + p] + cv[v];
      break;
    case EPI_RK4_FIRST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        a.out[v * N + p] = fma(a.a, K, a.un[v * N + p]);
        a.acc[v * N + p] = K;
      }
      break;
    case EPI_RK4_MID:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        a.out[v * N + p] = fma(a.a, K, a.un[v * N + p]);
        a.acc[v * N + p] = fma(2.0, K, a.acc[v * N + p]);
      }
      break;
    case EPI_RK4_LAST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        a.out[v * N + p] = fma(a.a, a.acc[v * N + p] + K, a.un[v * N + p]);
      }
      break;
    case EPI_SSP_1:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        a.out[v * N + p] = fma(a.a, K, a.un[v * N + p]);
      }
      break;
    case EPI_SSP_2:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        a.out[v * N + p] = 0.75 * a.un[v * N + p] + 0.25 * fma(a.a, K, a.u[v * N + p]);
      }
      break;
    case EPI_SSP_3:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        a.out[v * N + p] = (1.0 / 3.0) * a.un[v * N + p] + (2.0 / 3.0) * fma(a.a, K, a.u[v * N + p]);
      }
      break;
    default:
      break;
  }
}

// Number of FP64 operands per point the epilogue reads (k, then U_n, then acc or the stage input).
__host__ __device__ __forceinline__ int epilogue_operands(int epi) {
  switch (epi) {
    case EPI_ACC_WRITE: return 0;
    case EPI_ACC_ADD:
    case EPI_RHS_OUT: return 5;
    case EPI_RK4_FIRST:
    case EPI_SSP_1: return 10;
    default: return 15;
  }
}

// Asynchronous 8-byte global -> shared copy (cp.async, cached at all levels).
__device__ __forceinline__ void cp_async8(double* dst_smem, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Start fetching the epilogue operands of point p into pre[0 .. epilogue_operands(a.epi)).
__device__ __forceinline__ void epilogue_prefetch(const DirArgs& a, long long p, double* pre) {
  const long long N = a.g.N;
  const int n = epilogue_operands(a.epi);
  if (n == 0) return;
#pragma unroll
  for (int v = 0; v < 5; ++v) cp_async8(pre + v, a.k + v * N + p);
  if (n >= 10) {
#pragma unroll
    for (int v = 0; v < 5; ++v) cp_async8(pre + 5 + v, a.un + v * N + p);
  }
  if (n == 15) {
    const double* third = (a.epi == EPI_SSP_2 || a.epi == EPI_SSP_3) ? a.u : a.acc;
#pragma unroll
    for (int v = 0; v < 5; ++v) cp_async8(pre + 10 + v, third + v * N + p);
  }
}

// dir_epilogue with the operands read from pre (filled by epilogue_prefetch) instead of
// global memory; the same arithmetic, so the same bits.
__device__ __forceinline__ void dir_epilogue_pre(const DirArgs& a, long long p, const double cv[5],
                                                 const double* pre) {
  const long long N = a.g.N;
  switch (a.epi) {
    case EPI_ACC_WRITE:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] = cv[v];
      break;
    case EPI_ACC_ADD:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] = pre[v] + cv[v];
      break;
    case EPI_RHS_OUT:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.out[v * N + p] = pre[v] + cv[v];
      break;
    case EPI_RK4_FIRST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = pre[v] + cv[v];
        a.out[v * N + p] = fma(a.a, K, pre[5 + v]);
        a.acc[v * N + p] = K;
      }
      break;
    case EPI_RK4_MID:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = pre[v] + cv[v];
        a.out[v * N + p] = fma(a.a, K, pre[5 + v]);
        a.acc[v * N + p] = fma(2.0, K, pre[10 + v]);
      }
      break;
    case EPI_RK4_LAST:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = pre[v] + cv[v];
        a.out[v * N + p] = fma(a.a, pre[10 + v] + K, pre[5 + v]);
      }
      break;
    case EPI_SSP_1:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = pre[v] + cv[v];
        a.out[v * N + p] = fma(a.a, K, pre[5 + v]);
      }
      break;
    case EPI_SSP_2:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = pre[v] + cv[v];
        a.out[v * N + p] = 0.75 * pre[5 + v] + 0.25 * fma(a.a, K, pre[10 + v]);
      }
      break;
    case EPI_SSP_3:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = pre[v] + cv[v];
        a.out[v * N + p] = (1.0 / 3.0) * pre[5 + v] + (2.0 / 3.0) * fma(a.a, K, pre[10 + v]);
      }
      break;
    default:
      break;
  }
}

}  // namespace ns3d
