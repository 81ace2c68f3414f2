// Arithmetic-throughput probe of the current device (measurement support for
// the roofline of the FP64-bound right-hand side; no counterpart in the paper).
// Register-only kernels with 8 independent dependency chains per thread; every
// thread writes one double so that nothing is optimised away.
#include "ns3d_internal.cuh"

namespace ns3d {

namespace {

constexpr int PILP = 8;
constexpr int PTHREADS = 256;

template <int OP>
__global__ void __launch_bounds__(PTHREADS) k_probe64(double* out, int iters, double a, double b) {
  double x[PILP];
#pragma unroll
  for (int i = 0; i < PILP; ++i) x[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PILP; ++i) {
      if (OP == 0) x[i] = fma(x[i], a, b);
      else if (OP == 1) x[i] = x[i] + a;
      else if (OP == 2) x[i] = b / x[i];
      else x[i] = sqrt(x[i] + a);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < PILP; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PTHREADS) k_probe32(double* out, int iters, float a, float b) {
  float x[PILP];
#pragma unroll
  for (int i = 0; i < PILP; ++i) x[i] = 1.0f + 1e-3f * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < PILP; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PILP; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int alu_probe(double res[5]) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NS3D_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NS3D_ECUDA;
  const int blocks = sms * 8;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * PTHREADS) != cudaSuccess) return NS3D_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters[5] = {2000, 2000, 200, 200, 100000};
  int rc = NS3D_OK;
  for (int op = 0; op < 5 && rc == NS3D_OK; ++op) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, 0);
      switch (op) {
        case 0: k_probe64<0><<<blocks, PTHREADS>>>(out, iters[op], 0.999999, 1e-7); break;
        case 1: k_probe64<1><<<blocks, PTHREADS>>>(out, iters[op], 1e-9, 0.0); break;
        case 2: k_probe64<2><<<blocks, PTHREADS>>>(out, iters[op], 0.0, 1.0000001); break;
        case 3: k_probe64<3><<<blocks, PTHREADS>>>(out, iters[op], 1e-9, 0.0); break;
        default: k_probe32<<<blocks, PTHREADS>>>(out, iters[op], 0.999999f, 1e-7f); break;
      }
      cudaEventRecord(e1, 0);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        rc = NS3D_ECUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    res[op] = (double)blocks * PTHREADS * iters[op] * PILP / (best * 1e-3) * 1e-9;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace ns3d
