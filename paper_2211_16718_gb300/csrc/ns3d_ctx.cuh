// Host-side context of libns3d.so (the opaque ns3d_ctx of include/ns3d.h) and the
// helpers shared by the translation units that implement its calls.
#pragma once

#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "ns3d_internal.cuh"

struct TimedLaunch {
  int kid;
  cudaEvent_t e0, e1;
};

struct ns3d_ctx {
  ns3d_params p;
  ns3d::Grid g;
  cudaStream_t stream;
  int device;
  double* pm = nullptr;        // [NPRIM][N]
  double* fv = nullptr;        // [NVISC][N] (viscous only)
  double* k = nullptr;         // [5][N] RHS accumulator
  double* ua = nullptr;        // [5][N] stage state
  double* ub = nullptr;        // [5][N] stage state
  double* acc = nullptr;       // [5][N] RK4 accumulator
  double* partials = nullptr;  // [stats blocks][10]
  double* stats_dev = nullptr; // [NS3D_STATS_NDOUBLE]
  int* status = nullptr;       // sticky status word
  double* uhost_dev = nullptr; // device state for ns3d_step_host (lazy)
  // ns3d_step_host: a stream for the host<->device copies of z-slabs, overlapped with the kernels,
  // and the events that order them (lazy): [0, MAX) slabs in, [MAX, 2 MAX) slabs out, [2 MAX] entry
  static constexpr int MAX_SLABS = 16;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t slab_ev[2 * MAX_SLABS + 1] = {};
  double* stats_host = nullptr;// pinned [NS3D_STATS_NDOUBLE]
  int nstat_blocks = 0;
  int variant = 0;             // tile-shape variant of the direction passes
  int zorder = -1;             // CTA order of the z pass (DirArgs::zorder); -1: dir_zorder by grid size
  int lean = 0;                // viscous fluxes one direction at a time ([4][N] instead of [12][N])
  size_t bytes = 0;            // library-owned device bytes
  // adjoint (allocated on first use): RK stage states, incoming adjoint copy,
  // two stage-adjoint buffers, viscous-adjoint scratch [16][N]
  double* adj = nullptr;
  // trajectory checkpoints (allocated by ns3d_traj_forward)
  double* ckpt = nullptr;      // [nckpt][5][N] states at steps 0, every, 2 every, ...
  double* seg = nullptr;       // [every][5][N] recomputed states of one segment
  int ckpt_cap = 0, seg_cap = 0;
  int traj_nsteps = -1, traj_every = 0;
  double traj_dt = 0.0;
  char err[512] = {0};
  // timing
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> pool;
  double ms[NS3D_K_COUNT] = {0};
  long long launches[NS3D_K_COUNT] = {0};
};

namespace ns3d {

inline int set_err(ns3d_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

inline int cuda_fail(ns3d_ctx* c, cudaError_t e, const char* what) {
  return set_err(c, NS3D_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

inline cudaEvent_t pool_get(ns3d_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch wrapper: records events around the launch when timing is on.
template <typename F>
int timed(ns3d_ctx* c, int kid, F&& fn, const char* what) {
  TimedLaunch t{kid, nullptr, nullptr};
  if (c->timing) {
    t.e0 = pool_get(c);
    t.e1 = pool_get(c);
    cudaEventRecord(t.e0, c->stream);
  }
  cudaError_t e = fn();
  if (c->timing) {
    cudaEventRecord(t.e1, c->stream);
    c->pending.push_back(t);
  }
  c->launches[kid] += 1;
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return NS3D_OK;
}

// cudaMalloc counted in c->bytes; false (and a cleared CUDA error) if it fails.
inline bool dev_alloc(ns3d_ctx* c, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  c->bytes += bytes;
  return true;
}

// Allocate the Runge-Kutta stage states (and the RK4 accumulator) on first use (ns3d_api.cu).
int ensure_stage_buffers(ns3d_ctx* c);
// z-slabs of a state moving between host and device while the kernels run (ns3d_step_host):
// slab j is [lo[j], lo[j+1]) in planes (copies in) or in tiles of the z pass (copies out).
struct SlabPipe {
  int n = 0;
  int lo[ns3d_ctx::MAX_SLABS + 1] = {};
  cudaEvent_t* ev = nullptr;  // ev[j]: slab j is on the device (in) / final on the device (out)
  double* host = nullptr;     // out: destination of the slabs ([5][N] like the device state)
  int tp = 0;                 // out: points along z of a z-pass tile
};
// One right-hand-side evaluation of u with the given z-pass epilogue (ns3d_api.cu).  pin: u arrives
// slab by slab (the primitive, viscous, x and y kernels run per slab after its event); pout: the z
// pass runs per slab of tiles, each followed by the copy of that slab of out to pout->host on
// c->copy_stream.
int rhs_pass(ns3d_ctx* c, const double* u, int epi, double* out, const double* un, double coef,
             const SlabPipe* pin = nullptr, const SlabPipe* pout = nullptr);
// Statistics of u into out_dev[NS3D_STATS_NDOUBLE] (ns3d_api.cu).
int stats_pass(ns3d_ctx* c, const double* u, double* out_dev);
// One Runge-Kutta step of u in place (ns3d_api.cu); pin / pout as for rhs_pass, applied to the
// first / last stage.
int rk_one_step(ns3d_ctx* c, double* u, double dt, const SlabPipe* pin = nullptr, const SlabPipe* pout = nullptr);
// Release the adjoint and trajectory buffers (ns3d_adjoint.cu).
void adjoint_free(ns3d_ctx* c);

}  // namespace ns3d
