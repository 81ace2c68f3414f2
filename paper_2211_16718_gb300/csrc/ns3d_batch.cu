// Batched ensembles of independent grids of uneven sizes (e.g. many turbulence
// realisations), advanced together.  Three schedules of the same arithmetic
// (bitwise identical results):
//   SEQUENTIAL  every instance with its own launches (5 per RK stage per instance),
//               one instance after the other on the caller's stream;
//   GRAPH       the same per-instance launches for one step, captured once in a CUDA
//               graph whose parallel branches each advance a share of the instances
//               (balanced by points), so that small instances run beside large ones
//               instead of behind them; the graph is replayed once per step;
//   PERSISTENT  one cooperative kernel for all steps, stages, phases and
//               instances over a flattened (instance, tile) work list; phases are
//               separated by grid-wide barriers (cooperative groups), so co-residency
//               of all CTAs is guaranteed by the cooperative launch and there is no
//               hand-written spin-wait.
// ns3d_batch_autotune picks, per grid size present in the ensemble, the tile shape of
// the direction passes (timing every candidate on that size's instances), and the
// number of graph branches, and caches both in a JSON-lines file keyed by device and
// size (or ensemble).
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "k_dir_impl.cuh"
#include "k_point_impl.cuh"
#include "ns3d_internal.cuh"

namespace cg = cooperative_groups;
using namespace ns3d;

namespace {

constexpr int MAX_STAGES = 4;
constexpr int BT = 256;  // threads of the pointwise batched kernels

struct Inst {
  Grid g;
  int variant;                    // tile shape of this instance's direction passes (SEQUENTIAL, GRAPH)
  double gamma, mu, kappa;
  double r12[3];
  const double* uin[MAX_STAGES];  // stage input states
  double* pm;
  double* fv;                     // nullptr if inviscid
  DirArgs dir[MAX_STAGES][3];
  int ntile[3][2];                // tiles along the pencil, along the lines (per direction)
};

struct BatchView {
  int count, nstages;
  int df;                     // viscous fluxes in the NS3D_FP64 form (precision NS3D_FP64)
  const Inst* inst;
  const long long* pt_off;    // [count + 1] prefix sums of points
  const long long* tile_off;  // [3][count + 1] prefix sums of tiles per direction
  int* status;
};

// Largest i with off[i] <= x (off[0] = 0 <= x < off[count]).
__device__ __forceinline__ int find_inst(const long long* off, int count, long long x) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void phase_prim(const BatchView& b, int s, long long t0, long long stride, int& bad) {
  const long long tot = b.pt_off[b.count];
  for (long long x = t0; x < tot; x += stride) {
    const int i = find_inst(b.pt_off, b.count, x);
    const Inst& in = b.inst[i];
    bad |= b.df ? prim_point<true>(in.uin[s], in.pm, in.g.N, x - b.pt_off[i], in.gamma)
                : prim_point<false>(in.uin[s], in.pm, in.g.N, x - b.pt_off[i], in.gamma);
  }
}

template <bool NC>
__device__ __forceinline__ void phase_visc(const BatchView& b, long long t0, long long stride) {
  const long long tot = b.pt_off[b.count];
  for (long long x = t0; x < tot; x += stride) {
    const int i = find_inst(b.pt_off, b.count, x);
    const Inst& in = b.inst[i];
    if (in.fv == nullptr) continue;
    if (b.df) visc_point_df<NC>(in.pm, in.fv, in.g.n[0], in.g.n[1], in.g.n[2], x - b.pt_off[i], in.r12, in.mu, in.kappa);
    else visc_point<NC>(in.pm, in.fv, in.g.n[0], in.g.n[1], in.g.n[2], x - b.pt_off[i], in.r12, in.mu, in.kappa);
  }
}

template <int D, int MODE, int TP, int W, bool NC>
__device__ __forceinline__ void phase_dir(const BatchView& b, int s, double* sm, long long t0, long long stride) {
  const long long* off = b.tile_off + D * (b.count + 1);
  const long long tot = off[b.count];
  for (long long t = t0; t < tot; t += stride) {
    const int i = find_inst(off, b.count, t);
    const Inst& in = b.inst[i];
    const long long lt = t - off[i];
    const int ntx = in.ntile[D][0], nty = in.ntile[D][1];
    const int tx = (int)(lt % ntx);
    const long long r = lt / ntx;
    const int ty = (int)(r % nty);
    const int tz = (int)(r / nty);
    dir_tile<D, MODE, TP, W, NC>(in.dir[s][D], sm, tx, ty, tz);
    __syncthreads();  // the next tile reuses the shared memory
  }
}

// ---- persistent kernel: every step, stage, phase and instance in one launch ---------
template <int MODE, int TP, int W>
__global__ void __launch_bounds__(Plan<MODE, TP, W>::THREADS, Plan<MODE, TP, W>::MIN_CTAS) kb_persistent(BatchView b,
                                                                                           int nsteps) {
  extern __shared__ __align__(16) double sm[];
  cg::grid_group grid = cg::this_grid();
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int bad = 0;
  for (int step = 0; step < nsteps; ++step) {
    for (int s = 0; s < b.nstages; ++s) {
      phase_prim(b, s, t0, stride, bad);
      grid.sync();
      phase_visc<false>(b, t0, stride);
      grid.sync();
      phase_dir<0, MODE, TP, W, false>(b, s, sm, blockIdx.x, gridDim.x);
      grid.sync();
      phase_dir<1, MODE, TP, W, false>(b, s, sm, blockIdx.x, gridDim.x);
      grid.sync();
      phase_dir<2, MODE, TP, W, false>(b, s, sm, blockIdx.x, gridDim.x);
      grid.sync();
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(b.status, ST_NONPHYS);
}

template <int MODE, int TP, int W>
struct Kernels {
  // dynamic shared memory of the tile plan and the largest carveout (Plan::MIN_CTAS per SM)
  template <typename K>
  static cudaError_t attr(K* kernel, int bytes) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
  }
  static cudaError_t set_attr() { return attr(kb_persistent<MODE, TP, W>, Plan<MODE, TP, W>::BYTES); }
  static cudaError_t persistent(const BatchView& v, int nsteps, int ctas_per_sm, int sms, cudaStream_t st) {
    const int bytes = Plan<MODE, TP, W>::BYTES, th = Plan<MODE, TP, W>::THREADS;
    BatchView vv = v;
    int ns = nsteps;
    void* args[] = {&vv, &ns};
    return cudaLaunchCooperativeKernel((const void*)kb_persistent<MODE, TP, W>, dim3(ctas_per_sm * sms), dim3(th),
                                       args, bytes, st);
  }
  static int max_ctas_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kb_persistent<MODE, TP, W>, Plan<MODE, TP, W>::THREADS,
                                                      Plan<MODE, TP, W>::BYTES) != cudaSuccess)
      return 0;
    return n;
  }
};

// Dispatch on (mode, variant) to the template instantiation.
template <typename F>
cudaError_t with_kernels(int mode, int variant, F&& f) {
  if (mode == 0) return f(Kernels<0, 32, 4>());
  if (variant == 1) return f(Kernels<1, 16, 4>());
  if (variant == 2) return f(Kernels<1, 40, 2>());
  return f(Kernels<1, 24, 4>());
}

std::mutex g_attr_mutex;
bool g_attr_done[64] = {false};

cudaError_t prepare_batch_kernels() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  if (dev >= 0 && dev < 64 && g_attr_done[dev]) return cudaSuccess;
  cudaError_t e = Kernels<0, 32, 4>::set_attr();
  if (e == cudaSuccess) e = Kernels<1, 24, 4>::set_attr();
  if (e == cudaSuccess) e = Kernels<1, 16, 4>::set_attr();
  if (e == cudaSuccess) e = Kernels<1, 40, 2>::set_attr();
  if (e == cudaSuccess) e = prepare_dir_kernels();
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_attr_done[dev] = true;
  return e;
}

}  // namespace

struct ns3d_batch {
  static constexpr int MAX_BRANCHES = 8;
  int count = 0;
  std::vector<ns3d_params> p;
  cudaStream_t stream = nullptr;      // caller's stream: every launch runs here
  cudaStream_t cap_stream = nullptr;  // private stream that graph captures record on
  cudaStream_t branch[MAX_BRANCHES] = {};  // captured branches of the GRAPH schedule
  cudaEvent_t fork = nullptr, join[MAX_BRANCHES] = {};
  int branches = 4;                   // parallel branches of the GRAPH schedule
  int mode = 1, variant = 0, nstages = 4, sms = 0;  // variant: tile shape of the PERSISTENT kernel
  std::vector<int> ivar;              // per-instance tile shape (SEQUENTIAL, GRAPH)
  std::vector<Inst> inst;
  std::vector<double*> bufs;  // per-instance scratch allocations
  std::vector<double*> u;
  std::vector<double> dt;
  std::vector<long long> pt_off, tile_off;
  Inst* d_inst = nullptr;
  long long* d_pt_off = nullptr;
  long long* d_tile_off = nullptr;
  int* d_status = nullptr;
  double* partials = nullptr;
  double* d_stats = nullptr;  // [count][NS3D_STATS_NDOUBLE] (ns3d_batch_set_dt_from_cfl)
  int nstat_blocks = 0;
  bool ready = false;
  cudaGraphExec_t gexec = nullptr;  // one step of the GRAPH schedule
  cudaGraphExec_t pexec = nullptr;
  int p_nsteps = -1;
  int persistent_graph = -1;  // 1: captured in a graph, 0: direct cooperative launch, -1: not yet
  int pers_ctas = 0;
  char err[256] = {0};
};

namespace {

int berr(ns3d_batch* b, int code, const char* msg) {
  if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
  return code;
}

void drop_graphs(ns3d_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->pexec) cudaGraphExecDestroy(b->pexec);
  b->gexec = nullptr;
  b->pexec = nullptr;
  b->p_nsteps = -1;
}

BatchView view_of(const ns3d_batch* b) {
  BatchView v;
  v.count = b->count;
  v.nstages = b->nstages;
  v.df = (b->mode == 1) ? 1 : 0;
  v.inst = b->d_inst;
  v.pt_off = b->d_pt_off;
  v.tile_off = b->d_tile_off;
  v.status = b->d_status;
  return v;
}

// Fill the per-instance launch descriptors for the current states, dt and variant
// and upload them.
int rebuild(ns3d_batch* b) {
  if (b->u.empty() || b->dt.empty()) return NS3D_OK;
  int tp = 0, w = 0;
  dir_tile_shape(b->mode, b->variant, &tp, &w);  // the persistent kernel's tile list
  b->tile_off.assign(3 * (b->count + 1), 0);
  for (int i = 0; i < b->count; ++i) {
    Inst& in = b->inst[i];
    in.variant = (b->mode == 1) ? b->ivar[i] : 0;
    double* u = b->u[i];
    double* ua = b->bufs[6 * i + 2];
    double* ub = b->bufs[6 * i + 3];
    double* acc = b->bufs[6 * i + 4];
    double* k = b->bufs[6 * i + 5];
    const double dt = b->dt[i];
    const double* uin4[4] = {u, ua, ub, ua};
    double* out4[4] = {ua, ub, ua, u};
    const int epi4[4] = {EPI_RK4_FIRST, EPI_RK4_MID, EPI_RK4_MID, EPI_RK4_LAST};
    const double coef4[4] = {0.5 * dt, 0.5 * dt, dt, dt / 6.0};
    const double* uin3[3] = {u, ua, ub};
    double* out3[3] = {ua, ub, u};
    const int epi3[3] = {EPI_SSP_1, EPI_SSP_2, EPI_SSP_3};
    for (int s = 0; s < b->nstages; ++s) {
      in.uin[s] = (b->nstages == 4) ? uin4[s] : uin3[s];
      for (int d = 0; d < 3; ++d) {
        DirArgs& a = in.dir[s][d];
        memset(&a, 0, sizeof(a));
        a.g = in.g;
        a.u = in.uin[s];
        a.pm = in.pm;
        a.fv = in.fv;
        a.fv_dstride = 4;
        a.k = k;
        a.acc = acc;
        a.gamma = in.gamma;
        a.eps4 = 4.0 * b->p[i].weno_eps;
        a.hdelta = b->p[i].harten_delta;
        a.status = b->d_status;
        a.mode = b->mode;
        a.variant = in.variant;
        const double c133 = 13.0 / 3.0, eps4 = 4.0 * b->p[i].weno_eps;
        a.c133_hi = (float)c133;
        a.c133_lo = (float)(c133 - (double)a.c133_hi);
        a.eps4_hi = (float)eps4;
        a.eps4_lo = (float)(eps4 - (double)a.eps4_hi);
        const double gm1 = in.gamma - 1.0, hd = b->p[i].harten_delta;
        a.gm1_hi = (float)gm1;
        a.gm1_lo = (float)(gm1 - (double)a.gm1_hi);
        a.hd_hi = (float)hd;
        a.hd_lo = (float)(hd - (double)a.hd_hi);
        if (d == 0) {
          a.epi = EPI_ACC_WRITE;
        } else if (d == 1) {
          a.epi = EPI_ACC_ADD;
        } else {
          a.epi = (b->nstages == 4) ? epi4[s] : epi3[s];
          a.out = (b->nstages == 4) ? out4[s] : out3[s];
          a.un = u;
          a.a = (b->nstages == 4) ? coef4[s] : dt;
        }
      }
    }
    for (int d = 0; d < 3; ++d) {
      const int ax = (d == 0) ? 1 : 0, bx = (d == 2) ? 1 : 2;
      in.ntile[d][0] = (in.g.n[d] + tp - 1) / tp;
      in.ntile[d][1] = (in.g.n[ax] + w - 1) / w;
      const long long tiles = (long long)in.ntile[d][0] * in.ntile[d][1] * in.g.n[bx];
      b->tile_off[d * (b->count + 1) + i + 1] = b->tile_off[d * (b->count + 1) + i] + tiles;
    }
  }
  cudaError_t e = cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(Inst) * b->count, cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_tile_off, b->tile_off.data(), sizeof(long long) * b->tile_off.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  drop_graphs(b);
  b->ready = true;
  return NS3D_OK;
}

// One RK step of instance i with its own launches on stream st.
cudaError_t step_instance(const ns3d_batch* b, int i, cudaStream_t st) {
  const Inst& in = b->inst[i];
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < b->nstages && e == cudaSuccess; ++s) {
    e = launch_prim(in.g, in.uin[s], in.pm, in.gamma, b->d_status, st, b->mode);
    if (e == cudaSuccess && in.fv) e = launch_visc(in.g, in.pm, in.fv, in.mu, in.kappa, st, -1, b->mode);
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = launch_dir(d, in.dir[s][d], st);
  }
  return e;
}

// One step of the instances in `which` (all if empty), one after the other on the caller's stream.
int step_sequential(ns3d_batch* b, const std::vector<int>& which = {}) {
  const int n = which.empty() ? b->count : (int)which.size();
  for (int k = 0; k < n; ++k) {
    const cudaError_t e = step_instance(b, which.empty() ? k : which[k], b->stream);
    if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  }
  return NS3D_OK;
}

// Instances of each GRAPH branch: largest first, each to the branch with the fewest points so
// far (longest-processing-time rule; work per point is the same for every instance).
std::vector<std::vector<int>> branch_lists(const ns3d_batch* b, int nb) {
  std::vector<int> order(b->count);
  for (int i = 0; i < b->count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->inst[x].g.N > b->inst[y].g.N; });
  std::vector<std::vector<int>> lists(nb);
  std::vector<long long> load(nb, 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lists[k].push_back(i);
    load[k] += b->inst[i].g.N;
  }
  return lists;
}

// Capture one step of every instance (per-instance launches in parallel branches) and
// instantiate it.
int capture_graph(ns3d_batch* b) {
  const int nb = std::max(1, std::min(b->branches, std::min(b->count, (int)ns3d_batch::MAX_BRANCHES)));
  const std::vector<std::vector<int>> lists = branch_lists(b, nb);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  cudaError_t eq = cudaEventRecord(b->fork, b->cap_stream);
  for (int k = 0; k < nb && eq == cudaSuccess; ++k) {
    eq = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
    for (size_t j = 0; j < lists[k].size() && eq == cudaSuccess; ++j) eq = step_instance(b, lists[k][j], b->branch[k]);
    if (eq == cudaSuccess) eq = cudaEventRecord(b->join[k], b->branch[k]);
    if (eq == cudaSuccess) eq = cudaStreamWaitEvent(b->cap_stream, b->join[k], 0);
  }
  e = cudaStreamEndCapture(b->cap_stream, &g);
  if (eq != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return berr(b, NS3D_ECUDA, cudaGetErrorString(eq != cudaSuccess ? eq : e));
  }
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->gexec = nullptr;
    return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  }
  return NS3D_OK;
}

int step_graph(ns3d_batch* b, int nsteps) {
  if (!b->gexec) {
    const int rc = capture_graph(b);
    if (rc) return rc;
  }
  for (int s = 0; s < nsteps; ++s) {
    const cudaError_t e = cudaGraphLaunch(b->gexec, b->stream);
    if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  }
  return NS3D_OK;
}

int step_persistent(ns3d_batch* b, int nsteps) {
  if (b->pers_ctas <= 0) {
    if (b->mode == 0) b->pers_ctas = Kernels<0, 32, 4>::max_ctas_per_sm();
    else if (b->variant == 1) b->pers_ctas = Kernels<1, 16, 4>::max_ctas_per_sm();
    else if (b->variant == 2) b->pers_ctas = Kernels<1, 40, 2>::max_ctas_per_sm();
    else b->pers_ctas = Kernels<1, 24, 4>::max_ctas_per_sm();
    if (b->pers_ctas <= 0) return berr(b, NS3D_ECUDA, "persistent kernel does not fit on an SM");
  }
  const BatchView v = view_of(b);
  // Try once to capture the cooperative launch in a graph; fall back to a direct launch.
  if (b->persistent_graph != 0 && (!b->pexec || b->p_nsteps != nsteps)) {
    if (b->pexec) cudaGraphExecDestroy(b->pexec);
    b->pexec = nullptr;
    cudaGraph_t g = nullptr;
    bool ok = (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess);
    cudaError_t el = cudaSuccess;
    if (ok) el = with_kernels(b->mode, b->variant, [&](auto K) {
      return decltype(K)::persistent(v, nsteps, b->pers_ctas, b->sms, b->cap_stream);
    });
    cudaError_t ee = ok ? cudaStreamEndCapture(b->cap_stream, &g) : cudaErrorUnknown;
    ok = ok && el == cudaSuccess && ee == cudaSuccess && g != nullptr &&
         cudaGraphInstantiate(&b->pexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // clear any capture error
    b->persistent_graph = ok ? 1 : 0;
    if (ok) b->p_nsteps = nsteps;
  }
  cudaError_t e;
  if (b->persistent_graph == 1) {
    e = cudaGraphLaunch(b->pexec, b->stream);
  } else {
    e = with_kernels(b->mode, b->variant, [&](auto K) {
      return decltype(K)::persistent(v, nsteps, b->pers_ctas, b->sms, b->stream);
    });
  }
  if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  return NS3D_OK;
}

std::string device_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  return prop.name;
}

std::string params_key(const ns3d_params& p) {
  return std::to_string(p.nx) + "x" + std::to_string(p.ny) + "x" + std::to_string(p.nz) + ((p.mu_eff > 0.0) ? "v" : "e");
}

std::string key_prefix(const ns3d_batch* b) {
  return device_name() + "|batch|mode" + std::to_string(b->mode) + "|stages" + std::to_string(b->nstages) + "|";
}

// Cache key of the tile shape of one grid size.
std::string size_key(const ns3d_batch* b, int i) { return key_prefix(b) + "size|" + params_key(b->p[i]); }

// Cache key of the branch count of the whole ensemble.
std::string ensemble_key(const ns3d_batch* b) {
  std::string k = key_prefix(b) + "branches|";
  for (int i = 0; i < b->count; ++i) {
    k += params_key(b->p[i]);
    if (i + 1 < b->count) k += ",";
  }
  return k;
}

// Look the key up in a JSON-lines cache ({"key": "...", "<field>": N, ...} per line); the last
// matching line wins, -1 if none.
int cache_lookup(const char* path, const std::string& key, const char* field) {
  if (!path) return -1;
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  const std::string needle = "\"key\": \"" + key + "\",";
  const std::string fneedle = std::string("\"") + field + "\": ";
  std::vector<char> line(1 << 17);
  int found = -1;
  while (fgets(line.data(), (int)line.size(), f)) {
    if (strstr(line.data(), needle.c_str())) {
      const char* v = strstr(line.data(), fneedle.c_str());
      if (v) found = atoi(v + fneedle.size());
    }
  }
  fclose(f);
  return found;
}

void cache_append(const char* path, const std::string& key, const char* field, int value, const double* ms, int nms) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"%s\": %d, \"ms_per_step\": [", key.c_str(), field, value);
  for (int k = 0; k < nms; ++k) fprintf(f, "%s%.4f", k ? ", " : "", ms[k]);
  fprintf(f, "]}\n");
  fclose(f);
}

// Time one step of fn() on b->stream (after one untimed warm-up step); -1 on failure.
template <typename F>
double time_step(ns3d_batch* b, F&& fn) {
  if (fn() != NS3D_OK) return -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
  float t = -1.f;
  cudaEventRecord(e0, b->stream);
  const int rc = fn();
  cudaEventRecord(e1, b->stream);
  if (rc != NS3D_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
    t = -1.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return t;
}

}  // namespace

extern "C" {

int ns3d_batch_init(const ns3d_params* params, int count, void* cuda_stream, ns3d_batch** out) {
  if (!out || !params || count < 1 || count > 4096) return NS3D_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    const ns3d_params& p = params[i];
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (long long)p.nx * p.ny * p.nz > (1LL << 31)) return NS3D_EINVAL;
    if (p.nx > 65535 * 2 || p.ny > 65535 || p.nz > 65535) return NS3D_EINVAL;
    if (!(p.lx > 0) || !(p.ly > 0) || !(p.lz > 0) || !(p.gamma > 1.0) || !(p.mu_eff >= 0.0)) return NS3D_EINVAL;
    if (p.mu_eff > 0.0 && !(p.prandtl > 0.0)) return NS3D_EINVAL;
    if (!(p.weno_eps >= 1e-15) || p.weno_p != 2 || !(p.harten_delta >= 0.0)) return NS3D_EINVAL;
    if (p.precision != params[0].precision || p.rk != params[0].rk) return NS3D_EINVAL;
  }
  if (params[0].precision != NS3D_FP64 && params[0].precision != NS3D_FP64_STRICT) return NS3D_EINVAL;
  if (params[0].rk != NS3D_RK4 && params[0].rk != NS3D_SSPRK3) return NS3D_EINVAL;
  ns3d_batch* b = new ns3d_batch();
  b->count = count;
  b->p.assign(params, params + count);
  b->stream = (cudaStream_t)cuda_stream;
  b->mode = (params[0].precision == NS3D_FP64_STRICT) ? 0 : 1;
  b->nstages = (params[0].rk == NS3D_RK4) ? 4 : 3;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  bool sok = prepare_batch_kernels() == cudaSuccess &&
             cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < ns3d_batch::MAX_BRANCHES && sok; ++k)
    sok = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking) == cudaSuccess &&
          cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!sok) {
    cudaGetLastError();
    ns3d_batch_free(b);
    return NS3D_ECUDA;
  }
  b->ivar.assign(count, 0);
  b->inst.resize(count);
  b->pt_off.assign(count + 1, 0);
  long long maxN = 0;
  for (int i = 0; i < count; ++i) {
    const ns3d_params& p = params[i];
    Inst& in = b->inst[i];
    memset(&in, 0, sizeof(in));
    in.g.n[0] = p.nx;
    in.g.n[1] = p.ny;
    in.g.n[2] = p.nz;
    in.g.N = (long long)p.nx * p.ny * p.nz;
    grid_set_spacing(in.g, p.lx, p.ly, p.lz);
    in.gamma = p.gamma;
    in.mu = p.mu_eff;
    in.kappa = (p.mu_eff > 0.0) ? p.mu_eff / ((p.gamma - 1.0) * p.prandtl) : 0.0;
    for (int d = 0; d < 3; ++d) in.r12[d] = 1.0 / (12.0 * in.g.h[d]);
    b->pt_off[i + 1] = b->pt_off[i] + in.g.N;
    if (in.g.N > maxN) maxN = in.g.N;
    // scratch: primitives, viscous fluxes, two stage states, RK accumulator, RHS accumulator
    const size_t sizes[6] = {7, 12, 5, 5, 5, 5};
    for (int a = 0; a < 6; ++a) {
      double* ptr = nullptr;
      if (a == 1 && p.mu_eff == 0.0) {
        b->bufs.push_back(nullptr);
        continue;
      }
      if (cudaMalloc(&ptr, sizeof(double) * sizes[a] * (size_t)in.g.N) != cudaSuccess) {
        cudaGetLastError();
        ns3d_batch_free(b);
        return NS3D_ENOMEM;
      }
      b->bufs.push_back(ptr);
    }
    in.pm = b->bufs[6 * i + 0];
    in.fv = b->bufs[6 * i + 1];
  }
  Grid gmax;
  gmax.N = maxN;
  b->nstat_blocks = stats_num_blocks(gmax);
  bool ok = cudaMalloc(&b->d_inst, sizeof(Inst) * count) == cudaSuccess &&
            cudaMalloc(&b->d_pt_off, sizeof(long long) * (count + 1)) == cudaSuccess &&
            cudaMalloc(&b->d_tile_off, sizeof(long long) * 3 * (count + 1)) == cudaSuccess &&
            cudaMalloc(&b->d_status, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->partials, sizeof(double) * 16 * (size_t)b->nstat_blocks) == cudaSuccess &&
            cudaMalloc(&b->d_stats, sizeof(double) * NS3D_STATS_NDOUBLE * (size_t)count) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ns3d_batch_free(b);
    return NS3D_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_pt_off, b->pt_off.data(), sizeof(long long) * (count + 1),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    ns3d_batch_free(b);
    return NS3D_ECUDA;
  }
  *out = b;
  return NS3D_OK;
}

void ns3d_batch_free(ns3d_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (double* p : b->bufs) cudaFree(p);
  cudaFree(b->d_inst);
  cudaFree(b->d_pt_off);
  cudaFree(b->d_tile_off);
  cudaFree(b->d_status);
  cudaFree(b->partials);
  cudaFree(b->d_stats);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (int k = 0; k < ns3d_batch::MAX_BRANCHES; ++k) {
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

int ns3d_batch_set_states(ns3d_batch* b, double* const* u_dev) {
  if (!b || !u_dev) return NS3D_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (!u_dev[i]) return berr(b, NS3D_EINVAL, "null state pointer");
  b->u.assign(u_dev, u_dev + b->count);
  return rebuild(b);
}

int ns3d_batch_set_dt(ns3d_batch* b, const double* dt) {
  if (!b || !dt) return NS3D_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (!isfinite(dt[i])) return berr(b, NS3D_EINVAL, "dt must be finite");
  b->dt.assign(dt, dt + b->count);
  return rebuild(b);
}

int ns3d_batch_set_variant(ns3d_batch* b, int variant) {
  if (!b || variant < 0 || variant >= DIR_VARIANTS) return NS3D_EINVAL;
  if (b->mode == 0 && variant != 0) return NS3D_EINVAL;
  b->variant = variant;
  b->ivar.assign(b->count, variant);
  b->pers_ctas = 0;
  b->persistent_graph = -1;
  drop_graphs(b);
  return rebuild(b);
}

int ns3d_batch_set_instance_variant(ns3d_batch* b, int i, int variant) {
  if (!b || i < 0 || i >= b->count || variant < 0 || variant >= DIR_VARIANTS) return NS3D_EINVAL;
  if (b->mode == 0 && variant != 0) return NS3D_EINVAL;
  b->ivar[i] = variant;
  drop_graphs(b);
  return rebuild(b);
}

int ns3d_batch_set_branches(ns3d_batch* b, int branches) {
  if (!b || branches < 1 || branches > ns3d_batch::MAX_BRANCHES) return NS3D_EINVAL;
  b->branches = branches;
  drop_graphs(b);
  return NS3D_OK;
}

int ns3d_batch_step(ns3d_batch* b, int nsteps, int schedule) {
  if (!b || nsteps < 0) return NS3D_EINVAL;
  if (!b->ready) return berr(b, NS3D_EINVAL, "set states and dt first");
  if (nsteps == 0) return NS3D_OK;
  if (schedule == NS3D_BATCH_SEQUENTIAL) {
    for (int s = 0; s < nsteps; ++s) {
      int rc = step_sequential(b);
      if (rc) return rc;
    }
    return NS3D_OK;
  }
  if (schedule == NS3D_BATCH_GRAPH) return step_graph(b, nsteps);
  if (schedule == NS3D_BATCH_PERSISTENT) return step_persistent(b, nsteps);
  return berr(b, NS3D_EINVAL, "unknown schedule");
}

int ns3d_batch_stats(ns3d_batch* b, double* out_dev) {
  if (!b || !out_dev) return NS3D_EINVAL;
  if (b->u.empty()) return berr(b, NS3D_EINVAL, "set states first");
  for (int i = 0; i < b->count; ++i) {
    const Inst& in = b->inst[i];
    cudaError_t e = launch_prim(in.g, b->u[i], in.pm, in.gamma, b->d_status, b->stream, b->mode);
    if (e == cudaSuccess) e = launch_stats(in.g, b->u[i], in.pm, in.gamma, b->partials, b->stream, b->mode);
    if (e == cudaSuccess)
      e = launch_stats_final(in.g, b->partials, stats_num_blocks(in.g), b->d_status,
                             out_dev + (size_t)i * NS3D_STATS_NDOUBLE, b->stream);
    if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  }
  return NS3D_OK;
}

int ns3d_batch_set_dt_from_cfl(ns3d_batch* b, double cfl, double* dt_out) {
  if (!b) return NS3D_EINVAL;
  if (!(cfl > 0.0) || !isfinite(cfl)) return berr(b, NS3D_EINVAL, "cfl must be finite and > 0");
  if (b->u.empty()) return berr(b, NS3D_EINVAL, "set states first");
  int rc = ns3d_batch_stats(b, b->d_stats);
  if (rc) return rc;
  std::vector<double> st((size_t)b->count * NS3D_STATS_NDOUBLE);
  cudaError_t e = cudaMemcpyAsync(st.data(), b->d_stats, sizeof(double) * st.size(), cudaMemcpyDeviceToHost,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  std::vector<double> dt(b->count);
  for (int i = 0; i < b->count; ++i) {
    const double w = st[(size_t)i * NS3D_STATS_NDOUBLE + 9];
    if (!(w > 0.0) || !isfinite(w)) return berr(b, NS3D_ENONPHYSICAL, "an instance has no finite positive wave speed");
    dt[i] = cfl / w;
  }
  rc = ns3d_batch_set_dt(b, dt.data());
  if (rc == NS3D_OK && dt_out) memcpy(dt_out, dt.data(), sizeof(double) * b->count);
  return rc;
}

int ns3d_batch_check(ns3d_batch* b) {
  if (!b) return NS3D_EINVAL;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return berr(b, NS3D_ECUDA, cudaGetErrorString(e));
  if (h & ST_NONPHYS) return NS3D_ENONPHYSICAL;
  if (h & ST_DF_RANGE) return NS3D_ERANGE;
  return NS3D_OK;
}

int ns3d_batch_autotune(ns3d_batch* b, const char* cache_path, double* ms_out) {
  if (!b) return NS3D_EINVAL;
  if (!b->ready) return berr(b, NS3D_EINVAL, "set states and dt first");
  if (ms_out)
    for (int k = 0; k < DIR_VARIANTS * b->count + ns3d_batch::MAX_BRANCHES; ++k) ms_out[k] = -1.0;
  // size classes: instances with the same grid (and viscous or not)
  std::vector<std::string> cls(b->count);
  std::vector<std::string> names;
  std::vector<std::vector<int>> members;
  for (int i = 0; i < b->count; ++i) {
    cls[i] = size_key(b, i);
    const size_t c = std::find(names.begin(), names.end(), cls[i]) - names.begin();
    if (c == names.size()) {
      names.push_back(cls[i]);
      members.emplace_back();
    }
    members[c].push_back(i);
  }
  std::vector<int> pending;  // classes that need timing
  for (size_t c = 0; c < names.size(); ++c) {
    const int v = (b->mode == 1) ? cache_lookup(cache_path, names[c], "variant") : 0;  // strict: one shape
    if (v >= 0 && v < DIR_VARIANTS) {
      for (int i : members[c]) b->ivar[i] = v;
    } else {
      pending.push_back((int)c);
    }
  }
  const std::string ekey = ensemble_key(b);
  const int cached_branches = cache_lookup(cache_path, ekey, "branches");
  if (pending.empty() && cached_branches >= 1 && cached_branches <= ns3d_batch::MAX_BRANCHES) {
    b->branches = cached_branches;
    drop_graphs(b);
    return rebuild(b);
  }
  // time the candidates on copies of the states (the caller's states are not advanced)
  std::vector<double*> saved = b->u, tmp(b->count, nullptr);
  int rc = NS3D_OK;
  for (int i = 0; i < b->count && rc == NS3D_OK; ++i) {
    const size_t bytes = sizeof(double) * 5 * (size_t)b->inst[i].g.N;
    if (cudaMalloc(&tmp[i], bytes) != cudaSuccess) {
      cudaGetLastError();
      rc = berr(b, NS3D_ENOMEM, "autotuner state copies");
    } else if (cudaMemcpyAsync(tmp[i], saved[i], bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess) {
      rc = berr(b, NS3D_ECUDA, "autotuner state copies");
    }
  }
  if (rc == NS3D_OK) {
    b->u = tmp;
    // tile shape per size class: one sequential step of the class's instances per candidate
    for (int c : pending) {
      double ms[DIR_VARIANTS];
      int best = 0;
      for (int v = 0; v < DIR_VARIANTS; ++v) {
        ms[v] = -1.0;
        if (b->mode == 0 && v > 0) continue;
        for (int i : members[c]) b->ivar[i] = v;
        if ((rc = rebuild(b)) != NS3D_OK) break;
        ms[v] = time_step(b, [&] { return step_sequential(b, members[c]); });
        if (ms[v] < 0) {
          rc = berr(b, NS3D_ECUDA, "autotuner timing");
          break;
        }
        if (ms[v] < ms[best]) best = v;
      }
      if (rc != NS3D_OK) break;
      for (int i : members[c]) {
        b->ivar[i] = best;
        if (ms_out)
          for (int v = 0; v < DIR_VARIANTS; ++v) ms_out[i * DIR_VARIANTS + v] = ms[v];
      }
      if (b->mode == 1) cache_append(cache_path, names[c], "variant", best, ms, DIR_VARIANTS);
    }
    // graph branches for the chosen shapes: one graph-scheduled step per candidate count
    if (rc == NS3D_OK && (rc = rebuild(b)) == NS3D_OK) {
      if (cached_branches >= 1 && cached_branches <= ns3d_batch::MAX_BRANCHES) {
        b->branches = cached_branches;
      } else {
        double ms[ns3d_batch::MAX_BRANCHES];
        int best = 1;
        for (int nb = 1; nb <= ns3d_batch::MAX_BRANCHES; ++nb) ms[nb - 1] = -1.0;
        for (int nb = 1; nb <= std::min(b->count, (int)ns3d_batch::MAX_BRANCHES); nb *= 2) {
          b->branches = nb;
          drop_graphs(b);
          ms[nb - 1] = time_step(b, [&] { return step_graph(b, 1); });
          if (ms[nb - 1] < 0) {
            rc = berr(b, NS3D_ECUDA, "autotuner timing");
            break;
          }
          if (ms[nb - 1] < ms[best - 1]) best = nb;
        }
        if (rc == NS3D_OK) {
          b->branches = best;
          if (ms_out)
            for (int k = 0; k < ns3d_batch::MAX_BRANCHES; ++k) ms_out[DIR_VARIANTS * b->count + k] = ms[k];
          cache_append(cache_path, ekey, "branches", best, ms, ns3d_batch::MAX_BRANCHES);
        }
      }
    }
  }
  cudaStreamSynchronize(b->stream);
  for (double* p : tmp) cudaFree(p);
  b->u = saved;
  drop_graphs(b);
  ns3d_batch_check(b);  // the timing runs may have flagged the copies; clear the word
  const int rc2 = rebuild(b);
  return rc != NS3D_OK ? rc : rc2;
}

int ns3d_batch_schedule_info(const ns3d_batch* b, int* variants, int* branches) {
  if (!b) return NS3D_EINVAL;
  if (variants)
    for (int i = 0; i < b->count; ++i) variants[i] = b->ivar[i];
  if (branches) *branches = b->branches;
  return NS3D_OK;
}

int ns3d_batch_info(const ns3d_batch* b, int* variant, int* persistent_ctas_per_sm, int* persistent_in_graph) {
  if (!b) return NS3D_EINVAL;
  if (variant) *variant = b->variant;
  if (persistent_ctas_per_sm) *persistent_ctas_per_sm = b->pers_ctas;
  if (persistent_in_graph) *persistent_in_graph = b->persistent_graph;
  return NS3D_OK;
}

const char* ns3d_batch_last_error(const ns3d_batch* b) { return b ? b->err : "batch is NULL"; }

}  // extern "C"
