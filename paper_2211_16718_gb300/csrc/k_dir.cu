// Standalone launches of the fused direction pass (one tile per CTA); the tile
// computation itself is dir_tile in k_dir_impl.cuh.  Tile shapes (points along
// the pencil x lines) are template variants: a context uses the one set by
// ns3d_set_variant (default 0); an ensemble's autotuner picks one per grid size.
//   MODE 0 (all FP64):              32 x 4
//   MODE 1 (FP64 + double-float):   variant 0: 24 x 4, 1: 16 x 4, 2: 40 x 2
// All variants compute bitwise identical results (the per-interface arithmetic
// does not depend on the tiling).
#include "k_dir_impl.cuh"

namespace ns3d {

namespace {

template <int D, int MODE, int TP, int W>
__global__ void __launch_bounds__(Plan<MODE, TP, W>::THREADS, Plan<MODE, TP, W>::MIN_CTAS) k_dir(const DirArgs a) {
  extern __shared__ __align__(16) double sm[];
  if (D == 2) {
    const int tz = a.zorder ? blockIdx.y : blockIdx.x, tl = a.zorder ? blockIdx.x : blockIdx.y;
    dir_tile<D, MODE, TP, W>(a, sm, a.t0 + tz, tl, blockIdx.z);
  } else {
    dir_tile<D, MODE, TP, W>(a, sm, blockIdx.x, blockIdx.y, a.t0 + blockIdx.z);
  }
}

// Tiles [lo, hi) along the range axis (hi < 0: all): the tiles along z for D = 2 (blockIdx.x, or
// blockIdx.y with a.zorder), blockIdx.z (planes z) for D = 0, 1.
template <int D, int MODE, int TP, int W>
cudaError_t launch_t(const DirArgs& a, cudaStream_t s, int lo = 0, int hi = -1) {
  using PL = Plan<MODE, TP, W>;
  constexpr int AX = (D == 0) ? 1 : 0;
  constexpr int BX = (D == 2) ? 1 : 2;
  dim3 grid((a.g.n[D] + TP - 1) / TP, (a.g.n[AX] + W - 1) / W, a.g.n[BX]);
  if (D == 2 && a.zorder) {
    const unsigned t = grid.x;
    grid.x = grid.y;
    grid.y = t;
  }
  unsigned& ext = (D == 2) ? (a.zorder ? grid.y : grid.x) : grid.z;
  if (hi < 0) hi = (int)ext;
  if (lo < 0 || hi > (int)ext || lo > hi) return cudaErrorInvalidValue;
  if (lo == hi) return cudaSuccess;
  ext = (unsigned)(hi - lo);
  DirArgs r = a;
  r.t0 = lo;
  k_dir<D, MODE, TP, W><<<grid, PL::THREADS, PL::BYTES, s>>>(r);
  return cudaGetLastError();
}

// Dynamic shared memory of the tile plan, and the largest shared-memory carveout so that
// Plan::MIN_CTAS tiles fit on an SM (the rest of the unified L1 stays cache).
template <typename K>
cudaError_t set_func_attr(K* kernel, int bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

template <int MODE, int TP, int W>
cudaError_t set_attr() {
  const int bytes = Plan<MODE, TP, W>::BYTES;
  cudaError_t e = set_func_attr(k_dir<0, MODE, TP, W>, bytes);
  if (e == cudaSuccess) e = set_func_attr(k_dir<1, MODE, TP, W>, bytes);
  if (e == cudaSuccess) e = set_func_attr(k_dir<2, MODE, TP, W>, bytes);
  return e;
}

template <int MODE, int TP, int W>
cudaError_t launch_dirs(int d, const DirArgs& a, cudaStream_t s, int lo = 0, int hi = -1) {
  switch (d) {
    case 0: return launch_t<0, MODE, TP, W>(a, s, lo, hi);
    case 1: return launch_t<1, MODE, TP, W>(a, s, lo, hi);
    default: return launch_t<2, MODE, TP, W>(a, s, lo, hi);
  }
}

}  // namespace

cudaError_t prepare_dir_kernels() {
  cudaError_t e = set_attr<0, 32, 4>();
  if (e == cudaSuccess) e = set_attr<1, 24, 4>();
  if (e == cudaSuccess) e = set_attr<1, 16, 4>();
  if (e == cudaSuccess) e = set_attr<1, 40, 2>();
  if (e == cudaSuccess) e = prepare_dir32_kernels();
  if (e == cudaSuccess) e = prepare_visc_kernels();
  return e;
}

// With the tiles along z fastest, the CTAs resident at one time cover every z-plane of a few
// line groups, i.e. one 32-byte piece of each of ~30 planes of ~30 arrays per tile.  On a 1024^3
// grid (8 MB between planes) that z pass took 2.8x the time of the x pass; walking the line
// groups of one z-tile row first (CTAs resident at once within a few tile rows) brought it to
// 1.26x.  On 256^3 the tiles-along-z order is 0.5 % faster overall, so the switch is by size:
// line groups first from 2^28 points (2 GB per array) up.
int dir_zorder(const Grid& g) { return g.N >= (1LL << 28) ? 1 : 0; }

void dir_tile_shape(int mode, int variant, int* tp, int* w) {
  if (mode == 0) {
    *tp = 32;
    *w = 4;
  } else if (mode == 1 && variant == 1) {
    *tp = 16;
    *w = 4;
  } else if (mode == 1 && variant == 2) {
    *tp = 40;
    *w = 2;
  } else if (mode == 1) {
    *tp = 24;
    *w = 4;
  } else {  // FP32 bulk
    *tp = 32;
    *w = 4;
  }
}

cudaError_t launch_dir(int d, const DirArgs& a, cudaStream_t s) {
  if (a.mode == 2) return launch_dir32(d, a, s);
  return launch_dir_range(d, a, s, 0, -1);
}

cudaError_t launch_dir_range(int d, const DirArgs& a, cudaStream_t s, int lo, int hi) {
  if (a.mode == 2) return cudaErrorInvalidValue;
  if (a.mode == 0) return launch_dirs<0, 32, 4>(d, a, s, lo, hi);
  switch (a.variant) {
    case 1: return launch_dirs<1, 16, 4>(d, a, s, lo, hi);
    case 2: return launch_dirs<1, 40, 2>(d, a, s, lo, hi);
    default: return launch_dirs<1, 24, 4>(d, a, s, lo, hi);
  }
}

}  // namespace ns3d
