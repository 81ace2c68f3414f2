// Internal declarations shared by the CUDA translation units of libns3d.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ns3d.h"

namespace ns3d {

// Primitive-variable planes written by the primitive kernel ([NPRIM][N]).
enum { PM_U = 0, PM_V = 1, PM_W = 2, PM_P = 3, PM_T = 4, PM_H = 5, PM_SR = 6, NPRIM = 7 };
// Viscous flux planes ([12][N]): direction d occupies planes 4d..4d+3 holding
// (tau_xd, tau_yd, tau_zd, u tau_xd + v tau_yd + w tau_zd - q_d).
enum { NVISC = 12 };

// Status bits of the sticky device status word.
enum { ST_NONPHYS = 1, ST_DF_RANGE = 2 };

// Epilogue of the z-direction kernel (the last of the three direction passes).
enum Epi {
  EPI_ACC_WRITE = 0,  // k = contribution                      (first direction)
  EPI_ACC_ADD = 1,    // k += contribution                     (middle direction)
  EPI_RHS_OUT = 2,    // out = k + contribution                (ns3d_rhs)
  EPI_RK4_FIRST = 3,  // K = k + c; uout = un + a K; acc = K
  EPI_RK4_MID = 4,    // K; uout = un + a K; acc += 2 K
  EPI_RK4_LAST = 5,   // K; uout = un + (dt/6)(acc + K)
  EPI_SSP_1 = 6,      // uout = un + dt K
  EPI_SSP_2 = 7,      // uout = 3/4 un + 1/4 (us + dt K)
  EPI_SSP_3 = 8       // uout = 1/3 un + 2/3 (us + dt K)
};

struct Grid {
  int n[3];          // nx, ny, nz
  long long N;       // nx*ny*nz
  double h[3];       // dx, dy, dz
  double rh[3];      // 1/dx, 1/dy, 1/dz            (host-computed: no FP64 division per thread)
  double r12h[3];    // 1/(12 dx), 1/(12 dy), 1/(12 dz)
  double hrh[3];     // 1/(2 dx), 1/(2 dy), 1/(2 dz)
  float rh_f[3];     // 1/dx, 1/dy, 1/dz rounded to FP32 (host-rounded: no FP64 conversion per thread)
};

// Spacing of the periodic box [0,lx) x [0,ly) x [0,lz) on the grid g.n (Sec. 2.2: x_i = i dx).
inline void grid_set_spacing(Grid& g, double lx, double ly, double lz) {
  const double len[3] = {lx, ly, lz};
  for (int d = 0; d < 3; ++d) {
    g.h[d] = len[d] / g.n[d];
    g.rh[d] = 1.0 / g.h[d];
    g.r12h[d] = 1.0 / (12.0 * g.h[d]);
    g.hrh[d] = 0.5 / g.h[d];
    g.rh_f[d] = (float)g.rh[d];
  }
}

struct DirArgs {
  Grid g;
  const double* u;   // stage input state [5][N]
  const double* pm;  // primitives of u [NPRIM][N]
  const double* fv;  // viscous fluxes [NVISC][N] or nullptr (inviscid); FP32-bulk: FP32 planes
  int fv_dstride;    // planes per direction in fv: 4 ([12][N], all directions) or 0 ([4][N], this direction)
  double* k;         // RHS accumulator [5][N]
  int epi;           // Epi
  double* out;       // EPI_RHS_OUT: destination; RK modes: next stage state
  const double* un;  // RK base state U_n
  double* acc;       // RK4 accumulator
  double a;          // RK stage coefficient (a_s * dt, or dt)
  double gamma;
  double eps4;       // 4 * weno_eps (smoothness indicators are scaled by 4)
  double hdelta;     // Harten entropy-fix fraction
  int* status;
  int mode;          // 0: all FP64; 1: FP64 values, double-float weights/offsets; 2: FP32 bulk
  int variant;       // tile-shape variant of MODE 1 (see dir_tile_shape)
  int t0;            // partial launches (launch_dir_range): index of the first tile row of the range
                     // (planes for D = 0, 1; tiles along z for D = 2); 0 for whole-grid launches
  int zorder;        // z pass: 0 = consecutive CTAs walk the tiles along z, 1 = the line groups (dir_zorder)
  float c133_hi, c133_lo;  // 13/3 as a double-float
  float eps4_hi, eps4_lo;  // 4 * weno_eps as a double-float
  float gm1_hi, gm1_lo;      // gamma - 1 as a double-float
  float hd_hi, hd_lo;        // Harten fraction as a double-float
};

// Launchers (return cudaGetLastError() of the launch).
// df: the NS3D_FP64 primitive layout (T, H and sqrt(rho) as double-float pairs, see
// prim_point); the viscous, direction and statistics kernels of the same context read it.
// [p0, p1): the points of a partial launch (p1 < 0: through N).
cudaError_t launch_prim(const Grid& g, const double* u, double* pm, double gamma, int* status, cudaStream_t s,
                        int df = 0, long long p0 = 0, long long p1 = -1);
// only_d < 0: all three viscous flux vectors into fv[12][N]; only_d = d: the flux along d into fv[4][N];
// df: the NS3D_FP64 form (double-float from the stencil values on; primitives from launch_prim(df=1))
// [z0, z1): the planes of a partial launch (z1 < 0: through nz); with df, z0 and z1 (unless nz) must be
// multiples of VISC_ZCHUNK, the z extent of one CTA of the tiled kernel.
constexpr int VISC_ZCHUNK = 16;
cudaError_t launch_visc(const Grid& g, const double* pm, double* fv, double mu, double kappa, cudaStream_t s,
                        int only_d = -1, int df = 0, int z0 = 0, int z1 = -1);
// FP32-bulk viscous fluxes, straight from the state u: FP32 planes fv[12][N] (only_d = d: fv[4][N])
// that the FP32-bulk direction passes read (DirArgs::fv then points at FP32 planes).
cudaError_t launch_visc32(const Grid& g, const double* u, float* fv, double gamma, double mu, double kappa,
                          cudaStream_t s, int only_d = -1);
cudaError_t prepare_dir_kernels();  // per device, before the first launch
cudaError_t launch_dir(int d, const DirArgs& a, cudaStream_t s);  // dispatches on a.mode, a.variant
// The tiles [lo, hi) of a direction pass along its range axis: planes z for d = 0, 1, tiles along z
// (dir_tile_shape points each) for d = 2.  MODE 0 and 1 only.
cudaError_t launch_dir_range(int d, const DirArgs& a, cudaStream_t s, int lo, int hi);
// CTA order of the z pass for grid g (DirArgs::zorder).
int dir_zorder(const Grid& g);
void dir_tile_shape(int mode, int variant, int* tp, int* w);      // points x lines of a tile
constexpr int DIR_VARIANTS = 3;                                   // tile variants of MODE 1
cudaError_t prepare_dir32_kernels();
cudaError_t prepare_visc_kernels();
cudaError_t launch_dir32(int d, const DirArgs& a, cudaStream_t s);  // FP32-bulk (a.mode == 2)
int stats_num_blocks(const Grid& g);
cudaError_t launch_stats(const Grid& g, const double* u, const double* pm, double gamma, double* partials,
                         cudaStream_t s, int df = 0);
cudaError_t launch_stats_final(const Grid& g, const double* partials, int nblocks, const int* status,
                               double* out, cudaStream_t s);
int alu_probe(double out[5]);

// ---- adjoint (vector-Jacobian product) of the right-hand side --------------------
// Epilogue of the last adjoint direction pass; K = k + contribution = J(u)^T lambda.
enum AdjEpi {
  AEPI_WRITE = 0,  // k = contribution
  AEPI_ADD = 1,    // k += contribution
  AEPI_OUT = 2,    // gout = K
  AEPI_RK4_4 = 3,  // gout = ubs + K;  lnext = c1 ubs + c2 K     (RK4, stage 4 in reverse)
  AEPI_RK4_M = 4,  // gout += K;       lnext = c1 ubs + c2 K     (stages 3, 2)
  AEPI_ACC = 5,    // gout += K                                  (RK4 and SSP-RK3, stage 1)
  AEPI_SSP_3 = 6,  // s = 2/3 ubs + K; gout = 1/3 ubs + 3/4 s; lnext = c2 s/4; sb = s/4
  AEPI_SSP_2 = 7   // s = sb + K;      gout += s;  lnext = c2 s  (sb and lnext may alias)
};

struct AdjArgs {
  Grid g;
  const double* u;    // state at which the Jacobian is taken [5][N]
  const double* pm;   // its primitives [NPRIM][N]
  const double* lam;  // adjoint input [5][N]; lambda = lam_scale * lam
  double lam_scale;
  double* k;          // accumulator [5][N]
  int epi;            // AdjEpi
  double* gout;       // AEPI_OUT / RK modes: adjoint of the step's initial state
  const double* ubs;  // incoming adjoint of the step's final state
  double* lnext;      // adjoint input of the next (earlier) stage
  double* sb;         // SSP stage adjoint
  double c1, c2;
  double gamma, eps4, hdelta;
  int* status;
  int mode;           // 0: all FP64; 1: reconstruction adjoints in double-float (NS3D_FP64)
};

constexpr int ADJ_SCRATCH_PLANES = 16;  // viscous-adjoint scratch: grad adjoint 12, velocity 3, rho 1
cudaError_t prepare_adj_kernels();
cudaError_t launch_adj_dir(int d, const AdjArgs& a, cudaStream_t s);
// scratch = adjoint of the velocity/temperature gradients and of the velocities
// expo non-null: the NS3D_FP64 (double-float) forms, whose scratch planes hold double-float pairs
// relative to 2^E, E = the largest binary exponent of lam_scale * lambda, kept in *expo by kernel 1
// for kernel 2
cudaError_t launch_visc_adj1(const Grid& g, const double* pm, const double* lam, double lam_scale, double* scratch,
                             double mu, double kappa, cudaStream_t s, int* expo = nullptr);
// out (= or +=) adjoint of u through the primitives, from the scratch planes;
// with_rho adds the direct density plane (scratch plane 15)
cudaError_t launch_visc_adj2(const Grid& g, const double* u, const double* scratch, double gamma, double* out,
                             int accumulate, int with_rho, cudaStream_t s, const int* expo = nullptr);
// gradient of the mean kinetic energy with respect to u
cudaError_t launch_ke_seed(const Grid& g, const double* u, double* grad, cudaStream_t s);
// scratch planes of the enstrophy gradient (finished by launch_visc_adj2 with with_rho)
cudaError_t launch_ens_seed(const Grid& g, const double* u, const double* pm, double* scratch, cudaStream_t s);

// Periodic wrap of an index that may be off by less than a few periods.
__host__ __device__ inline int wrap_idx(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

}  // namespace ns3d
