// Host side of the C ABI declared in include/ns3d.h: parameter validation,
// library-owned device scratch, launch sequences of the right-hand side and of
// the Runge-Kutta stages, statistics, error reporting and kernel timing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "ns3d_ctx.cuh"

using namespace ns3d;

namespace {

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}

DirArgs base_args(ns3d_ctx* c, const double* u) {
  DirArgs a;
  a.g = c->g;
  a.u = u;
  a.pm = c->pm;
  a.fv = (c->p.mu_eff > 0.0) ? c->fv : nullptr;
  a.fv_dstride = c->lean ? 0 : 4;
  a.k = c->k;
  a.epi = EPI_ACC_WRITE;
  a.out = nullptr;
  a.un = nullptr;
  a.acc = c->acc;
  a.a = 0.0;
  a.gamma = c->p.gamma;
  a.eps4 = 4.0 * c->p.weno_eps;
  a.hdelta = c->p.harten_delta;
  a.status = c->status;
  a.mode = (c->p.precision == NS3D_FP64_STRICT) ? 0 : (c->p.precision == NS3D_FP32_BULK) ? 2 : 1;
  a.variant = c->variant;
  a.t0 = 0;
  a.zorder = (c->zorder >= 0) ? c->zorder : dir_zorder(c->g);
  const double c133 = 13.0 / 3.0, eps4 = 4.0 * c->p.weno_eps;
  a.c133_hi = (float)c133;
  a.c133_lo = (float)(c133 - (double)a.c133_hi);
  a.eps4_hi = (float)eps4;
  a.eps4_lo = (float)(eps4 - (double)a.eps4_hi);
  const double gm1 = c->p.gamma - 1.0;
  a.gm1_hi = (float)gm1;
  a.gm1_lo = (float)(gm1 - (double)a.gm1_hi);
  a.hd_hi = (float)c->p.harten_delta;
  a.hd_lo = (float)(c->p.harten_delta - (double)a.hd_hi);
  return a;
}

// Map the sticky status word to an error code.
int status_code(int word) {
  if (word & ST_NONPHYS) return NS3D_ENONPHYSICAL;
  if (word & ST_DF_RANGE) return NS3D_ERANGE;
  return NS3D_OK;
}

}  // namespace

namespace ns3d {

// One full right-hand-side evaluation of state u: primitives, viscous fluxes,
// x and y passes accumulating into k, z pass with the given epilogue.
int rhs_pass(ns3d_ctx* c, const double* u, int epi, double* out, const double* un, double coef,
             const SlabPipe* pin, const SlabPipe* pout) {
  const bool f32 = (c->p.precision == NS3D_FP32_BULK);
  const int df = (c->p.precision == NS3D_FP64) ? 1 : 0;
  const Grid& g = c->g;
  const long long plane = (long long)g.n[0] * g.n[1];
  // FP32-bulk: the direction and viscous kernels form their primitive variables from u themselves
  auto prim = [&](int z0, int z1) {
    if (f32) return (int)NS3D_OK;
    return timed(c, NS3D_K_PRIM, [&] {
      return launch_prim(g, u, c->pm, c->p.gamma, c->status, c->stream, df, z0 * plane, z1 * plane);
    }, "primitive kernel");
  };
  const bool visc = c->p.mu_eff > 0.0;
  const double kappa = visc ? c->p.mu_eff / ((c->p.gamma - 1.0) * c->p.prandtl) : 0.0;
  // viscous fluxes of all directions (only_d < 0), or of direction only_d (lean storage), planes [z0, z1)
  auto visc_flux = [&](int only_d, int z0, int z1) {
    return timed(c, NS3D_K_VISC, [&] {
      return f32 ? launch_visc32(g, u, reinterpret_cast<float*>(c->fv), c->p.gamma, c->p.mu_eff, kappa, c->stream,
                                 only_d)
                 : launch_visc(g, c->pm, c->fv, c->p.mu_eff, kappa, c->stream, only_d, df, z0, z1);
    }, "viscous-flux kernel");
  };
  DirArgs a = base_args(c, u);
  static const int kid[3] = {NS3D_K_DIR_X, NS3D_K_DIR_Y, NS3D_K_DIR_Z};
  static const char* what[3] = {"x-direction kernel", "y-direction kernel", "z-direction kernel"};
  // direction pass d over the tiles [lo, hi) of its range axis (hi < 0: whole grid)
  auto dir = [&](int d, int lo, int hi) {
    a.epi = (d == 0) ? EPI_ACC_WRITE : (d == 1) ? EPI_ACC_ADD : epi;
    if (d == 2) {
      a.out = out;
      a.un = un;
      a.a = coef;
    }
    return timed(c, kid[d], [&] {
      return hi < 0 ? launch_dir(d, a, c->stream) : launch_dir_range(d, a, c->stream, lo, hi);
    }, what[d]);
  };
  int rc;
  if (pin) {
    // slab j of u is usable after pin->ev[j].  The viscous stencil reaches 2 planes into the
    // neighbouring slabs (periodically), so the viscous, x and y kernels of slab j run once the
    // primitives of slabs j - 1 .. j + 1 exist: slabs 1 .. n-2 as the copies land, then n-1 and 0.
    const int n = pin->n;
    auto xy_slab = [&](int j) {
      const int z0 = pin->lo[j], z1 = pin->lo[j + 1];
      int r = (visc ? visc_flux(-1, z0, z1) : NS3D_OK);
      if (!r) r = dir(0, z0, z1);
      if (!r) r = dir(1, z0, z1);
      return r;
    };
    for (int j = 0; j < n; ++j) {
      const cudaError_t e = cudaStreamWaitEvent(c->stream, pin->ev[j], 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "wait for a state slab");
      if ((rc = prim(pin->lo[j], pin->lo[j + 1]))) return rc;
      if (j >= 2 && (rc = xy_slab(j - 1))) return rc;
    }
    if (n > 1 && (rc = xy_slab(n - 1))) return rc;
    if ((rc = xy_slab(0))) return rc;
  } else {
    if ((rc = prim(0, g.n[2]))) return rc;
    if (visc && !c->lean && (rc = visc_flux(-1, 0, -1))) return rc;
    for (int d = 0; d < 2; ++d) {
      if (visc && c->lean && (rc = visc_flux(d, 0, -1))) return rc;
      if ((rc = dir(d, 0, -1))) return rc;
    }
  }
  if (visc && c->lean && (rc = visc_flux(2, 0, -1))) return rc;
  if (!pout) return dir(2, 0, -1);
  // the z pass per slab of tiles; each slab of out is final after its launch and goes to the host
  // on the copy stream while the next slabs compute
  for (int j = 0; j < pout->n; ++j) {
    if ((rc = dir(2, pout->lo[j], pout->lo[j + 1]))) return rc;
    const int z0 = pout->lo[j] * pout->tp, z1 = min(pout->lo[j + 1] * pout->tp, g.n[2]);
    cudaError_t e = cudaEventRecord(pout->ev[j], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, pout->ev[j], 0);
    for (int v = 0; v < 5 && e == cudaSuccess; ++v) {
      const long long off = v * g.N + z0 * plane;
      e = cudaMemcpyAsync(pout->host + off, out + off, sizeof(double) * (size_t)((z1 - z0) * plane),
                          cudaMemcpyDeviceToHost, c->copy_stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy of a state slab");
  }
  return NS3D_OK;
}

int stats_pass(ns3d_ctx* c, const double* u, double* out_dev) {
  // the double-float primitive layout for NS3D_FP64 and NS3D_FP32_BULK (FP64 reductions either way)
  const int df = (c->p.precision != NS3D_FP64_STRICT) ? 1 : 0;
  int rc = timed(c, NS3D_K_PRIM,
                 [&] { return launch_prim(c->g, u, c->pm, c->p.gamma, c->status, c->stream, df); },
                 "primitive kernel");
  if (rc) return rc;
  rc = timed(c, NS3D_K_STATS,
             [&] { return launch_stats(c->g, u, c->pm, c->p.gamma, c->partials, c->stream, df); },
             "statistics kernel");
  if (rc) return rc;
  return timed(c, NS3D_K_STATS_FINAL,
               [&] { return launch_stats_final(c->g, c->partials, c->nstat_blocks, c->status, out_dev, c->stream); },
               "statistics final kernel");
}

int ensure_stage_buffers(ns3d_ctx* c) {
  const size_t bytes = sizeof(double) * 5 * (size_t)c->g.N;
  if (!c->ua && !dev_alloc(c, (void**)&c->ua, bytes)) return set_err(c, NS3D_ENOMEM, "RK stage state");
  if (!c->ub && !dev_alloc(c, (void**)&c->ub, bytes)) return set_err(c, NS3D_ENOMEM, "RK stage state");
  if (c->p.rk == NS3D_RK4 && !c->acc && !dev_alloc(c, (void**)&c->acc, bytes))
    return set_err(c, NS3D_ENOMEM, "RK4 accumulator");
  return NS3D_OK;
}

int rk_one_step(ns3d_ctx* c, double* u, double dt, const SlabPipe* pin, const SlabPipe* pout) {
  int rc = ensure_stage_buffers(c);
  if (rc) return rc;
  if (c->p.rk == NS3D_RK4) {
    if ((rc = rhs_pass(c, u, EPI_RK4_FIRST, c->ua, u, 0.5 * dt, pin))) return rc;
    if ((rc = rhs_pass(c, c->ua, EPI_RK4_MID, c->ub, u, 0.5 * dt))) return rc;
    if ((rc = rhs_pass(c, c->ub, EPI_RK4_MID, c->ua, u, dt))) return rc;
    return rhs_pass(c, c->ua, EPI_RK4_LAST, u, u, dt / 6.0, nullptr, pout);
  }
  if ((rc = rhs_pass(c, u, EPI_SSP_1, c->ua, u, dt, pin))) return rc;
  if ((rc = rhs_pass(c, c->ua, EPI_SSP_2, c->ub, u, dt))) return rc;
  return rhs_pass(c, c->ub, EPI_SSP_3, u, u, dt, nullptr, pout);
}

}  // namespace ns3d

namespace {

int collect_timing(ns3d_ctx* c) {
  for (auto& t : c->pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "event timing");
    c->ms[t.kid] += ms;
    c->pool.push_back(t.e0);
    c->pool.push_back(t.e1);
  }
  c->pending.clear();
  return NS3D_OK;
}

int validate(const ns3d_params* p, char* msg, size_t n) {
  if (!p) return snprintf(msg, n, "params is NULL"), NS3D_EINVAL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return snprintf(msg, n, "grid sizes must be >= 1"), NS3D_EINVAL;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (1LL << 32)) return snprintf(msg, n, "grid too large (%lld points)", N), NS3D_EINVAL;
  if (p->nx > 65535 * 4 || p->ny > 65535 || p->nz > 65535)
    return snprintf(msg, n, "grid dimension beyond launch limits"), NS3D_EINVAL;
  if (!(p->lx > 0) || !(p->ly > 0) || !(p->lz > 0) || !isfinite(p->lx) || !isfinite(p->ly) || !isfinite(p->lz))
    return snprintf(msg, n, "box lengths must be finite and > 0"), NS3D_EINVAL;
  if (!(p->gamma > 1.0) || !isfinite(p->gamma)) return snprintf(msg, n, "gamma must be > 1"), NS3D_EINVAL;
  if (!(p->mu_eff >= 0.0) || !isfinite(p->mu_eff)) return snprintf(msg, n, "mu_eff must be >= 0"), NS3D_EINVAL;
  if (p->mu_eff > 0.0 && (!(p->prandtl > 0.0) || !isfinite(p->prandtl)))
    return snprintf(msg, n, "prandtl must be > 0"), NS3D_EINVAL;
  if (!(p->weno_eps > 0.0) || !isfinite(p->weno_eps)) return snprintf(msg, n, "weno_eps must be > 0"), NS3D_EINVAL;
  if (p->weno_p != 2) return snprintf(msg, n, "only weno_p = 2 is supported"), NS3D_EINVAL;
  if (!(p->harten_delta >= 0.0) || !isfinite(p->harten_delta))
    return snprintf(msg, n, "harten_delta must be >= 0"), NS3D_EINVAL;
  if (p->rk != NS3D_RK4 && p->rk != NS3D_SSPRK3) return snprintf(msg, n, "unknown rk scheme"), NS3D_EINVAL;
  if (p->precision != NS3D_FP64 && p->precision != NS3D_FP64_STRICT && p->precision != NS3D_FP32_BULK)
    return snprintf(msg, n, "unsupported precision mode"), NS3D_EINVAL;
  if (p->storage != NS3D_STORAGE_AUTO && p->storage != NS3D_STORAGE_FULL && p->storage != NS3D_STORAGE_LEAN)
    return snprintf(msg, n, "unknown storage mode"), NS3D_EINVAL;
  if (p->precision != NS3D_FP64_STRICT && !(p->weno_eps >= 1e-15))
    return snprintf(msg, n, "weno_eps below 1e-15 needs NS3D_FP64_STRICT"), NS3D_EINVAL;
  return NS3D_OK;
}

}  // namespace

extern "C" {

void ns3d_default_params(ns3d_params* p, int nx, int ny, int nz) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->rk = NS3D_RK4;
  p->precision = NS3D_FP64;
  p->weno_p = 2;
  p->lx = p->ly = p->lz = 2.0 * M_PI;
  p->gamma = 1.4;
  p->mu_eff = 0.0;
  p->prandtl = 0.72;
  p->weno_eps = 1e-6;
  p->harten_delta = 0.1;
}

const char* ns3d_strerror(int code) {
  switch (code) {
    case NS3D_OK: return "ok";
    case NS3D_EINVAL: return "invalid argument";
    case NS3D_ENOMEM: return "out of memory";
    case NS3D_ECUDA: return "CUDA error";
    case NS3D_ENONPHYSICAL: return "non-physical state (rho <= 0, p <= 0, or non-finite value)";
    case NS3D_ETIMEOUT: return "device-side wait timed out (reserved: no call returns it)";
    case NS3D_ERANGE: return "data beyond the range of the double-float WENO weights (use NS3D_FP64_STRICT)";
    default: return "unknown error";
  }
}

const char* ns3d_last_error(const ns3d_ctx* c) { return c ? c->err : "context is NULL"; }

int ns3d_init(const ns3d_params* p, void* cuda_stream, ns3d_ctx** out) {
  if (!out) return NS3D_EINVAL;
  *out = nullptr;
  char msg[256];
  int rc = validate(p, msg, sizeof(msg));
  if (rc) return rc;
  ns3d_ctx* c = new (std::nothrow) ns3d_ctx();
  if (!c) return NS3D_ENOMEM;
  c->p = *p;
  c->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&c->device);
  c->g.n[0] = p->nx;
  c->g.n[1] = p->ny;
  c->g.n[2] = p->nz;
  c->g.N = (long long)p->nx * p->ny * p->nz;
  grid_set_spacing(c->g, p->lx, p->ly, p->lz);
  const size_t N = (size_t)c->g.N;
  c->nstat_blocks = stats_num_blocks(c->g);
  cudaError_t e = prepare_dir_kernels();
  if (e != cudaSuccess) {
    rc = cuda_fail(c, e, "kernel attributes");
    ns3d_free(c);
    return rc;
  }
  const bool visc = p->mu_eff > 0.0;
  if (p->storage == NS3D_STORAGE_LEAN) {
    c->lean = 1;
  } else if (p->storage == NS3D_STORAGE_AUTO && visc) {
    // FULL unless its scratch (incl. stage states and accumulator) would not fit with a margin
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    const size_t full = sizeof(double) * N * (NPRIM + 5 + NVISC + 10 + (p->rk == NS3D_RK4 ? 5 : 0));
    const size_t margin = (size_t)4 << 30;
    c->lean = (free_b > 0 && full + margin > free_b) ? 1 : 0;
  }
  struct {
    void** ptr;
    size_t bytes;
  } allocs[] = {
      {(void**)&c->pm, sizeof(double) * NPRIM * N},
      {(void**)&c->k, sizeof(double) * 5 * N},
      {(void**)&c->partials, sizeof(double) * 16 * (size_t)c->nstat_blocks},
      {(void**)&c->stats_dev, sizeof(double) * NS3D_STATS_NDOUBLE},
      {(void**)&c->status, sizeof(int)},
  };
  for (auto& a : allocs) {
    if (!dev_alloc(c, a.ptr, a.bytes)) {
      ns3d_free(c);
      return NS3D_ENOMEM;
    }
  }
  if (visc && !dev_alloc(c, (void**)&c->fv, sizeof(double) * (c->lean ? 4 : NVISC) * N)) {
    ns3d_free(c);
    return NS3D_ENOMEM;
  }
  if (cudaMallocHost((void**)&c->stats_host, sizeof(double) * NS3D_STATS_NDOUBLE) != cudaSuccess) {
    cudaGetLastError();
    ns3d_free(c);
    return NS3D_ENOMEM;
  }
  e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    ns3d_free(c);
    return NS3D_ECUDA;
  }
  *out = c;
  return NS3D_OK;
}

void ns3d_free(ns3d_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& t : c->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (auto e : c->slab_ev)
    if (e) cudaEventDestroy(e);
  cudaFree(c->pm);
  cudaFree(c->fv);
  cudaFree(c->k);
  cudaFree(c->ua);
  cudaFree(c->ub);
  cudaFree(c->acc);
  cudaFree(c->partials);
  cudaFree(c->stats_dev);
  cudaFree(c->status);
  cudaFree(c->uhost_dev);
  adjoint_free(c);
  if (c->stats_host) cudaFreeHost(c->stats_host);
  delete c;
}

int ns3d_set_stream(ns3d_ctx* c, void* s) {
  if (!c) return NS3D_EINVAL;
  c->stream = (cudaStream_t)s;
  return NS3D_OK;
}

int ns3d_rhs(ns3d_ctx* c, const double* u, double* rhs) {
  if (!c) return NS3D_EINVAL;
  if (!u || !rhs) return set_err(c, NS3D_EINVAL, "null state or rhs pointer");
  const size_t bytes = sizeof(double) * 5 * (size_t)c->g.N;
  if (overlaps(u, rhs, bytes)) return set_err(c, NS3D_EINVAL, "u and rhs overlap");
  return rhs_pass(c, u, EPI_RHS_OUT, rhs, nullptr, 0.0);
}

int ns3d_rk_step(ns3d_ctx* c, double* u, double dt, int nsteps) {
  if (!c) return NS3D_EINVAL;
  if (!u) return set_err(c, NS3D_EINVAL, "null state pointer");
  if (nsteps < 0 || !isfinite(dt)) return set_err(c, NS3D_EINVAL, "nsteps must be >= 0 and dt finite");
  for (int s = 0; s < nsteps; ++s) {
    int rc = rk_one_step(c, u, dt);
    if (rc) return rc;
  }
  return NS3D_OK;
}

int ns3d_stats_async(ns3d_ctx* c, const double* u, double* out_dev) {
  if (!c) return NS3D_EINVAL;
  if (!u || !out_dev) return set_err(c, NS3D_EINVAL, "null pointer");
  return stats_pass(c, u, out_dev);
}

static void fill_stats(const double* s, ns3d_stats_t* o) {
  o->mass = s[0];
  o->momx = s[1];
  o->momy = s[2];
  o->momz = s[3];
  o->energy = s[4];
  o->ke = s[5];
  o->enstrophy = s[6];
  o->rho_min = s[7];
  o->p_min = s[8];
  o->max_wavespeed_over_dx = s[9];
  o->status = status_code((int)s[10]);
  o->reserved = 0;
}

int ns3d_stats(ns3d_ctx* c, const double* u, ns3d_stats_t* out) {
  if (!c) return NS3D_EINVAL;
  if (!u || !out) return set_err(c, NS3D_EINVAL, "null pointer");
  int rc = stats_pass(c, u, c->stats_dev);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(c->stats_host, c->stats_dev, sizeof(double) * NS3D_STATS_NDOUBLE,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "statistics copy");
  fill_stats(c->stats_host, out);
  if (out->status) return set_err(c, out->status, "%s", ns3d_strerror(out->status));
  return NS3D_OK;
}

int ns3d_dt_from_cfl(ns3d_ctx* c, const double* u, double cfl, double* dt_out) {
  if (!c) return NS3D_EINVAL;
  if (!u || !dt_out) return set_err(c, NS3D_EINVAL, "null pointer");
  if (!(cfl > 0.0) || !isfinite(cfl)) return set_err(c, NS3D_EINVAL, "cfl must be finite and > 0");
  ns3d_stats_t st;
  int rc = ns3d_stats(c, u, &st);
  if (rc) return rc;
  const double w = st.max_wavespeed_over_dx;
  if (!(w > 0.0) || !isfinite(w)) return set_err(c, NS3D_ENONPHYSICAL, "no finite positive wave speed");
  *dt_out = cfl / w;
  return NS3D_OK;
}

int ns3d_check(ns3d_ctx* c) {
  if (!c) return NS3D_EINVAL;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  if (h) return set_err(c, status_code(h), "%s", ns3d_strerror(status_code(h)));
  return NS3D_OK;
}

namespace {

// Whether ns3d_step_host overlaps its copies with the kernels: the direction passes of
// NS3D_FP64 / NS3D_FP64_STRICT with all viscous fluxes stored, on grids of at least four
// viscous z chunks (smaller grids copy in well under a millisecond).
bool slab_pipeline_ok(const ns3d_ctx* c, int nsteps) {
  return nsteps >= 1 && !c->lean && c->p.precision != NS3D_FP32_BULK && c->g.n[2] >= 4 * VISC_ZCHUNK;
}

int ensure_copy_stream(ns3d_ctx* c) {
  if (c->copy_stream) return NS3D_OK;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (int k = 0; k < 2 * ns3d_ctx::MAX_SLABS + 1 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&c->slab_ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {  // leave nothing half made: the next call starts over
    for (auto& ev : c->slab_ev) {
      if (ev) cudaEventDestroy(ev);
      ev = nullptr;
    }
    if (s) cudaStreamDestroy(s);
    return cuda_fail(c, e, "copy stream");
  }
  c->copy_stream = s;
  return NS3D_OK;
}

// n slabs with boundaries at multiples of unit: lo[j] = unit * round(j * units / n), lo[n] = end
// (units = end / unit, the last slab taking the remainder).
void slab_bounds(SlabPipe& s, int n, int units, int unit, int end) {
  s.n = n;
  for (int j = 0; j < n; ++j) s.lo[j] = unit * (int)(((long long)j * units + n / 2) / n);
  s.lo[n] = end;
}

}  // namespace

int ns3d_step_host(ns3d_ctx* c, double* u_host, double dt, int nsteps, ns3d_stats_t* stats_host) {
  if (!c) return NS3D_EINVAL;
  if (!u_host) return set_err(c, NS3D_EINVAL, "null host state");
  if (nsteps < 0 || !isfinite(dt)) return set_err(c, NS3D_EINVAL, "nsteps must be >= 0 and dt finite");
  const size_t bytes = sizeof(double) * 5 * (size_t)c->g.N;
  if (!c->uhost_dev && !dev_alloc(c, (void**)&c->uhost_dev, bytes))
    return set_err(c, NS3D_ENOMEM, "device state for host stepping");
  int rc = NS3D_OK;
  cudaError_t e = cudaSuccess;
  if (slab_pipeline_ok(c, nsteps)) {
    // z-slabs in on the copy stream, the first stage's kernels following them slab by slab; the
    // last stage's z pass per slab of tiles, each slab out on the copy stream behind it
    if ((rc = ensure_copy_stream(c)) || (rc = ensure_stage_buffers(c))) return rc;
    const Grid& g = c->g;
    const long long plane = (long long)g.n[0] * g.n[1];
    SlabPipe pin, pout;
    const int chunks = g.n[2] / VISC_ZCHUNK;
    slab_bounds(pin, min(chunks, (int)ns3d_ctx::MAX_SLABS), chunks, VISC_ZCHUNK, g.n[2]);
    pin.ev = c->slab_ev;
    int tp = 0, w = 0;
    dir_tile_shape(c->p.precision == NS3D_FP64_STRICT ? 0 : 1, c->variant, &tp, &w);
    const int ztiles = (g.n[2] + tp - 1) / tp;
    slab_bounds(pout, min(ztiles, (int)ns3d_ctx::MAX_SLABS), ztiles, 1, ztiles);
    pout.ev = c->slab_ev + ns3d_ctx::MAX_SLABS;
    pout.host = u_host;
    pout.tp = tp;
    cudaEvent_t entry = c->slab_ev[2 * ns3d_ctx::MAX_SLABS];
    e = cudaEventRecord(entry, c->stream);  // the copies follow the work already on the stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, entry, 0);
    for (int j = 0; j < pin.n && e == cudaSuccess; ++j) {
      const long long z0 = pin.lo[j], z1 = pin.lo[j + 1];
      for (int v = 0; v < 5 && e == cudaSuccess; ++v) {
        const long long off = v * g.N + z0 * plane;
        e = cudaMemcpyAsync(c->uhost_dev + off, u_host + off, sizeof(double) * (size_t)((z1 - z0) * plane),
                            cudaMemcpyHostToDevice, c->copy_stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(pin.ev[j], c->copy_stream);
    }
    if (e != cudaSuccess) rc = cuda_fail(c, e, "host-to-device copy of a state slab");
    for (int s = 0; s < nsteps && !rc; ++s)
      rc = rk_one_step(c, c->uhost_dev, dt, s == 0 ? &pin : nullptr, s == nsteps - 1 ? &pout : nullptr);
    if (!rc && stats_host) rc = stats_pass(c, c->uhost_dev, c->stats_dev);
    if (!rc && stats_host) {
      e = cudaMemcpyAsync(c->stats_host, c->stats_dev, sizeof(double) * NS3D_STATS_NDOUBLE, cudaMemcpyDeviceToHost,
                          c->stream);
      if (e != cudaSuccess) rc = cuda_fail(c, e, "statistics copy");
    }
    // the host buffer is in use until both streams are done, also after a failure
    const cudaError_t e1 = cudaStreamSynchronize(c->copy_stream);
    const cudaError_t e2 = cudaStreamSynchronize(c->stream);
    if (rc) return rc;
    if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(c, e1 != cudaSuccess ? e1 : e2, "host stepping");
  } else {
    e = cudaMemcpyAsync(c->uhost_dev, u_host, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
    rc = ns3d_rk_step(c, c->uhost_dev, dt, nsteps);
    if (rc) return rc;
    if (stats_host) {
      rc = stats_pass(c, c->uhost_dev, c->stats_dev);
      if (rc) return rc;
      e = cudaMemcpyAsync(c->stats_host, c->stats_dev, sizeof(double) * NS3D_STATS_NDOUBLE, cudaMemcpyDeviceToHost,
                          c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "statistics copy");
    }
    e = cudaMemcpyAsync(u_host, c->uhost_dev, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  }
  if (stats_host) {
    fill_stats(c->stats_host, stats_host);
    if (stats_host->status) return set_err(c, stats_host->status, "%s", ns3d_strerror(stats_host->status));
  }
  return NS3D_OK;
}

int ns3d_timing_enable(ns3d_ctx* c, int on) {
  if (!c) return NS3D_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (auto& t : c->pending) {
    c->pool.push_back(t.e0);
    c->pool.push_back(t.e1);
  }
  c->pending.clear();
  for (int k = 0; k < NS3D_K_COUNT; ++k) {
    c->ms[k] = 0.0;
    c->launches[k] = 0;
  }
  c->timing = (on != 0);
  return NS3D_OK;
}

int ns3d_timing_read(ns3d_ctx* c, double* ms_out, long long* launches_out, int n) {
  if (!c || n < 0 || n > NS3D_K_COUNT) return NS3D_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "timing sync");
  int rc = collect_timing(c);
  if (rc) return rc;
  for (int k = 0; k < n; ++k) {
    if (ms_out) ms_out[k] = c->ms[k];
    if (launches_out) launches_out[k] = c->launches[k];
  }
  return NS3D_OK;
}

int ns3d_set_zorder(ns3d_ctx* c, int order) {
  if (!c || order < -1 || order > 1) return NS3D_EINVAL;
  c->zorder = order;
  return NS3D_OK;
}

int ns3d_set_variant(ns3d_ctx* c, int variant) {
  if (!c || variant < 0 || variant >= DIR_VARIANTS) return NS3D_EINVAL;
  c->variant = variant;
  return NS3D_OK;
}

int ns3d_storage_info(const ns3d_ctx* c, int* storage, size_t* device_bytes) {
  if (!c) return NS3D_EINVAL;
  if (storage) *storage = c->lean ? NS3D_STORAGE_LEAN : NS3D_STORAGE_FULL;
  if (device_bytes) *device_bytes = c->bytes;
  return NS3D_OK;
}

int ns3d_alu_probe(double out[5]) {
  if (!out) return NS3D_EINVAL;
  return alu_probe(out);
}

}  // extern "C"
