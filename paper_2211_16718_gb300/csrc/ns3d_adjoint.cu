// Host side of the adjoint calls of include/ns3d.h: vector-Jacobian products of the
// right-hand side and of one Runge-Kutta step (stage states recomputed, stages
// reversed), gradients of the kinetic-energy and enstrophy functionals, and the
// checkpointed reverse sweep over a trajectory.
#include <math.h>
#include <string.h>

#include "ns3d_ctx.cuh"

using namespace ns3d;

namespace {

// Adjoint buffers: stage states S2, S3, S4, the incoming adjoint copy and two
// stage-adjoint buffers (5N each), then the viscous-adjoint scratch.
enum { AB_S2 = 0, AB_S3 = 1, AB_S4 = 2, AB_UBS = 3, AB_LA = 4, AB_LB = 5, AB_STATES = 6 };

double* adj_buf(ns3d_ctx* c, int i) { return c->adj + (size_t)i * 5 * (size_t)c->g.N; }
double* adj_scratch(ns3d_ctx* c) { return c->adj + (size_t)AB_STATES * 5 * (size_t)c->g.N; }
// the exponent word of the double-float viscous adjoint (after the scratch planes)
int* adj_expo(ns3d_ctx* c) {
  return reinterpret_cast<int*>(c->adj + ((size_t)AB_STATES * 5 + ADJ_SCRATCH_PLANES) * (size_t)c->g.N);
}

int adj_ready(ns3d_ctx* c) {
  if (c->p.precision == NS3D_FP32_BULK)
    return set_err(c, NS3D_EINVAL, "the adjoint is available for NS3D_FP64 and NS3D_FP64_STRICT contexts");
  if (c->adj) return NS3D_OK;
  const size_t words = ((size_t)AB_STATES * 5 + ADJ_SCRATCH_PLANES) * (size_t)c->g.N + 1;  // + adj_expo
  cudaError_t e = prepare_adj_kernels();
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint kernel attributes");
  if (!dev_alloc(c, (void**)&c->adj, words * sizeof(double)))
    return set_err(c, NS3D_ENOMEM, "adjoint buffers (%zu bytes)", words * sizeof(double));
  return NS3D_OK;
}

bool overlaps5(const ns3d_ctx* c, const void* a, const void* b) {
  const size_t bytes = sizeof(double) * 5 * (size_t)c->g.N;
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bytes && y < x + bytes;
}

int copy_state(ns3d_ctx* c, double* dst, const double* src, const char* what) {
  const size_t bytes = sizeof(double) * 5 * (size_t)c->g.N;
  return timed(c, NS3D_K_ADJ_MISC, [&] { return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream); },
               what);
}

// K = J(u)^T (scale * lam), delivered through the epilogue of e (epi, gout, ubs,
// lnext, sb, c1, c2): primitives of u, viscous adjoint (writes k), then the three
// direction adjoints (accumulate into k; the z pass runs the epilogue).
int vjp_pass(ns3d_ctx* c, const double* u, const double* lam, double scale, AdjArgs e) {
  int rc = timed(c, NS3D_K_PRIM, [&] { return launch_prim(c->g, u, c->pm, c->p.gamma, c->status, c->stream); },
                 "primitive kernel");
  if (rc) return rc;
  const bool visc = c->p.mu_eff > 0.0;
  const int df = (c->p.precision == NS3D_FP64_STRICT) ? 0 : 1;
  if (visc) {
    const double kappa = c->p.mu_eff / ((c->p.gamma - 1.0) * c->p.prandtl);
    rc = timed(c, NS3D_K_ADJ_VISC, [&] {
      return launch_visc_adj1(c->g, c->pm, lam, scale, adj_scratch(c), c->p.mu_eff, kappa, c->stream,
                              df ? adj_expo(c) : nullptr);
    }, "viscous adjoint kernel 1");
    if (rc) return rc;
    rc = timed(c, NS3D_K_ADJ_VISC, [&] {
      return launch_visc_adj2(c->g, u, adj_scratch(c), c->p.gamma, c->k, 0, 0, c->stream, df ? adj_expo(c) : nullptr);
    }, "viscous adjoint kernel 2");
    if (rc) return rc;
  }
  AdjArgs a = e;
  a.g = c->g;
  a.u = u;
  a.pm = c->pm;
  a.lam = lam;
  a.lam_scale = scale;
  a.k = c->k;
  a.gamma = c->p.gamma;
  a.eps4 = 4.0 * c->p.weno_eps;
  a.hdelta = c->p.harten_delta;
  a.status = c->status;
  a.mode = (c->p.precision == NS3D_FP64_STRICT) ? 0 : 1;
  a.epi = visc ? AEPI_ADD : AEPI_WRITE;
  rc = timed(c, NS3D_K_ADJ_DIR, [&] { return launch_adj_dir(0, a, c->stream); }, "x-direction adjoint kernel");
  if (rc) return rc;
  a.epi = AEPI_ADD;
  rc = timed(c, NS3D_K_ADJ_DIR, [&] { return launch_adj_dir(1, a, c->stream); }, "y-direction adjoint kernel");
  if (rc) return rc;
  a.epi = e.epi;
  return timed(c, NS3D_K_ADJ_DIR, [&] { return launch_adj_dir(2, a, c->stream); }, "z-direction adjoint kernel");
}

AdjArgs epi_args(int epi, double* gout, const double* ubs, double* lnext, double* sb, double c1, double c2) {
  AdjArgs e;
  memset(&e, 0, sizeof(e));
  e.epi = epi;
  e.gout = gout;
  e.ubs = ubs;
  e.lnext = lnext;
  e.sb = sb;
  e.c1 = c1;
  e.c2 = c2;
  return e;
}

// Stage states of one step from u0, with the launches (and so the rounding) of the
// forward step: RK4 S2, S3, S4; SSP-RK3 S2, S3.  If next != nullptr the step is completed
// into next (the forward step's last pass).
int stage_states(ns3d_ctx* c, const double* u0, double* S2, double* S3, double* S4, double* next, double dt) {
  int rc = ensure_stage_buffers(c);  // the RK4 stage epilogues also update the accumulator
  if (rc) return rc;
  if (c->p.rk == NS3D_RK4) {
    if ((rc = rhs_pass(c, u0, EPI_RK4_FIRST, S2, u0, 0.5 * dt))) return rc;
    if ((rc = rhs_pass(c, S2, EPI_RK4_MID, S3, u0, 0.5 * dt))) return rc;
    if ((rc = rhs_pass(c, S3, EPI_RK4_MID, S4, u0, dt))) return rc;
    return next ? rhs_pass(c, S4, EPI_RK4_LAST, next, u0, dt / 6.0) : NS3D_OK;
  }
  if ((rc = rhs_pass(c, u0, EPI_SSP_1, S2, u0, dt))) return rc;
  if ((rc = rhs_pass(c, S2, EPI_SSP_2, S3, u0, dt))) return rc;
  return next ? rhs_pass(c, S3, EPI_SSP_3, next, u0, dt) : NS3D_OK;
}

// ubar <- (d step(u0)/d u0)^T ubar, given the step's stage states (S4 unused for SSP-RK3).
int rk_vjp_core(ns3d_ctx* c, const double* u0, const double* S2, const double* S3, const double* S4, double* ubar,
                double dt) {
  double* ubs = adj_buf(c, AB_UBS);
  double* La = adj_buf(c, AB_LA);
  double* Lb = adj_buf(c, AB_LB);
  int rc;
  if ((rc = copy_state(c, ubs, ubar, "adjoint copy"))) return rc;
  if (c->p.rk == NS3D_RK4) {
    if ((rc = vjp_pass(c, S4, ubs, dt / 6.0, epi_args(AEPI_RK4_4, ubar, ubs, La, nullptr, dt / 3.0, dt)))) return rc;
    if ((rc = vjp_pass(c, S3, La, 1.0, epi_args(AEPI_RK4_M, ubar, ubs, Lb, nullptr, dt / 3.0, 0.5 * dt)))) return rc;
    if ((rc = vjp_pass(c, S2, Lb, 1.0, epi_args(AEPI_RK4_M, ubar, ubs, La, nullptr, dt / 6.0, 0.5 * dt)))) return rc;
    return vjp_pass(c, u0, La, 1.0, epi_args(AEPI_ACC, ubar, nullptr, nullptr, nullptr, 0.0, 0.0));
  }
  if ((rc = vjp_pass(c, S3, ubs, (2.0 / 3.0) * dt, epi_args(AEPI_SSP_3, ubar, ubs, Lb, La, 0.0, dt)))) return rc;
  if ((rc = vjp_pass(c, S2, Lb, 1.0, epi_args(AEPI_SSP_2, ubar, nullptr, La, La, 0.0, dt)))) return rc;
  return vjp_pass(c, u0, La, 1.0, epi_args(AEPI_ACC, ubar, nullptr, nullptr, nullptr, 0.0, 0.0));
}

// ubar <- (d step(u0)/d u0)^T ubar for one step of the context's integrator.
int rk_vjp_step(ns3d_ctx* c, const double* u0, double* ubar, double dt) {
  double* S2 = adj_buf(c, AB_S2);
  double* S3 = adj_buf(c, AB_S3);
  double* S4 = adj_buf(c, AB_S4);
  int rc = stage_states(c, u0, S2, S3, S4, nullptr, dt);
  if (rc) return rc;
  return rk_vjp_core(c, u0, S2, S3, S4, ubar, dt);
}

int grow(ns3d_ctx* c, double** buf, int* cap, int states, const char* what) {
  if (*cap >= states) return NS3D_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronise before reallocation");
  cudaFree(*buf);
  c->bytes -= sizeof(double) * 5 * (size_t)c->g.N * (size_t)(*cap);
  *buf = nullptr;
  *cap = 0;
  const size_t bytes = sizeof(double) * 5 * (size_t)c->g.N * (size_t)states;
  if (!dev_alloc(c, (void**)buf, bytes)) return set_err(c, NS3D_ENOMEM, "%s (%zu bytes)", what, bytes);
  *cap = states;
  return NS3D_OK;
}

}  // namespace

namespace ns3d {

void adjoint_free(ns3d_ctx* c) {
  cudaFree(c->adj);
  cudaFree(c->ckpt);
  cudaFree(c->seg);
  c->adj = c->ckpt = c->seg = nullptr;
  c->ckpt_cap = c->seg_cap = 0;
}

}  // namespace ns3d

extern "C" {

int ns3d_rhs_vjp(ns3d_ctx* c, const double* u, const double* lam, double* out) {
  if (!c) return NS3D_EINVAL;
  if (!u || !lam || !out) return set_err(c, NS3D_EINVAL, "null pointer");
  if (overlaps5(c, out, u) || overlaps5(c, out, lam)) return set_err(c, NS3D_EINVAL, "out overlaps u or lam");
  int rc = adj_ready(c);
  if (rc) return rc;
  return vjp_pass(c, u, lam, 1.0, epi_args(AEPI_OUT, out, nullptr, nullptr, nullptr, 0.0, 0.0));
}

int ns3d_rk_step_vjp(ns3d_ctx* c, const double* u, double* ubar, double dt) {
  if (!c) return NS3D_EINVAL;
  if (!u || !ubar) return set_err(c, NS3D_EINVAL, "null pointer");
  if (!isfinite(dt)) return set_err(c, NS3D_EINVAL, "dt must be finite");
  if (overlaps5(c, u, ubar)) return set_err(c, NS3D_EINVAL, "u and ubar overlap");
  int rc = adj_ready(c);
  if (rc) return rc;
  return rk_vjp_step(c, u, ubar, dt);
}

int ns3d_functional(ns3d_ctx* c, const double* u, int which, double* value_host, double* grad) {
  if (!c) return NS3D_EINVAL;
  if (!u) return set_err(c, NS3D_EINVAL, "null state");
  if (which != NS3D_FUNC_KE && which != NS3D_FUNC_ENSTROPHY) return set_err(c, NS3D_EINVAL, "unknown functional");
  if (grad && overlaps5(c, u, grad)) return set_err(c, NS3D_EINVAL, "u and grad overlap");
  int rc;
  if (grad) {
    if ((rc = adj_ready(c))) return rc;
    if (which == NS3D_FUNC_KE) {
      rc = timed(c, NS3D_K_ADJ_MISC, [&] { return launch_ke_seed(c->g, u, grad, c->stream); }, "seed kernel");
    } else {
      rc = timed(c, NS3D_K_PRIM, [&] { return launch_prim(c->g, u, c->pm, c->p.gamma, c->status, c->stream); },
                 "primitive kernel");
      if (!rc)
        rc = timed(c, NS3D_K_ADJ_MISC, [&] { return launch_ens_seed(c->g, u, c->pm, adj_scratch(c), c->stream); },
                   "seed kernel");
      if (!rc)
        rc = timed(c, NS3D_K_ADJ_VISC,
                   [&] { return launch_visc_adj2(c->g, u, adj_scratch(c), c->p.gamma, grad, 0, 1, c->stream); },
                   "viscous adjoint kernel 2");
    }
    if (rc) return rc;
  }
  if (value_host) {
    if ((rc = stats_pass(c, u, c->stats_dev))) return rc;
    cudaError_t e = cudaMemcpyAsync(c->stats_host, c->stats_dev, sizeof(double) * NS3D_STATS_NDOUBLE,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "functional value copy");
    *value_host = c->stats_host[which == NS3D_FUNC_KE ? 5 : 6];
  }
  return NS3D_OK;
}

int ns3d_traj_forward(ns3d_ctx* c, double* u, double dt, int nsteps, int every) {
  if (!c) return NS3D_EINVAL;
  if (!u) return set_err(c, NS3D_EINVAL, "null state");
  if (nsteps < 0 || every < 1 || !isfinite(dt)) return set_err(c, NS3D_EINVAL, "need nsteps >= 0, every >= 1, finite dt");
  c->traj_nsteps = -1;
  const int nck = (nsteps + every - 1) / every;
  int rc = grow(c, &c->ckpt, &c->ckpt_cap, nck, "trajectory checkpoints");
  if (rc) return rc;
  for (int s = 0; s < nsteps; ++s) {
    if (s % every == 0 && (rc = copy_state(c, c->ckpt + (size_t)(s / every) * 5 * (size_t)c->g.N, u, "checkpoint copy")))
      return rc;
    if ((rc = rk_one_step(c, u, dt))) return rc;
  }
  c->traj_nsteps = nsteps;
  c->traj_every = every;
  c->traj_dt = dt;
  return NS3D_OK;
}

int ns3d_traj_vjp(ns3d_ctx* c, double* ubar) {
  if (!c) return NS3D_EINVAL;
  if (!ubar) return set_err(c, NS3D_EINVAL, "null adjoint");
  if (c->traj_nsteps < 0) return set_err(c, NS3D_EINVAL, "no recorded trajectory (call ns3d_traj_forward first)");
  int rc = adj_ready(c);
  if (rc) return rc;
  const int nsteps = c->traj_nsteps, every = c->traj_every;
  const double dt = c->traj_dt;
  // one segment: per step its state and stage states (RK4: 4 slots, SSP-RK3: 3), so the
  // stages are computed once, by the same launches as the forward step
  const int slots = (c->p.rk == NS3D_RK4) ? 4 : 3;
  if ((rc = grow(c, &c->seg, &c->seg_cap, every * slots, "trajectory segment"))) return rc;
  const size_t S = 5 * (size_t)c->g.N;
  auto slot = [&](int j, int k) { return c->seg + ((size_t)j * slots + k) * S; };
  const int nck = (nsteps + every - 1) / every;
  for (int sg = nck - 1; sg >= 0; --sg) {
    const int s0 = sg * every;
    const int len = (s0 + every <= nsteps) ? every : nsteps - s0;
    if ((rc = copy_state(c, slot(0, 0), c->ckpt + (size_t)sg * S, "segment copy"))) return rc;
    for (int j = 0; j < len; ++j) {
      double* S4 = (slots == 4) ? slot(j, 3) : nullptr;
      if ((rc = stage_states(c, slot(j, 0), slot(j, 1), slot(j, 2), S4, j + 1 < len ? slot(j + 1, 0) : nullptr, dt)))
        return rc;
    }
    for (int j = len - 1; j >= 0; --j) {
      const double* S4 = (slots == 4) ? slot(j, 3) : nullptr;
      if ((rc = rk_vjp_core(c, slot(j, 0), slot(j, 1), slot(j, 2), S4, ubar, dt))) return rc;
    }
  }
  return NS3D_OK;
}

}  // extern "C"
