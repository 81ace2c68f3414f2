// Hand-written adjoint (vector-Jacobian product g = J(u)^T lambda) of the
// right-hand side of arXiv 2211.16718, Sec. 2.1-2.2: all in FP64 for NS3D_FP64_STRICT
// contexts (k_adj_dir, k_visc_adj1/2); for NS3D_FP64 contexts the WENO5, Roe and viscous
// adjoints in double-float on the FP32 pipe (k_adj_dir_df, k_visc_adj1_df/2_df), with FP64
// for the point-flux adjoint and the final point algebra.
//
// Hyperbolic part, per direction D: R_i -= (Fhat_{i+1/2} - Fhat_{i-1/2})/h, so the
// adjoint of the interface flux is Lhat_{i+1/2} = (lambda_{i+1} - lambda_i)/h.  With
//   Fhat = (f^L + f^R)/2 - X |Lambda| X^{-1} (u^R - u^L)/2   (Roe average of U_i, U_{i+1}),
// the adjoint flows into the 18 reconstructions of the interface (u^L, u^R of the five
// conserved variables with the mass flux f_0 = rho u_D folded into u_{1+D}, f^L, f^R of
// f_1..f_4) and into the Roe-averaged state.  Each WENO5 reconstruction
//   q = sum_k omega_k q_k,   omega_k = (c_k/b_k^2) / sum_j (c_j/b_j^2),   b_k = 4(eps + beta_k)
// has the exact derivative dq/dq_t = sum_k omega_k dq_k/dq_t
//   + sum_k (-2 omega_k (q_k - q)/b_k) db_k/dq_t,
// b_k = 4 eps + (13/3) s_k^2 + v_k^2 with s_k the second difference and v_k the first-
// derivative combination of window k.  |lambda| has the subgradient sign(0) = 0 at its
// kink; Harten's quadratic branch is differentiated as written (Sec. 2.2).
//
// One CTA owns TP points along D times W lines; every interface whose stencil touches
// one of the tile's points (TP + 5 of them per line, halo of 5 points each side) is
// processed, and each point then gathers its contributions in a fixed order, so the
// result is deterministic and independent of the tiling.  Phases:
//   A  load u, primitives, point fluxes f_1..f_4, lambda                   [NP x W]
//   C  left/right WENO5 values and weights of the 9 scalars               [9 x NI x W]
//   D  Roe flux adjoint: adjoint of du = u^R - u^L and of the two states  [NI x W]
//   E  WENO5 adjoints -> six stencil contributions per scalar, interface [9 x NI x W]
//   F  gather, point-flux adjoint (f_1..f_4 of U), epilogue                [TP x W]
//
// Viscous part: G[q][e] = D_e W_q (W = u, v, w, T), viscous fluxes built from G and the
// velocities at each point, R_{1+c} += D_d Fv_d[c]; D_d^T = -D_d for the periodic
// 4th-order central difference.  Two point kernels: (1) adjoint of Fv -> adjoint of G
// and of the velocities, (2) -sum_e D_e of the G adjoint plus the velocity adjoint ->
// adjoint of u through u_k = m_k/rho, T = gamma (gamma - 1)(e/rho - |m|^2/(2 rho^2)).
// The double-float forms work relative to one power of two of lambda for the whole grid
// (k_lam_expo), so that their result scales exactly with lambda.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "df.cuh"
#include "df2.cuh"
#include "k_dir_common.cuh"
#include "k_point_impl.cuh"
#include "ns3d_internal.cuh"

namespace ns3d {

namespace {

template <int TP_, int W_>
struct AdjPlan {
  static constexpr int TP = TP_;
  static constexpr int W = W_;
  static constexpr int THREADS = 256;
  static constexpr int NP = TP + 10;  // points incl. a halo of 5 each side
  static constexpr int NI = TP + 5;   // interfaces i+1/2, i = s0-3 .. s0+TP+1
  static constexpr int OFF_Q = 0;                       // [9][NP*W] u_0..u_4, f_1..f_4
  static constexpr int OFF_RI = OFF_Q + 9 * NP * W;     // [6][NP*W] sqrt(rho), u, v, w, H, p
  static constexpr int OFF_L = OFF_RI + 6 * NP * W;     // [5][NP*W] lambda
  static constexpr int OFF_REC = OFF_L + 5 * NP * W;    // [18][NI*W] left/right values
  static constexpr int OFF_RD = OFF_REC + 18 * NI * W;  // [15][NI*W] adjoint of du; Roe-state adjoints a, b
  static constexpr int OFF_WC = OFF_RD + 15 * NI * W;   // [9][6][NI*W] weights, then contributions
  static constexpr int WORDS = OFF_WC + 54 * NI * W;
  static constexpr int BYTES = WORDS * 8;
};

constexpr int ADJ_TP = 16, ADJ_W = 4;
using APL = AdjPlan<ADJ_TP, ADJ_W>;

// Smoothness terms of the three windows of a left-biased stencil q0..q4:
// s_k (second difference), v_k (first-derivative combination), b_k = 4 eps + 13/3 s^2 + v^2.
struct Windows {
  double s[3], v[3], b[3];
};

__device__ __forceinline__ Windows windows(double q0, double q1, double q2, double q3, double q4, double eps4) {
  Windows w;
  const double g0 = q1 - q0, g1 = q2 - q1, g2 = q3 - q2, g3 = q4 - q3;
  w.s[0] = g1 - g0;
  w.s[1] = g2 - g1;
  w.s[2] = g3 - g2;
  w.v[0] = fma(3.0, g1, -g0);  // q0 - 4 q1 + 3 q2
  w.v[1] = g1 + g2;            // q3 - q1
  w.v[2] = fma(-3.0, g2, g3);  // 3 q2 - 4 q3 + q4
#pragma unroll
  for (int k = 0; k < 3; ++k) w.b[k] = fma(w.v[k], w.v[k], fma((13.0 / 3.0) * w.s[k], w.s[k], eps4));
  return w;
}

__device__ __forceinline__ void candidates(double q0, double q1, double q2, double q3, double q4, double c[3]) {
  c[0] = fma(11.0 / 6.0, q2, fma(-7.0 / 6.0, q1, (1.0 / 3.0) * q0));
  c[1] = fma(1.0 / 3.0, q3, fma(5.0 / 6.0, q2, (-1.0 / 6.0) * q1));
  c[2] = fma(-1.0 / 6.0, q4, fma(5.0 / 6.0, q3, (1.0 / 3.0) * q2));
}

// WENO5 value and weights of the stencil q0..q4 (value at the interface right of q2).
__device__ __forceinline__ double weno_value(double q0, double q1, double q2, double q3, double q4, double eps4,
                                             double om[3]) {
  const Windows w = windows(q0, q1, q2, q3, q4, eps4);
  double c[3];
  candidates(q0, q1, q2, q3, q4, c);
  const double B0 = w.b[0] * w.b[0], B1 = w.b[1] * w.b[1], B2 = w.b[2] * w.b[2];
  const double a0 = B1 * B2, a1 = 6.0 * (B0 * B2), a2 = 3.0 * (B0 * B1);
  const double r = 1.0 / (a0 + a1 + a2);
  om[0] = a0 * r;
  om[1] = a1 * r;
  om[2] = a2 * r;
  return fma(om[0], c[0], fma(om[1], c[1], om[2] * c[2]));
}

// Adjoint of one reconstruction: out[t] = y * d(value)/d(q_t), t = 0..4.
__device__ __forceinline__ void weno_adjoint(double q0, double q1, double q2, double q3, double q4, double eps4,
                                             const double om[3], double val, double y, double out[5]) {
  const Windows w = windows(q0, q1, q2, q3, q4, eps4);
  double c[3];
  candidates(q0, q1, q2, q3, q4, c);
  const double y0 = y * om[0], y1 = y * om[1], y2 = y * om[2];
  out[0] = (1.0 / 3.0) * y0;
  out[1] = fma(-7.0 / 6.0, y0, (-1.0 / 6.0) * y1);
  out[2] = fma(11.0 / 6.0, y0, fma(5.0 / 6.0, y1, (1.0 / 3.0) * y2));
  out[3] = fma(1.0 / 3.0, y1, (5.0 / 6.0) * y2);
  out[4] = (-1.0 / 6.0) * y2;
  // adjoint of b_k: -2 y omega_k (q_k - val) / b_k, with one division for the three
  const double rb = 1.0 / (w.b[0] * w.b[1] * w.b[2]);
  const double ib0 = (w.b[1] * w.b[2]) * rb, ib1 = (w.b[0] * w.b[2]) * rb, ib2 = (w.b[0] * w.b[1]) * rb;
  const double k0 = -2.0 * y0 * (c[0] - val) * ib0;
  const double k1 = -2.0 * y1 * (c[1] - val) * ib1;
  const double k2 = -2.0 * y2 * (c[2] - val) * ib2;
  // db/d(x, y, z) of a window = 26/3 s (1, -2, 1) + 2 v dv/d(x, y, z)
  double t = (26.0 / 3.0) * w.s[0] * k0, r = 2.0 * w.v[0] * k0;  // dv = (1, -4, 3)
  out[0] += t + r;
  out[1] += fma(-2.0, t, -4.0 * r);
  out[2] += fma(3.0, r, t);
  t = (26.0 / 3.0) * w.s[1] * k1;
  r = 2.0 * w.v[1] * k1;  // dv = (-1, 0, 1)
  out[1] += t - r;
  out[2] += -2.0 * t;
  out[3] += t + r;
  t = (26.0 / 3.0) * w.s[2] * k2;
  r = 2.0 * w.v[2] * k2;  // dv = (3, -4, 1)
  out[2] += fma(3.0, r, t);
  out[3] += fma(-2.0, t, -4.0 * r);
  out[4] += t + r;
}

// |lambda| with Harten's fix (acoustic fields): value and derivatives d/dlambda, d/ddelta.
template <bool FAST>
__device__ __forceinline__ double harten(double lam, double delta, double& dl, double& dd) {
  const double a = fabs(lam);
  if (a < delta) {
    const double rd = FAST ? rcp_newton(delta) : 1.0 / delta;
    dl = lam * rd;
    dd = 0.5 - 0.5 * (lam * rd) * (lam * rd);
    return 0.5 * (lam * lam + delta * delta) * rd;
  }
  dl = (lam > 0.0) ? 1.0 : (lam < 0.0 ? -1.0 : 0.0);
  dd = 0.0;
  return a;
}

// Adjoint of the Roe flux at one interface (Sec. 2.2, Eq. Roe, with the wave-strength
// algebra of the forward pass): given du = u^R - u^L, Lh = adjoint of the interface flux,
// and the two point states a = i, b = i+1 (sqrt(rho), velocity, H, rho, e), returns
// dub = adjoint of du and ga, gb = adjoint of the conserved states a, b through the Roe
// average.  FAST: FP32-seeded Newton reciprocals instead of IEEE division and square
// root (FP64-accurate).  Returns 1 for a non-physical Roe state, 2 for values outside the
// range of the Newton seeds.
template <int D, bool FAST>
__device__ __forceinline__ int roe_adjoint(const double du[5], const double Lh[5], double ra, double rb,
                                           const double Va[3], const double Vb[3], double Ha, double Hb,
                                           double rho_a, double e_a, double rho_b, double e_b, double gamma,
                                           double hdelta, double dub[5], double ga[5], double gb[5]) {
  constexpr int T1 = (D == 0) ? 1 : 0;
  constexpr int T2 = (D == 2) ? 1 : 2;
  const double gm1 = gamma - 1.0;
  const double rsum = ra + rb;
  const double rs = FAST ? rcp_newton(rsum) : 1.0 / rsum;
  const double wa = ra * rs, wb = rb * rs;
  double V[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) V[m] = fma(wa, Va[m], wb * Vb[m]);
  const double H = fma(wa, Ha, wb * Hb);
  const double q2h = 0.5 * fma(V[0], V[0], fma(V[1], V[1], V[2] * V[2]));
  const double c2 = gm1 * (H - q2h);
  int flags = !(c2 > 0.0) ? 1 : 0;
  double c, rc;
  if (FAST) {
    // the float seeds of the Newton reciprocals need these inside the float range
    flags |= (c2 > 1e-36 && c2 < 1e36 && rsum > 1e-36 && rsum < 1e36 && rho_a > 1e-36 && rho_a < 1e36 &&
              rho_b > 1e-36 && rho_b < 1e36) ? 0 : 2;
    rc = rsqrt_newton(c2);
    c = c2 * rc;
  } else {
    c = sqrt(c2);
    rc = 1.0 / c;
  }
  const double un = V[D], vt1 = V[T1], vt2 = V[T2];
  const double b1 = gm1 * (rc * rc);
  const double vdm = fma(V[0], du[1], fma(V[1], du[2], V[2] * du[3]));
  const double Y = fma(q2h, du[0], du[4]) - vdm;
  const double phi = b1 * Y;
  const double X = fma(un, du[0], -du[1 + D]);
  const double ach = 0.5 * (X * rc);
  const double a2 = du[0] - phi;
  const double a3 = fma(-vt1, du[0], du[1 + T1]);
  const double a4 = fma(-vt2, du[0], du[1 + T2]);
  const double a1 = 0.5 * phi + ach, a5 = 0.5 * phi - ach;
  const double delta = hdelta * c;
  double dl1, dd1, dl5, dd5;
  const double l1 = harten<FAST>(un - c, delta, dl1, dd1);
  const double l5 = harten<FAST>(un + c, delta, dl5, dd5);
  const double l2 = fabs(un);
  const double sg2 = (un > 0.0) ? 1.0 : (un < 0.0 ? -1.0 : 0.0);
  const double A1 = l1 * a1, A2 = l2 * a2, A3 = l2 * a3, A4 = l2 * a4, A5 = l5 * a5;
  const double S = A1 + A5, d0 = S + A2, cD = c * (A5 - A1);
  // backward: Dbar = adjoint of the dissipation vector = -Lhat/2
  double Db[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Db[v] = -0.5 * Lh[v];
  const double d0b = fma(Db[1 + D], un, fma(Db[1 + T1], vt1, fma(Db[1 + T2], vt2, Db[0])));
  const double cDb = fma(Db[4], un, Db[1 + D]);
  const double Sb = fma(Db[4], H, d0b);
  const double A2b = fma(Db[4], q2h, d0b);
  const double A3b = fma(Db[4], vt1, Db[1 + T1]);
  const double A4b = fma(Db[4], vt2, Db[1 + T2]);
  const double A1b = fma(-c, cDb, Sb), A5b = fma(c, cDb, Sb);
  double unb = fma(Db[1 + D], d0, Db[4] * cD);
  double vt1b = fma(Db[1 + T1], d0, Db[4] * A3);
  double vt2b = fma(Db[1 + T2], d0, Db[4] * A4);
  double Hbar = Db[4] * S;
  double q2hb = Db[4] * A2;
  double cb = cDb * (A5 - A1);
  // A_k = l_k a_k
  const double a1b = A1b * l1, a2b = A2b * l2, a3b = A3b * l2, a4b = A4b * l2, a5b = A5b * l5;
  const double l1b = A1b * a1, l5b = A5b * a5;
  const double l2b = fma(A2b, a2, fma(A3b, a3, A4b * a4));
  unb = fma(dl1, l1b, fma(dl5, l5b, fma(sg2, l2b, unb)));
  cb = fma(-dl1, l1b, fma(dl5, l5b, fma(hdelta, fma(dd1, l1b, dd5 * l5b), cb)));
  // wave strengths
  const double phib = fma(0.5, a1b + a5b, -a2b);
  const double achb = a1b - a5b;
  dub[0] = fma(-vt1, a3b, fma(-vt2, a4b, a2b));
  dub[1 + T1] = a3b;
  dub[1 + T2] = a4b;
  dub[1 + D] = 0.0;
  dub[4] = 0.0;
  vt1b = fma(-a3b, du[0], vt1b);
  vt2b = fma(-a4b, du[0], vt2b);
  const double Xb = 0.5 * rc * achb;
  double rcb = 0.5 * X * achb;
  unb = fma(Xb, du[0], unb);
  dub[0] = fma(Xb, un, dub[0]);
  dub[1 + D] -= Xb;
  const double b1b = phib * Y;
  const double Yb = phib * b1;
  q2hb = fma(Yb, du[0], q2hb);
  dub[0] = fma(Yb, q2h, dub[0]);
  dub[4] += Yb;
  double Vbar[3];
  Vbar[D] = unb;
  Vbar[T1] = vt1b;
  Vbar[T2] = vt2b;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    Vbar[m] = fma(-Yb, du[1 + m], Vbar[m]);  // vdm = V . du_m
    dub[1 + m] = fma(-Yb, V[m], dub[1 + m]);
  }
  rcb = fma(b1b, 2.0 * gm1 * rc, rcb);
  cb = fma(-rcb, rc * rc, cb);
  // c = sqrt(gm1 (H - q2h))
  const double c2b = 0.5 * cb * rc;
  Hbar = fma(gm1, c2b, Hbar);
  q2hb = fma(-gm1, c2b, q2hb);
#pragma unroll
  for (int m = 0; m < 3; ++m) Vbar[m] = fma(q2hb, V[m], Vbar[m]);
  // Roe average of the point states a, b
  double rab = Hbar * (Ha - H), rbb = Hbar * (Hb - H);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    rab = fma(Vbar[m], Va[m] - V[m], rab);
    rbb = fma(Vbar[m], Vb[m] - V[m], rbb);
  }
  rab *= rs;
  rbb *= rs;
  // point primitives: V = m/rho, H = gamma e/rho - gm1 |V|^2/2, sqrt(rho)
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const double wgt = side ? wb : wa;
    const double* Vp = side ? Vb : Va;
    const double rho = side ? rho_b : rho_a, e = side ? e_b : e_a, sr = side ? rb : ra;
    const double rr = FAST ? rcp_newton(rho) : 1.0 / rho;
    const double Hb_ = wgt * Hbar;
    const double srb = side ? rbb : rab;
    double Vt[3], vdot = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      Vt[m] = fma(-Hb_ * gm1, Vp[m], wgt * Vbar[m]);
      vdot = fma(Vt[m], Vp[m], vdot);
    }
    double* gs = side ? gb : ga;
    gs[4] = Hb_ * gamma * rr;
    // d sqrt(rho)/d rho = 1/(2 sqrt(rho)) = sqrt(rho) / (2 rho)
    gs[0] = fma(0.5 * srb, sr * rr, -fma(Hb_ * gamma, e * rr, vdot) * rr);
#pragma unroll
    for (int m = 0; m < 3; ++m) gs[1 + m] = Vt[m] * rr;
  }
  return flags;
}

__device__ __forceinline__ void adj_epilogue(const AdjArgs& a, long long p, const double cv[5]) {
  const long long N = a.g.N;
  switch (a.epi) {
    case AEPI_WRITE:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] = cv[v];
      break;
    case AEPI_ADD:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.k[v * N + p] += cv[v];
      break;
    case AEPI_OUT:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.gout[v * N + p] = a.k[v * N + p] + cv[v];
      break;
    case AEPI_RK4_4:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v], ub = a.ubs[v * N + p];
        a.gout[v * N + p] = ub + K;
        a.lnext[v * N + p] = fma(a.c1, ub, a.c2 * K);
      }
      break;
    case AEPI_RK4_M:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v], ub = a.ubs[v * N + p];
        a.gout[v * N + p] += K;
        a.lnext[v * N + p] = fma(a.c1, ub, a.c2 * K);
      }
      break;
    case AEPI_ACC:
#pragma unroll
      for (int v = 0; v < 5; ++v) a.gout[v * N + p] += a.k[v * N + p] + cv[v];
      break;
    case AEPI_SSP_3:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v], ub = a.ubs[v * N + p];
        const double s = fma(2.0 / 3.0, ub, K);
        a.gout[v * N + p] = fma(1.0 / 3.0, ub, 0.75 * s);
        a.lnext[v * N + p] = (0.25 * a.c2) * s;
        a.sb[v * N + p] = 0.25 * s;
      }
      break;
    case AEPI_SSP_2:
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double K = a.k[v * N + p] + cv[v];
        const double s = a.sb[v * N + p] + K;
        a.gout[v * N + p] += s;
        a.lnext[v * N + p] = a.c2 * s;
      }
      break;
    default:
      break;
  }
}

template <int D>
__global__ void __launch_bounds__(APL::THREADS, 2) k_adj_dir(const AdjArgs a) {
  extern __shared__ double sm[];
  constexpr int TP = APL::TP, NP = APL::NP, NI = APL::NI, W = APL::W;
  constexpr int AX = (D == 0) ? 1 : 0;
  const int nD = a.g.n[D];
  const int na = a.g.n[AX];
  const long long N = a.g.N;
  const int s0 = blockIdx.x * TP;
  const int a0 = blockIdx.y * W;
  const int bz = blockIdx.z;
  const int tid = threadIdx.x;
  const double rdx = a.g.rh[D];
  const double gm1 = a.gamma - 1.0;
  double* q = sm + APL::OFF_Q;
  double* ri = sm + APL::OFF_RI;
  double* lm = sm + APL::OFF_L;
  double* rec = sm + APL::OFF_REC;
  double* rd = sm + APL::OFF_RD;
  double* wc = sm + APL::OFF_WC;

  // ---- A: load -------------------------------------------------------------------
  for (int item = tid; item < NP * W; item += APL::THREADS) {
    int pos, line;
    tile_split<D, W>(item, NP, pos, line);
    const int c = wrap_idx(s0 - 5 + pos, nD);
    const int la = min(a0 + line, na - 1);
    const long long p = tile_flat<D>(a.g, c, la, bz);
    double U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.u + v * N + p);
    const double vx = __ldg(a.pm + PM_U * N + p), vy = __ldg(a.pm + PM_V * N + p), vz = __ldg(a.pm + PM_W * N + p);
    const double pr = __ldg(a.pm + PM_P * N + p);
    const double un = (D == 0) ? vx : (D == 1) ? vy : vz;
    const int s = tile_idx<D, W>(pos, line, NP);
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v * NP * W + s] = U[v];
    q[5 * NP * W + s] = (D == 0) ? fma(U[1], un, pr) : U[1] * un;
    q[6 * NP * W + s] = (D == 1) ? fma(U[2], un, pr) : U[2] * un;
    q[7 * NP * W + s] = (D == 2) ? fma(U[3], un, pr) : U[3] * un;
    q[8 * NP * W + s] = (U[4] + pr) * un;
    ri[0 * NP * W + s] = __ldg(a.pm + PM_SR * N + p);
    ri[1 * NP * W + s] = vx;
    ri[2 * NP * W + s] = vy;
    ri[3 * NP * W + s] = vz;
    ri[4 * NP * W + s] = __ldg(a.pm + PM_H * N + p);
    ri[5 * NP * W + s] = pr;
#pragma unroll
    for (int v = 0; v < 5; ++v) lm[v * NP * W + s] = a.lam_scale * __ldg(a.lam + v * N + p);
  }
  __syncthreads();

  // ---- C: values and weights of the left/right reconstructions -----------------------
  for (int item = tid; item < 9 * NI * W; item += APL::THREADS) {
    const int m = item / (NI * W);
    int f, line;
    tile_split<D, W>(item - m * NI * W, NI, f, line);
    const double* qm = q + m * NP * W;
    double P[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) P[j] = qm[tile_idx<D, W>(f + j, line, NP)];
    double wL[3], wR[3];
    const double vL = weno_value(P[0], P[1], P[2], P[3], P[4], a.eps4, wL);
    const double vR = weno_value(P[5], P[4], P[3], P[2], P[1], a.eps4, wR);
    const int o = tile_idx<D, W>(f, line, NI);
    rec[(2 * m) * NI * W + o] = vL;
    rec[(2 * m + 1) * NI * W + o] = vR;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wc[(m * 6 + k) * NI * W + o] = wL[k];
      wc[(m * 6 + 3 + k) * NI * W + o] = wR[k];
    }
  }
  __syncthreads();

  // ---- D: adjoint of the Roe flux at every interface --------------------------------------
  {
    int bad = 0;
    for (int item = tid; item < NI * W; item += APL::THREADS) {
      int f, line;
      tile_split<D, W>(item, NI, f, line);
      const int o = tile_idx<D, W>(f, line, NI);
      const int sa = tile_idx<D, W>(f + 2, line, NP), sb = tile_idx<D, W>(f + 3, line, NP);
      double du[5], Lh[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        du[v] = rec[(2 * v + 1) * NI * W + o] - rec[(2 * v) * NI * W + o];
        Lh[v] = (lm[v * NP * W + sb] - lm[v * NP * W + sa]) * rdx;
      }
      double Va[3], Vb[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Va[m] = ri[(1 + m) * NP * W + sa];
        Vb[m] = ri[(1 + m) * NP * W + sb];
      }
      double dub[5], ga[5], gb[5];
      bad |= roe_adjoint<D, false>(du, Lh, ri[sa], ri[sb], Va, Vb, ri[4 * NP * W + sa], ri[4 * NP * W + sb], q[sa],
                                   q[4 * NP * W + sa], q[sb], q[4 * NP * W + sb], a.gamma, a.hdelta, dub, ga, gb);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        rd[(5 + v) * NI * W + o] = ga[v];
        rd[(10 + v) * NI * W + o] = gb[v];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) rd[v * NI * W + o] = dub[v];
    }
    if (__any_sync(0xffffffffu, bad & 1) && (tid & 31) == 0) atomicOr(a.status, ST_NONPHYS);
  }
  __syncthreads();

  // ---- E: adjoints of the reconstructions -> stencil contributions --------------------
  for (int item = tid; item < 9 * NI * W; item += APL::THREADS) {
    const int m = item / (NI * W);
    int f, line;
    tile_split<D, W>(item - m * NI * W, NI, f, line);
    const int o = tile_idx<D, W>(f, line, NI);
    const int sa = tile_idx<D, W>(f + 2, line, NP), sb = tile_idx<D, W>(f + 3, line, NP);
    double yL, yR;
    if (m < 5) {
      const double g = rd[m * NI * W + o];
      yL = -g;
      yR = g;
      if (m == 1 + D) {  // mass flux f_0 = u_{1+D}: (f^L + f^R)/2 part
        const double h0 = 0.5 * ((lm[sb] - lm[sa]) * rdx);
        yL += h0;
        yR += h0;
      }
    } else {
      const double hm = 0.5 * ((lm[(m - 4) * NP * W + sb] - lm[(m - 4) * NP * W + sa]) * rdx);
      yL = hm;
      yR = hm;
    }
    const double* qm = q + m * NP * W;
    double P[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) P[j] = qm[tile_idx<D, W>(f + j, line, NP)];
    double wL[3], wR[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wL[k] = wc[(m * 6 + k) * NI * W + o];
      wR[k] = wc[(m * 6 + 3 + k) * NI * W + o];
    }
    const double vL = rec[(2 * m) * NI * W + o], vR = rec[(2 * m + 1) * NI * W + o];
    double cL[5], cR[5];
    weno_adjoint(P[0], P[1], P[2], P[3], P[4], a.eps4, wL, vL, yL, cL);
    weno_adjoint(P[5], P[4], P[3], P[2], P[1], a.eps4, wR, vR, yR, cR);
    // position f + j: left stencil index j, right stencil index 5 - j
    wc[(m * 6 + 0) * NI * W + o] = cL[0];
#pragma unroll
    for (int j = 1; j < 5; ++j) wc[(m * 6 + j) * NI * W + o] = cL[j] + cR[5 - j];
    wc[(m * 6 + 5) * NI * W + o] = cR[0];
  }
  __syncthreads();

  // ---- F: gather, adjoint of the point fluxes, epilogue ----------------------------------
  for (int item = tid; item < TP * W; item += APL::THREADS) {
    int pp, line;
    tile_split<D, W>(item, TP, pp, line);
    if (s0 + pp >= nD || a0 + line >= na) continue;
    const int pos = pp + 5;
    double g[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < 6; ++j) acc += wc[(m * 6 + j) * NI * W + tile_idx<D, W>(pos - j, line, NI)];
      g[m] = acc;
    }
    const int oa = tile_idx<D, W>(pos - 2, line, NI), ob = tile_idx<D, W>(pos - 3, line, NI);
    double cv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) cv[v] = g[v] + (rd[(5 + v) * NI * W + oa] + rd[(10 + v) * NI * W + ob]);
    // f_{1+k} = m_k u_D + [k = D] p, f_4 = (e + p) u_D
    const int s = tile_idx<D, W>(pos, line, NP);
    const double rho = q[s], e = q[4 * NP * W + s], pr = ri[5 * NP * W + s];
    const double V[3] = {ri[1 * NP * W + s], ri[2 * NP * W + s], ri[3 * NP * W + s]};
    const double un = V[D];
    const double Fb1 = g[5], Fb2 = g[6], Fb3 = g[7], Fb4 = g[8];
    const double Fbm[3] = {Fb1, Fb2, Fb3};
    const double pb = fma(Fb4, un, Fbm[D]);
    double unb = Fb4 * (e + pr);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unb = fma(Fbm[k], q[(1 + k) * NP * W + s], unb);
      cv[1 + k] = fma(Fbm[k], un, cv[1 + k]);
    }
    cv[4] = fma(Fb4, un, cv[4]);
    const double rr = 1.0 / rho;
    cv[1 + D] = fma(unb, rr, cv[1 + D]);
    cv[0] = fma(-unb * un, rr, cv[0]);
    const double gp = gm1 * pb;
    cv[4] += gp;
    double v2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cv[1 + k] = fma(-gp, V[k], cv[1 + k]);
      v2 = fma(V[k], V[k], v2);
    }
    cv[0] = fma(0.5 * gp, v2, cv[0]);
    const long long p = tile_flat<D>(a.g, s0 + pp, a0 + line, bz);
    adj_epilogue(a, p, cv);
  }
}


// ============================================================================================
// NS3D_FP64 form: the reconstruction adjoints in double-float arithmetic on the FP32 pipe.
// Everything the WENO5 derivative needs is a function of the first differences g_j of the
// data: s_k (second differences), v_k, b_k = 4 eps + 13/3 s_k^2 + v_k^2, the weights, the
// candidate differences q_0 - q_1 = (s_0 - s_1)/3 and q_2 - q_1 = (s_1 - s_2)/6, and
// q_k - q = (q_k - q_1) - M with M = omega_0 (q_0 - q_1) + omega_2 (q_2 - q_1).  The value
// itself is q = P_c + (2 g_2 + g_1)/6 + M (P_c the stencil centre), the same offset form as
// the forward pass.  The Roe-flux adjoint is double-float too (one interface per item); the
// window terms, weights, reconstruction adjoints and the per-point gather take the tile's two
// lines at once with the packed FP32 instructions (df2.cuh).  The per-point sums of the
// reconstruction contributions are converted back to FP64 once.  To keep double-float values inside the float range whatever the scale of
// the adjoint input, each tile divides lambda by the power of two of its largest magnitude
// and multiplies its results back (exact).
// ============================================================================================
template <int TP_, int W_, int THREADS_, int MIN_CTAS_>
struct AdjPlanDF {
  static constexpr int TP = TP_;
  static constexpr int W = W_;
  static constexpr int THREADS = THREADS_;
  static constexpr int MIN_CTAS = MIN_CTAS_;
  static constexpr int NP = TP + 10;  // points incl. a halo of 5 each side
  static constexpr int NI = TP + 5;   // interfaces
  static constexpr int NW = TP + 8;   // 3-point windows starting at 0 .. NW-1
  static constexpr int OFF_Q = 0;                        // [9][NP*W] doubles
  static constexpr int OFF_RI = OFF_Q + 9 * NP * W;      // [8][NP*W] double-float sqrt(rho), u, v, w, H;
                                                         //   FP64 p; double-float rho, e
  static constexpr int OFF_L = OFF_RI + 8 * NP * W;      // [5][NP*W] lambda / 2^E
  static constexpr int OFF_G = OFF_L + 5 * NP * W;       // [9][NP] first differences of both lines
  static constexpr int OFF_B = OFF_G + 9 * NP * W;       // [9][3][NW] 1/b_k of every window, both lines
  static constexpr int OFF_REC = OFF_B + 27 * NW * W;    // [10][NI*W] doubles: u^L, u^R of u_0..u_4
  static constexpr int OFF_RD = OFF_REC + 10 * NI * W;   // [15][NI*W] double-float Roe adjoints
  static constexpr int OFF_WC = OFF_RD + 15 * NI * W;    // [9][6][NI] stencil contributions, both lines
  static constexpr int WORDS = OFF_WC + 54 * NI * W;
  static constexpr int BYTES = WORDS * 8;
};
using APF = AdjPlanDF<32, 2, 256, 2>;

__device__ __forceinline__ df df_sub(df x, df y) { return df_add_fast(x, df_neg(y)); }
__device__ __forceinline__ float2 df_pack(df x) { return make_float2(x.hi, x.lo); }
__device__ __forceinline__ df df_unpack(float2 v) { return df{v.x, v.y}; }

struct DFConst {
  df third, sixth, c263;  // 1/3, 1/6, 26/3
};

// The WENO pieces below take the two lines of a tile at once (two-lane double-float,
// df2.cuh: each lane computes what one line would).
// Products and positive sums in this section are left unnormalised where they feed another
// double-float operation (df2_mul_u and friends: the same values, |lo| a few ulp(hi)).
struct DF2Const {
  df2 third, sixth, c263;
};
__device__ __forceinline__ df2 df2_sub(df2 x, df2 y) { return df2_add_fast(x, df2_neg(y)); }

// The three weights of one reconstruction from the reciprocals r_k = 1/b_k of its window
// terms (candidate order 0, 1, 2; optimal weights 1, 6, 3 over 10):
// omega_k = c_k r_k^2 / sum_j c_j r_j^2.  With the window terms' range checked (b <= 1e18,
// b >= 4 eps), r^2 stays inside the float range and needs no rescaling.
__device__ __forceinline__ void df2_omega(df2 r0, df2 r1, df2 r2, df2 om[3]) {
  const df2 a0 = df2_sqr_u(r0);
  const df2 a1 = df2_mul_f_u(df2_sqr_u(r1), 6.0f);
  const df2 a2 = df2_mul_f_u(df2_sqr_u(r2), 3.0f);
  const df2 r = df2_div(df2{f2splat(1.0f), f2splat(0.0f)}, df2_add_pos_u(a0, df2_add_pos_u(a1, a2)));
  om[0] = df2_mul_u(a0, r);
  om[1] = df2_mul_u(a1, r);
  om[2] = df2_mul_u(a2, r);
}

// Offset M of the reconstruction from its candidate 1, and the candidate differences.
__device__ __forceinline__ df2 df2_adj_offset(df2 g0, df2 g1, df2 g2, df2 g3, const df2 om[3], const DF2Const& k,
                                              df2& E0, df2& E2, df2 s[3]) {
  s[0] = df2_sub(g1, g0);
  s[1] = df2_sub(g2, g1);
  s[2] = df2_sub(g3, g2);
  E0 = df2_mul_u(df2_sub(s[0], s[1]), k.third);
  E2 = df2_mul_u(df2_sub(s[1], s[2]), k.sixth);
  return df2_add_fast(df2_mul_u(om[0], E0), df2_mul_u(om[2], E2));
}

// y * d(value)/d(q_t), t = 0..4, of the reconstruction of stencil differences g0..g3 with
// the reciprocals rb0..rb2 of its window terms and weights om (as weno_adjoint, in
// double-float).
__device__ __forceinline__ void df2_recon_adjoint(df2 g0, df2 g1, df2 g2, df2 g3, df2 rb0, df2 rb1, df2 rb2,
                                                  const df2 om[3], df2 y, const DF2Const& k, df2 out[5]) {
  df2 s[3], E0, E2;
  const df2 M = df2_adj_offset(g0, g1, g2, g3, om, k, E0, E2, s);
  const df2 v0 = df2_sub(df2_mul_f_u(g1, 3.0f), g0);
  const df2 v1 = df2_add_fast(g1, g2);
  const df2 v2 = df2_sub(g3, df2_mul_f_u(g2, 3.0f));
  const df2 y0 = df2_mul_u(y, om[0]), y1 = df2_mul_u(y, om[1]), y2 = df2_mul_u(y, om[2]);
  // adjoints of b_k: -2 y_k (q_k - q) / b_k with q_0 - q = E0 - M, q_1 - q = -M, q_2 - q = E2 - M
  const df2 k0 = df2_twice(df2_mul(df2_mul_u(y0, df2_sub(M, E0)), rb0));
  const df2 k1 = df2_twice(df2_mul(df2_mul_u(y1, M), rb1));
  const df2 k2 = df2_twice(df2_mul(df2_mul_u(y2, df2_sub(M, E2)), rb2));
  // direct term sum_k y_k dq_k/dq_t
  out[0] = df2_mul_u(y0, k.third);
  out[1] = df2_neg(df2_mul_u(df2_add_fast(df2_mul_f_u(y0, 7.0f), y1), k.sixth));
  out[2] = df2_mul_u(df2_add_fast(df2_mul_f_u(y0, 11.0f), df2_add_fast(df2_mul_f_u(y1, 5.0f), df2_twice(y2))), k.sixth);
  out[3] = df2_mul_u(df2_add_fast(df2_twice(y1), df2_mul_f_u(y2, 5.0f)), k.sixth);
  out[4] = df2_neg(df2_mul_u(y2, k.sixth));
  // db/d(x, y, z) of a window = 26/3 s (1, -2, 1) + 2 v dv/d(x, y, z)
  df2 t = df2_mul_u(df2_mul_u(s[0], k0), k.c263), r = df2_twice(df2_mul_u(v0, k0));  // dv = (1, -4, 3)
  out[0] = df2_add_fast(out[0], df2_add_fast(t, r));
  out[1] = df2_sub(out[1], df2_add_fast(df2_twice(t), df2_twice(df2_twice(r))));
  out[2] = df2_add_fast(out[2], df2_add_fast(t, df2_mul_f_u(r, 3.0f)));
  t = df2_mul_u(df2_mul_u(s[1], k1), k.c263);
  r = df2_twice(df2_mul_u(v1, k1));  // dv = (-1, 0, 1)
  out[1] = df2_add_fast(out[1], df2_sub(t, r));
  out[2] = df2_sub(out[2], df2_twice(t));
  out[3] = df2_add_fast(out[3], df2_add_fast(t, r));
  t = df2_mul_u(df2_mul_u(s[2], k2), k.c263);
  r = df2_twice(df2_mul_u(v2, k2));  // dv = (3, -4, 1)
  out[2] = df2_add_fast(out[2], df2_add_fast(t, df2_mul_f_u(r, 3.0f)));
  out[3] = df2_sub(out[3], df2_add_fast(df2_twice(t), df2_twice(df2_twice(r))));
  out[4] = df2_add_fast(out[4], df2_add_fast(t, r));
}

__device__ __forceinline__ double pow2d(int k) { return __hiloint2double((k + 1023) << 20, 0); }

__device__ __forceinline__ df df_half(df x) { return df{0.5f * x.hi, 0.5f * x.lo}; }
// a * b + c with an unnormalised product (normalised result)
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add_fast(df_mul_u(a, b), c); }

// |lambda| with Harten's fix in double-float (harten<> in FP64): value, d/dlambda, d/ddelta.
__device__ __forceinline__ df harten_df(df lam, df delta, df& dl, df& dd) {
  const df a = df_abs(lam);
  if (df_lt(a, delta)) {
    const df rd = df_div(df{1.0f, 0.0f}, delta);
    const df lr = df_mul(lam, rd);
    dl = lr;
    dd = df_sub(df{0.5f, 0.0f}, df_half(df_sqr(lr)));
    return df_half(df_mul(df_add_pos(df_sqr(lam), df_sqr(delta)), rd));
  }
  dl = df{(lam.hi > 0.0f) ? 1.0f : ((lam.hi < 0.0f) ? -1.0f : 0.0f), 0.0f};
  dd = df{0.0f, 0.0f};
  return a;
}

// Adjoint of the Roe flux at one interface in double-float arithmetic on the FP32 pipe: the
// algebra of roe_adjoint (Sec. 2.2, Eq. Roe, wave strengths, Harten's fix, Roe average of the
// grid-point states a = i, b = i+1), every quantity as a double-float (~48 bits) instead of
// FP64.  du: the jump of the conserved reconstructions, Lh: the adjoint of the interface flux;
// returns dub (adjoint of du) and ga, gb (adjoints of the two conserved point states).  Returns
// 1 for a non-physical Roe state, 2 for values outside the float range of the double-float
// arithmetic.
template <int D>
__device__ __forceinline__ int roe_adjoint_df(const df du[5], const df Lh[5], df ra, df rb, const df Va[3],
                                              const df Vb[3], df Ha, df Hb, df rho_a, df e_a, df rho_b, df e_b,
                                              df gamma, df gm1, df hdelta, df dub[5], df ga[5], df gb[5]) {
  constexpr int T1 = (D == 0) ? 1 : 0;
  constexpr int T2 = (D == 2) ? 1 : 2;
  const df one{1.0f, 0.0f}, zero{0.0f, 0.0f};
  const df rsum = df_add_pos(ra, rb);
  const df rs = df_div(one, rsum);
  const df wa = df_mul(ra, rs), wb = df_mul(rb, rs);
  df V[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) V[m] = df_add_fast(df_mul_u(wa, Va[m]), df_mul_u(wb, Vb[m]));
  const df H = df_add_pos(df_mul_u(wa, Ha), df_mul_u(wb, Hb));
  const df q2 = df_add_pos_u(df_sqr_u(V[0]), df_add_pos_u(df_sqr_u(V[1]), df_sqr_u(V[2])));
  const df q2h = fast_two_sum(0.5f * q2.hi, 0.5f * q2.lo);
  const df c2 = df_mul(df_sub(H, q2h), gm1);
  int flags = (c2.hi > 0.0f) ? 0 : 1;
  flags |= (c2.hi > 1e-30f && c2.hi < 1e30f && rsum.hi > 1e-30f && rsum.hi < 1e30f && rho_a.hi > 1e-30f &&
            rho_a.hi < 1e30f && rho_b.hi > 1e-30f && rho_b.hi < 1e30f && fabsf(H.hi) < 1e30f)
               ? 0
               : 2;
  const df c = df_sqrt(c2);
  const df rc = df_div(one, c);
  const df un = V[D], vt1 = V[T1], vt2 = V[T2];
  const df rc2 = df_sqr(rc);
  const df b1 = df_mul(gm1, rc2);
  const df vdm = df_add_fast(df_mul_u(V[0], du[1]), df_add_fast(df_mul_u(V[1], du[2]), df_mul_u(V[2], du[3])));
  const df Y = df_sub(df_fma(q2h, du[0], du[4]), vdm);
  const df phi = df_mul(b1, Y);
  const df X = df_sub(df_mul_u(un, du[0]), du[1 + D]);
  const df ach = df_half(df_mul(X, rc));
  const df a2 = df_sub(du[0], phi);
  const df a3 = df_sub(du[1 + T1], df_mul_u(vt1, du[0]));
  const df a4 = df_sub(du[1 + T2], df_mul_u(vt2, du[0]));
  const df phh = df_half(phi);
  const df a1 = df_add_fast(phh, ach), a5 = df_sub(phh, ach);
  const df delta = df_mul(hdelta, c);
  df dl1, dd1, dl5, dd5;
  const df l1 = harten_df(df_sub(un, c), delta, dl1, dd1);
  const df l5 = harten_df(df_add_fast(un, c), delta, dl5, dd5);
  const df l2 = df_abs(un);
  const float sg2 = (un.hi > 0.0f) ? 1.0f : ((un.hi < 0.0f) ? -1.0f : 0.0f);
  const df A1 = df_mul(l1, a1), A2 = df_mul(l2, a2), A3 = df_mul(l2, a3), A4 = df_mul(l2, a4), A5 = df_mul(l5, a5);
  const df S = df_add_fast(A1, A5), d0 = df_add_fast(S, A2), cD = df_mul(c, df_sub(A5, A1));
  // backward: the adjoint of the dissipation vector is -Lhat/2
  df Db[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) Db[v] = df{-0.5f * Lh[v].hi, -0.5f * Lh[v].lo};
  const df d0b = df_fma(Db[1 + D], un, df_fma(Db[1 + T1], vt1, df_fma(Db[1 + T2], vt2, Db[0])));
  const df cDb = df_fma(Db[4], un, Db[1 + D]);
  const df Sb = df_fma(Db[4], H, d0b);
  const df A2b = df_fma(Db[4], q2h, d0b);
  const df A3b = df_fma(Db[4], vt1, Db[1 + T1]);
  const df A4b = df_fma(Db[4], vt2, Db[1 + T2]);
  const df ccDb = df_mul(c, cDb);
  const df A1b = df_sub(Sb, ccDb), A5b = df_add_fast(Sb, ccDb);
  df unb = df_add_fast(df_mul_u(Db[1 + D], d0), df_mul_u(Db[4], cD));
  df vt1b = df_add_fast(df_mul_u(Db[1 + T1], d0), df_mul_u(Db[4], A3));
  df vt2b = df_add_fast(df_mul_u(Db[1 + T2], d0), df_mul_u(Db[4], A4));
  df Hbar = df_mul(Db[4], S);
  df q2hb = df_mul(Db[4], A2);
  df cb = df_mul(cDb, df_sub(A5, A1));
  // A_k = l_k a_k
  const df a1b = df_mul(A1b, l1), a2b = df_mul(A2b, l2), a3b = df_mul(A3b, l2), a4b = df_mul(A4b, l2);
  const df a5b = df_mul(A5b, l5);
  const df l1b = df_mul(A1b, a1), l5b = df_mul(A5b, a5);
  const df l2b = df_fma(A2b, a2, df_fma(A3b, a3, df_mul_u(A4b, a4)));
  const df t1 = df_mul_u(dl1, l1b), t5 = df_mul_u(dl5, l5b);
  unb = df_add_fast(df_add_fast(t1, t5), df_add_fast(df{sg2 * l2b.hi, sg2 * l2b.lo}, unb));
  cb = df_add_fast(df_add_fast(df_sub(t5, t1), df_mul_u(hdelta, df_fma(dd1, l1b, df_mul_u(dd5, l5b)))), cb);
  // wave strengths
  const df phib = df_sub(df_half(df_add_fast(a1b, a5b)), a2b);
  const df achb = df_sub(a1b, a5b);
  dub[0] = df_sub(a2b, df_add_fast(df_mul_u(vt1, a3b), df_mul_u(vt2, a4b)));
  dub[1 + T1] = a3b;
  dub[1 + T2] = a4b;
  vt1b = df_sub(vt1b, df_mul_u(a3b, du[0]));
  vt2b = df_sub(vt2b, df_mul_u(a4b, du[0]));
  const df Xb = df_half(df_mul(rc, achb));
  df rcb = df_half(df_mul(X, achb));
  unb = df_fma(Xb, du[0], unb);
  dub[0] = df_fma(Xb, un, dub[0]);
  dub[1 + D] = df_neg(Xb);
  const df b1b = df_mul(phib, Y);
  const df Yb = df_mul(phib, b1);
  q2hb = df_fma(Yb, du[0], q2hb);
  dub[0] = df_fma(Yb, q2h, dub[0]);
  dub[4] = Yb;
  df Vbar[3];
  Vbar[D] = unb;
  Vbar[T1] = vt1b;
  Vbar[T2] = vt2b;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    Vbar[m] = df_sub(Vbar[m], df_mul_u(Yb, du[1 + m]));  // vdm = V . du_m
    dub[1 + m] = df_sub(dub[1 + m], df_mul_u(Yb, V[m]));
  }
  rcb = df_fma(b1b, df_twice(df_mul(gm1, rc)), rcb);
  cb = df_sub(cb, df_mul_u(rcb, rc2));
  // c = sqrt(gm1 (H - q2h))
  const df c2b = df_half(df_mul(cb, rc));
  Hbar = df_fma(gm1, c2b, Hbar);
  q2hb = df_sub(q2hb, df_mul_u(gm1, c2b));
#pragma unroll
  for (int m = 0; m < 3; ++m) Vbar[m] = df_fma(q2hb, V[m], Vbar[m]);
  // Roe average of the point states a, b
  df rab = df_mul_u(Hbar, df_sub(Ha, H)), rbb = df_mul_u(Hbar, df_sub(Hb, H));
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    rab = df_fma(Vbar[m], df_sub(Va[m], V[m]), rab);
    rbb = df_fma(Vbar[m], df_sub(Vb[m], V[m]), rbb);
  }
  rab = df_mul(rab, rs);
  rbb = df_mul(rbb, rs);
  // point primitives: V = m/rho, H = gamma e/rho - gm1 |V|^2/2, sqrt(rho)
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const df wgt = side ? wb : wa;
    const df* Vp = side ? Vb : Va;
    const df rho = side ? rho_b : rho_a, e = side ? e_b : e_a, sr = side ? rb : ra;
    const df rr = df_div(one, rho);
    const df Hb_ = df_mul(wgt, Hbar);
    const df gH = df_mul(Hb_, gm1);
    const df srb = side ? rbb : rab;
    df Vt[3], vdot = zero;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      Vt[m] = df_sub(df_mul_u(wgt, Vbar[m]), df_mul_u(gH, Vp[m]));
      vdot = df_fma(Vt[m], Vp[m], vdot);
    }
    df* gs = side ? gb : ga;
    const df Hg = df_mul(Hb_, gamma);
    gs[4] = df_mul(Hg, rr);
    // d sqrt(rho)/d rho = 1/(2 sqrt(rho)) = sqrt(rho) / (2 rho)
    gs[0] = df_sub(df_mul_u(df_half(srb), df_mul(sr, rr)), df_mul_u(df_fma(Hg, df_mul(e, rr), vdot), rr));
#pragma unroll
    for (int m = 0; m < 3; ++m) gs[1 + m] = df_mul(Vt[m], rr);
  }
  return flags;
}

template <int D>
__global__ void __launch_bounds__(APF::THREADS, APF::MIN_CTAS) k_adj_dir_df(const AdjArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_emax;
  constexpr int TP = APF::TP, NP = APF::NP, NI = APF::NI, NW = APF::NW, W = APF::W;
  constexpr int AX = (D == 0) ? 1 : 0;
  const int nD = a.g.n[D];
  const int na = a.g.n[AX];
  const long long N = a.g.N;
  const int s0 = blockIdx.x * TP;
  const int a0 = blockIdx.y * W;
  const int bz = blockIdx.z;
  const int tid = threadIdx.x;
  const double rdx = a.g.rh[D];
  double* q = sm + APF::OFF_Q;
  double* ri = sm + APF::OFF_RI;
  double* lm = sm + APF::OFF_L;
  // G, Bw and wc hold the two lines of the tile side by side (hi0, hi1, lo0, lo1)
  static_assert(W == 2, "the two-lane phases take the tile's two lines together");
  float4* G4 = reinterpret_cast<float4*>(sm + APF::OFF_G);    // [9][NP]
  float4* Bw4 = reinterpret_cast<float4*>(sm + APF::OFF_B);   // [9][3][NW]
  double* rec = sm + APF::OFF_REC;
  double* rd = sm + APF::OFF_RD;
  float4* wc4 = reinterpret_cast<float4*>(sm + APF::OFF_WC);  // [9][6][NI]
  DFConst kc;
  {
    const double third = 1.0 / 3.0, sixth = 1.0 / 6.0, c263 = 26.0 / 3.0;
    kc.third = df{(float)third, (float)(third - (double)(float)third)};
    kc.sixth = df{(float)sixth, (float)(sixth - (double)(float)sixth)};
    kc.c263 = df{(float)c263, (float)(c263 - (double)(float)c263)};
  }
  const DF2Const kc2{df2_splat(kc.third), df2_splat(kc.sixth), df2_splat(kc.c263)};
  const df eps4{(float)a.eps4, (float)(a.eps4 - (double)(float)a.eps4)};
  const df c133{(float)(13.0 / 3.0), (float)(13.0 / 3.0 - (double)(float)(13.0 / 3.0))};
  if (tid == 0) s_emax = -2000;
  __syncthreads();

  // ---- A: load; largest binary exponent of lambda in the tile ----------------------------
  int emax = -2000;
  for (int item = tid; item < NP * W; item += APF::THREADS) {
    int pos, line;
    tile_split<D, W>(item, NP, pos, line);
    const int c = wrap_idx(s0 - 5 + pos, nD);
    const int la = min(a0 + line, na - 1);
    const long long p = tile_flat<D>(a.g, c, la, bz);
    double U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = __ldg(a.u + v * N + p);
    const double vx = __ldg(a.pm + PM_U * N + p), vy = __ldg(a.pm + PM_V * N + p), vz = __ldg(a.pm + PM_W * N + p);
    const double pr = __ldg(a.pm + PM_P * N + p);
    const double un = (D == 0) ? vx : (D == 1) ? vy : vz;
    const int s = tile_idx<D, W>(pos, line, NP);
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v * NP * W + s] = U[v];
    q[5 * NP * W + s] = (D == 0) ? fma(U[1], un, pr) : U[1] * un;
    q[6 * NP * W + s] = (D == 1) ? fma(U[2], un, pr) : U[2] * un;
    q[7 * NP * W + s] = (D == 2) ? fma(U[3], un, pr) : U[3] * un;
    q[8 * NP * W + s] = (U[4] + pr) * un;
    float2* rf = reinterpret_cast<float2*>(ri);
    rf[0 * NP * W + s] = df_pack(d2df_bits(__ldg(a.pm + PM_SR * N + p)));
    rf[1 * NP * W + s] = df_pack(d2df_bits(vx));
    rf[2 * NP * W + s] = df_pack(d2df_bits(vy));
    rf[3 * NP * W + s] = df_pack(d2df_bits(vz));
    rf[4 * NP * W + s] = df_pack(d2df_bits(__ldg(a.pm + PM_H * N + p)));
    ri[5 * NP * W + s] = pr;
    rf[6 * NP * W + s] = df_pack(d2df_bits(U[0]));
    rf[7 * NP * W + s] = df_pack(d2df_bits(U[4]));
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double l = a.lam_scale * __ldg(a.lam + v * N + p);
      lm[v * NP * W + s] = l;
      const int e = ((__double2hiint(l) >> 20) & 0x7ff) - 1023;
      if (l != 0.0 && e > emax) emax = e;
    }
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  if ((tid & 31) == 0) atomicMax(&s_emax, emax);
  __syncthreads();
  // E = exponent of the largest |lambda| (0 if lambda vanishes on the tile); lambda / 2^E
  const int E = (s_emax == -2000) ? 0 : max(-1000, min(1000, s_emax));
  const double down = pow2d(-E);
  int range_bad = 0;
  for (int item = tid; item < NP * W; item += APF::THREADS) {
    int pos, line;
    tile_split<D, W>(item, NP, pos, line);
    const int s = tile_idx<D, W>(pos, line, NP);
#pragma unroll
    for (int v = 0; v < 5; ++v) lm[v * NP * W + s] *= down;
  }
  // first differences of the 9 scalars, FP64, kept as double-float; both lines of the tile
  // per item, stored side by side (hi0, hi1, lo0, lo1) for the two-lane phases below
  for (int item = tid; item < 9 * (NP - 1); item += APF::THREADS) {
    const int m = item / (NP - 1);
    const int j = item - m * (NP - 1);
    const double* qm = q + m * NP * W;
    const double d0 = qm[tile_idx<D, W>(j + 1, 0, NP)] - qm[tile_idx<D, W>(j, 0, NP)];
    const double d1 = qm[tile_idx<D, W>(j + 1, 1, NP)] - qm[tile_idx<D, W>(j, 1, NP)];
    G4[m * NP + j] = df2_to4(df2_pack(d2df_bits(d0), d2df_bits(d1)));
  }
  __syncthreads();

  // ---- B: window terms b_k of every window, stored as 1/b_k (both lines at once) -----------------
  {
    const df2 c133_2 = df2_splat(c133), eps4_2 = df2_splat(eps4);
    const df2 one{f2splat(1.0f), f2splat(0.0f)};
    for (int item = tid; item < 9 * NW; item += APF::THREADS) {
      const int m = item / NW;
      const int w = item - m * NW;
      const float4* Gm = G4 + m * NP;
      const df2 g0 = df2_from4(Gm[w]), g1 = df2_from4(Gm[w + 1]);
      const df2 sw = df2_sub(g1, g0);
      const df2 aa = df2_add_pos_u(df2_mul_u(df2_sqr_u(sw), c133_2), eps4_2);
      const df2 b0 = df2_add_pos_u(df2_sqr_u(df2_sub(df2_mul_f_u(g1, 3.0f), g0)), aa);
      const df2 b1 = df2_add_pos_u(df2_sqr_u(df2_add_fast(g0, g1)), aa);
      const df2 b2 = df2_add_pos_u(df2_sqr_u(df2_sub(g1, df2_mul_f_u(g0, 3.0f))), aa);
      // their reciprocals: the weights (c_k / b_k^2) and the adjoints of b_k (omega_k / b_k) need only those
      Bw4[(m * 3 + 0) * NW + w] = df2_to4(df2_div(one, b0));
      Bw4[(m * 3 + 1) * NW + w] = df2_to4(df2_div(one, b1));
      Bw4[(m * 3 + 2) * NW + w] = df2_to4(df2_div(one, b2));
      // b^2 must stay inside the float range (differences of the data up to ~1e9)
      range_bad |= !(fmaxf(b0.hi.x, fmaxf(b1.hi.x, b2.hi.x)) < 1e18f) || !(fmaxf(b0.hi.y, fmaxf(b1.hi.y, b2.hi.y)) < 1e18f);
    }
  }
  __syncthreads();

  // ---- C: jumps of the u reconstructions (for the Roe adjoint), both lines at once -----------
  for (int item = tid; item < 5 * NI; item += APF::THREADS) {
    const int m = item / NI;
    const int f = item - m * NI;
    const float4* Gm = G4 + m * NP;
    df2 g[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) g[j] = df2_from4(Gm[f + j]);
    const float4* B = Bw4 + m * 3 * NW;
    auto ldb = [&](int k, int w) { return df2_from4(B[k * NW + w]); };
    df2 omL[3], omR[3], s[3], E0, E2;
    df2_omega(ldb(0, f), ldb(1, f + 1), ldb(2, f + 2), omL);
    const df2 ML = df2_adj_offset(g[0], g[1], g[2], g[3], omL, kc2, E0, E2, s);
    df2_omega(ldb(2, f + 3), ldb(1, f + 2), ldb(0, f + 1), omR);
    const df2 MR = df2_adj_offset(df2_neg(g[4]), df2_neg(g[3]), df2_neg(g[2]), df2_neg(g[1]), omR, kc2, E0, E2, s);
    // the jump ûR - ûL = (P3 - P2) - (2 g2 + g3)/6 + MR - (2 g2 + g1)/6 - ML, in double-float
    // (the values themselves are not needed)
    const df2 g22 = df2_twice(g[2]);
    const df2 lin = df2_mul_u(df2_add_fast(df2_add_fast(g22, g[1]), df2_add_fast(g22, g[3])), kc2.sixth);
    const df2 du = df2_add_fast(df2_add_fast(g[2], df2_neg(lin)), df2_add_fast(MR, df2_neg(ML)));
    float2* rj = reinterpret_cast<float2*>(rec) + m * NI * W;
    rj[tile_idx<D, W>(f, 0, NI)] = df_pack(df2_lane0(du));
    rj[tile_idx<D, W>(f, 1, NI)] = df_pack(df2_lane1(du));
    // the weights, for phase E (which overwrites these slots with its contributions)
    float4* wm = wc4 + m * 6 * NI;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wm[k * NI + f] = df2_to4(omL[k]);
      wm[(3 + k) * NI + f] = df2_to4(omR[k]);
    }
  }
  __syncthreads();

  // ---- D: adjoint of the Roe flux, in double-float -----------------------------------------
  {
    int bad = 0;
    const df gam = d2df_bits(a.gamma), gm1 = d2df_bits(a.gamma - 1.0), hd = d2df_bits(a.hdelta);
    const float2* rf = reinterpret_cast<const float2*>(ri);
    float2* rdf = reinterpret_cast<float2*>(rd);
    for (int item = tid; item < NI * W; item += APF::THREADS) {
      int f, line;
      tile_split<D, W>(item, NI, f, line);
      const int o = tile_idx<D, W>(f, line, NI);
      const int sa = tile_idx<D, W>(f + 2, line, NP), sb = tile_idx<D, W>(f + 3, line, NP);
      df du[5], Lh[5], Va[3], Vb[3];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        du[v] = df_unpack(reinterpret_cast<const float2*>(rec)[v * NI * W + o]);
        Lh[v] = d2df_bits((lm[v * NP * W + sb] - lm[v * NP * W + sa]) * rdx);
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Va[m] = df_unpack(rf[(1 + m) * NP * W + sa]);
        Vb[m] = df_unpack(rf[(1 + m) * NP * W + sb]);
      }
      df dub[5], ga[5], gb[5];
      bad |= roe_adjoint_df<D>(du, Lh, df_unpack(rf[sa]), df_unpack(rf[sb]), Va, Vb, df_unpack(rf[4 * NP * W + sa]),
                               df_unpack(rf[4 * NP * W + sb]), df_unpack(rf[6 * NP * W + sa]),
                               df_unpack(rf[7 * NP * W + sa]), df_unpack(rf[6 * NP * W + sb]),
                               df_unpack(rf[7 * NP * W + sb]), gam, gm1, hd, dub, ga, gb);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        rdf[v * NI * W + o] = df_pack(dub[v]);
        rdf[(5 + v) * NI * W + o] = df_pack(ga[v]);
        rdf[(10 + v) * NI * W + o] = df_pack(gb[v]);
      }
    }
    if (__any_sync(0xffffffffu, bad & 1) && (tid & 31) == 0) atomicOr(a.status, ST_NONPHYS);
    range_bad |= bad & 2;
  }
  __syncthreads();

  // ---- E: reconstruction adjoints -> six stencil contributions per scalar and interface, -----
  //      both lines at once
  for (int item = tid; item < 9 * NI; item += APF::THREADS) {
    const int m = item / NI;
    const int f = item - m * NI;
    df y2[2][2];  // [line][left, right]
#pragma unroll
    for (int line = 0; line < 2; ++line) {
      const int o = tile_idx<D, W>(f, line, NI);
      const int sa = tile_idx<D, W>(f + 2, line, NP), sb = tile_idx<D, W>(f + 3, line, NP);
      df yL, yR;
      if (m < 5) {
        const df gdu = df_unpack(reinterpret_cast<const float2*>(rd)[m * NI * W + o]);
        yL = df_neg(gdu);
        yR = gdu;
        if (m == 1 + D) {  // mass flux f_0 = u_{1+D}: (f^L + f^R)/2 part
          const df h0 = d2df_bits(0.5 * ((lm[sb] - lm[sa]) * rdx));
          yL = df_add_fast(yL, h0);
          yR = df_add_fast(yR, h0);
        }
      } else {
        yL = yR = d2df_bits(0.5 * ((lm[(m - 4) * NP * W + sb] - lm[(m - 4) * NP * W + sa]) * rdx));
      }
      range_bad |= !(fabsf(yL.hi) < 1e30f && fabsf(yR.hi) < 1e30f);
      y2[line][0] = yL;
      y2[line][1] = yR;
    }
    const float4* Gm = G4 + m * NP;
    df2 g[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) g[j] = df2_from4(Gm[f + j]);
    const float4* B = Bw4 + m * 3 * NW;
    auto ldb = [&](int k, int w) { return df2_from4(B[k * NW + w]); };
    float4* wm = wc4 + m * 6 * NI;
    df2 omL[3], omR[3];
    if (m < 5) {  // stored by phase C
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        omL[k] = df2_from4(wm[k * NI + f]);
        omR[k] = df2_from4(wm[(3 + k) * NI + f]);
      }
    } else {
      df2_omega(ldb(0, f), ldb(1, f + 1), ldb(2, f + 2), omL);
      df2_omega(ldb(2, f + 3), ldb(1, f + 2), ldb(0, f + 1), omR);
    }
    df2 cL[5], cR[5];
    df2_recon_adjoint(g[0], g[1], g[2], g[3], ldb(0, f), ldb(1, f + 1), ldb(2, f + 2), omL,
                             df2_pack(y2[0][0], y2[1][0]), kc2, cL);
    df2_recon_adjoint(df2_neg(g[4]), df2_neg(g[3]), df2_neg(g[2]), df2_neg(g[1]), ldb(2, f + 3),
                             ldb(1, f + 2), ldb(0, f + 1), omR, df2_pack(y2[0][1], y2[1][1]), kc2, cR);
    wm[0 * NI + f] = df2_to4(cL[0]);
#pragma unroll
    for (int j = 1; j < 5; ++j) wm[j * NI + f] = df2_to4(df2_add_fast(cL[j], cR[5 - j]));
    wm[5 * NI + f] = df2_to4(cR[0]);
  }
  if (__any_sync(0xffffffffu, range_bad) && (tid & 31) == 0) atomicOr(a.status, ST_DF_RANGE);
  __syncthreads();

  // ---- F: gather, adjoint of the point fluxes, scale back, epilogue ----------------------------
  const double up = pow2d(E);
  const double gm1 = a.gamma - 1.0;
  // F1: the gather, one (scalar, point, line) per item, into the dead window-term space
  static_assert(9 * TP * W <= 27 * NW * W, "gathered sums fit the window-term space");
  double* gsm = sm + APF::OFF_B;  // [9][TP*W]
  {
    const float* wcf = reinterpret_cast<const float*>(wc4);  // lane `line` of a pair: hi at +line, lo at +2+line
    const float2* rdf = reinterpret_cast<const float2*>(rd);
    for (int item = tid; item < 9 * TP * W; item += APF::THREADS) {
      const int m = item / (TP * W);
      int pp, line;
      tile_split<D, W>(item - m * TP * W, TP, pp, line);
      const int pos = pp + 5;
      auto ldw = [&](int slot) { return df{wcf[4 * slot + line], wcf[4 * slot + 2 + line]}; };
      df acc = ldw(m * 6 * NI + pos);
#pragma unroll
      for (int j = 1; j < 6; ++j) acc = df_add_fast(acc, ldw((m * 6 + j) * NI + pos - j));
      if (m < 5) {  // the Roe-average adjoints of the two interfaces next to the point
        const int oa = tile_idx<D, W>(pos - 2, line, NI), ob = tile_idx<D, W>(pos - 3, line, NI);
        acc = df_add_fast(acc, df_add_fast(df_unpack(rdf[(5 + m) * NI * W + oa]), df_unpack(rdf[(10 + m) * NI * W + ob])));
      }
      gsm[m * TP * W + tile_idx<D, W>(pp, line, TP)] = f2d_bits(acc.hi) + f2d_bits(acc.lo);
    }
  }
  __syncthreads();
  // F2: adjoint of the point fluxes, scale back, epilogue (one point per item)
  for (int item = tid; item < TP * W; item += APF::THREADS) {
    int pp, line;
    tile_split<D, W>(item, TP, pp, line);
    if (s0 + pp >= nD || a0 + line >= na) continue;
    const int pos = pp + 5;
    double gsum[9], cv[5];
#pragma unroll
    for (int m = 0; m < 9; ++m) gsum[m] = gsm[m * TP * W + tile_idx<D, W>(pp, line, TP)];
#pragma unroll
    for (int v = 0; v < 5; ++v) cv[v] = gsum[v];
    const int s = tile_idx<D, W>(pos, line, NP);
    const double rho = q[s], e = q[4 * NP * W + s], pr = ri[5 * NP * W + s];
    const float2* rfs = reinterpret_cast<const float2*>(ri) + s;
    double V[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 vk = rfs[(1 + k) * NP * W];
      V[k] = f2d_bits(vk.x) + f2d_bits(vk.y);
    }
    const double un = V[D];
    const double Fbm[3] = {gsum[5], gsum[6], gsum[7]};
    const double Fb4 = gsum[8];
    const double pb = fma(Fb4, un, Fbm[D]);
    double unb = Fb4 * (e + pr);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unb = fma(Fbm[k], q[(1 + k) * NP * W + s], unb);
      cv[1 + k] = fma(Fbm[k], un, cv[1 + k]);
    }
    cv[4] = fma(Fb4, un, cv[4]);
    const double rr = rcp_newton(rho);
    cv[1 + D] = fma(unb, rr, cv[1 + D]);
    cv[0] = fma(-unb * un, rr, cv[0]);
    const double gp = gm1 * pb;
    cv[4] += gp;
    double v2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cv[1 + k] = fma(-gp, V[k], cv[1 + k]);
      v2 = fma(V[k], V[k], v2);
    }
    cv[0] = fma(0.5 * gp, v2, cv[0]);
#pragma unroll
    for (int v = 0; v < 5; ++v) cv[v] *= up;
    const long long p = tile_flat<D>(a.g, s0 + pp, a0 + line, bz);
    adj_epilogue(a, p, cv);
  }
}

// Neighbour flat indices at offsets -2, -1, +1, +2 along direction d.
__device__ __forceinline__ void neighbours(int i, int j, int k, int d, const Grid& g, long long nb[4]) {
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int off = (o < 2) ? (o - 2) : (o - 1);
    int c[3] = {i, j, k};
    c[d] = wrap_near(c[d], off, g.n[d]);
    nb[o] = flat3(c[0], c[1], c[2], g.n[0], g.n[1]);
  }
}

// Gradients G[q][e] of (u, v, w, T) at point p (the same stencil as the viscous fluxes).
__device__ __forceinline__ void point_gradients(const Grid& g, const double* pm, int i, int j, int k, double G[4][3]) {
  const long long N = g.N;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long nb[4];
    neighbours(i, j, k, d, g, nb);
    const double r12 = g.r12h[d];
#pragma unroll
    for (int qv = 0; qv < 4; ++qv) {
      const int plane = (qv < 3) ? qv : PM_T;
      const double* A = pm + (long long)plane * N;
      G[qv][d] = d4(__ldg(A + nb[0]), __ldg(A + nb[1]), __ldg(A + nb[2]), __ldg(A + nb[3]), r12);
    }
  }
}

__global__ void __launch_bounds__(256) k_visc_adj1(const Grid g, const double* __restrict__ pm,
                                                   const double* __restrict__ lam, double lam_scale,
                                                   double* __restrict__ sc, double mu, double kappa) {
  const long long N = g.N;
  // one thread per point of a 32 x 8 block of an x-y plane; blockIdx.z = the plane
  const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
  if (i < g.n[0] && j < g.n[1]) {
    const long long p = flat3(i, j, k, g.n[0], g.n[1]);
    double G[4][3];
    point_gradients(g, pm, i, j, k, G);
    const double vel[3] = {pm[PM_U * N + p], pm[PM_V * N + p], pm[PM_W * N + p]};
    const double tdiv = (2.0 / 3.0) * (G[0][0] + G[1][1] + G[2][2]);
    double Gb[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double vb[3] = {0, 0, 0};
    double divb = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      long long nb[4];
      neighbours(i, j, k, d, g, nb);
      const double r12 = g.r12h[d];
      double Fb[4];  // adjoint of the viscous flux along d: -D_d lambda_{1+c}
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const double* L = lam + (long long)(1 + cc) * N;
        Fb[cc] = -lam_scale * d4(__ldg(L + nb[0]), __ldg(L + nb[1]), __ldg(L + nb[2]), __ldg(L + nb[3]), r12);
      }
      Gb[3][d] = fma(kappa, Fb[3], Gb[3][d]);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double tau = (m == d) ? mu * fma(2.0, G[d][d], -tdiv) : mu * (G[m][d] + G[d][m]);
        const double tb = fma(Fb[3], vel[m], Fb[m]);
        vb[m] = fma(Fb[3], tau, vb[m]);
        if (m == d) {
          Gb[d][d] = fma(2.0 * mu, tb, Gb[d][d]);
          divb = fma(-(2.0 / 3.0) * mu, tb, divb);
        } else {
          Gb[m][d] = fma(mu, tb, Gb[m][d]);
          Gb[d][m] = fma(mu, tb, Gb[d][m]);
        }
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Gb[d][d] += divb;
#pragma unroll
    for (int qv = 0; qv < 4; ++qv)
#pragma unroll
      for (int e = 0; e < 3; ++e) sc[(long long)(qv * 3 + e) * N + p] = Gb[qv][e];
#pragma unroll
    for (int m = 0; m < 3; ++m) sc[(long long)(12 + m) * N + p] = vb[m];
  }
}

__global__ void __launch_bounds__(256) k_visc_adj2(const Grid g, const double* __restrict__ u,
                                                   const double* __restrict__ sc, double gamma,
                                                   double* __restrict__ out, int accumulate, int with_rho) {
  const long long N = g.N;
  // one thread per point of a 32 x 8 block of an x-y plane; blockIdx.z = the plane
  const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
  if (i < g.n[0] && j < g.n[1]) {
    const long long p = flat3(i, j, k, g.n[0], g.n[1]);
    double Wb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      long long nb[4];
      neighbours(i, j, k, e, g, nb);
      const double r12 = g.r12h[e];
#pragma unroll
      for (int qv = 0; qv < 4; ++qv) {
        const double* A = sc + (long long)(qv * 3 + e) * N;
        Wb[qv] -= d4(__ldg(A + nb[0]), __ldg(A + nb[1]), __ldg(A + nb[2]), __ldg(A + nb[3]), r12);
      }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) Wb[m] += sc[(long long)(12 + m) * N + p];
    const double rho = u[p], e = u[4 * N + p];
    const double rr = 1.0 / rho;
    const double V[3] = {u[N + p] * rr, u[2 * N + p] * rr, u[3 * N + p] * rr};
    const double gg = gamma * (gamma - 1.0);
    const double Tb = gg * Wb[3];
    double ub[5];
    ub[4] = Tb * rr;
    double v2 = 0.0, wv = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      ub[1 + m] = fma(-Tb, V[m], Wb[m]) * rr;
      v2 = fma(V[m], V[m], v2);
      wv = fma(Wb[m], V[m], wv);
    }
    ub[0] = fma(Tb, v2 - e * rr, -wv) * rr;
    if (with_rho) ub[0] += sc[15 * N + p];
    if (accumulate) {
#pragma unroll
      for (int v = 0; v < 5; ++v) out[v * N + p] += ub[v];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) out[v * N + p] = ub[v];
    }
  }
}

// The two viscous adjoint kernels in the NS3D_FP64 form: the stencils, stresses, heat flux and
// their adjoints in double-float on the FP32 pipe (the same algebra as k_visc_adj1/2), the 15
// scratch planes stored as double-float pairs; kernel 2 converts the adjoint of (u, v, w, T)
// to FP64 once and finishes as k_visc_adj2.  The viscous terms are ~mu |grad u| in size, so
// the double-float rounding (2^-48) lands far below the FP64 rounding of the direction
// adjoints they are added to, as in the forward viscous kernel.
// Largest binary exponent of lam_scale * lambda over the planes 1..4 of lambda, into *out (which
// holds a large negative value before; it stays so if they all vanish).
__global__ void __launch_bounds__(256) k_lam_expo(const double* __restrict__ lam, long long N, double lam_scale,
                                                  int* out) {
  int emax = INT_MIN;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < 4 * N; i += (long long)gridDim.x * 256) {
    const double l = lam_scale * __ldg(lam + N + i);
    if (l != 0.0) emax = max(emax, ((__double2hiint(l) >> 20) & 0x7ff) - 1023);
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  if ((threadIdx.x & 31) == 0 && emax != INT_MIN) atomicMax(out, emax);
}

// The common exponent E of the two kernels (0 if lambda vanishes), inside the FP64 range.
__device__ __forceinline__ int visc_adj_expo(const int* expo) {
  const int e = *expo;
  return (e < -1000) ? 0 : min(e, 1000);
}

__global__ void __launch_bounds__(256) k_visc_adj1_df(const Grid g, const double* __restrict__ pm,
                                                      const double* __restrict__ lam, double lam_scale,
                                                      double* __restrict__ sc, double mu, double kappa,
                                                      const int* __restrict__ expo) {
  const long long N = g.N;
  // lambda * lam_scale relative to 2^E (exact power-of-two scaling): every double-float value of
  // this kernel stays inside the float range whatever the scale of lambda
  const double ls = lam_scale * pow2d(-visc_adj_expo(expo));
  const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  const long long p = flat3(i, j, k, g.n[0], g.n[1]);
  df G[4][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long nb[4];
    neighbours(i, j, k, d, g, nb);
    const df r12 = d2df_bits(g.r12h[d]);
#pragma unroll
    for (int qv = 0; qv < 4; ++qv) {
      const double* A = pm + (long long)((qv < 3) ? qv : PM_T) * N;
      G[qv][d] = d4_df(__ldg(A + nb[0]), __ldg(A + nb[1]), __ldg(A + nb[2]), __ldg(A + nb[3]), r12);
    }
  }
  const df vel[3] = {d2df_bits(pm[PM_U * N + p]), d2df_bits(pm[PM_V * N + p]), d2df_bits(pm[PM_W * N + p])};
  const double two3 = 2.0 / 3.0;
  const df c23{(float)two3, (float)(two3 - (double)(float)two3)};
  const df dmu = d2df_bits(mu), dkap = d2df_bits(kappa);
  const df mu2 = df_twice(dmu), mmu23 = df_neg(df_mul(dmu, c23));  // 2 mu and -(2/3) mu
  const df tdiv = df_mul_u(df_add_fast(G[0][0], df_add_fast(G[1][1], G[2][2])), c23);
  const df zero{0.0f, 0.0f};
  df Gb[4][3], vb[3] = {zero, zero, zero}, divb = zero;
#pragma unroll
  for (int qv = 0; qv < 4; ++qv)
#pragma unroll
    for (int e = 0; e < 3; ++e) Gb[qv][e] = zero;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    long long nb[4];
    neighbours(i, j, k, d, g, nb);
    const df r12 = d2df_bits(g.r12h[d]);
    df Fb[4];  // adjoint of the viscous flux along d: -D_d lambda_{1+c}
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const double* L = lam + (long long)(1 + cc) * N;
      Fb[cc] = df_neg(d4_df(ls * __ldg(L + nb[0]), ls * __ldg(L + nb[1]), ls * __ldg(L + nb[2]), ls * __ldg(L + nb[3]),
                            r12));
    }
    Gb[3][d] = df_add_fast(df_mul_u(dkap, Fb[3]), Gb[3][d]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const df tau = (m == d) ? df_mul(dmu, df_add_fast(df_twice(G[d][d]), df_neg(tdiv)))
                              : df_mul(dmu, df_add_fast(G[m][d], G[d][m]));
      const df tb = df_add_fast(df_mul_u(Fb[3], vel[m]), Fb[m]);
      vb[m] = df_add_fast(df_mul_u(Fb[3], tau), vb[m]);
      if (m == d) {
        Gb[d][d] = df_add_fast(df_mul_u(mu2, tb), Gb[d][d]);
        divb = df_add_fast(df_mul_u(mmu23, tb), divb);
      } else {
        const df t = df_mul_u(dmu, tb);
        Gb[m][d] = df_add_fast(t, Gb[m][d]);
        Gb[d][m] = df_add_fast(t, Gb[d][m]);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) Gb[d][d] = df_add_fast(Gb[d][d], divb);
#pragma unroll
  for (int qv = 0; qv < 4; ++qv)
#pragma unroll
    for (int e = 0; e < 3; ++e) store_df(sc + (long long)(qv * 3 + e) * N + p, Gb[qv][e]);
#pragma unroll
  for (int m = 0; m < 3; ++m) store_df(sc + (long long)(12 + m) * N + p, vb[m]);
}

__global__ void __launch_bounds__(256) k_visc_adj2_df(const Grid g, const double* __restrict__ u,
                                                      const double* __restrict__ sc, double gamma,
                                                      double* __restrict__ out, int accumulate,
                                                      const int* __restrict__ expo) {
  const long long N = g.N;
  const double up = pow2d(visc_adj_expo(expo));  // back from the scale of k_visc_adj1_df
  const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
  if (i >= g.n[0] || j >= g.n[1]) return;
  const long long p = flat3(i, j, k, g.n[0], g.n[1]);
  const float2* S = reinterpret_cast<const float2*>(sc);
  auto ld = [&](long long idx) { const float2 v = __ldg(S + idx); return df{v.x, v.y}; };
  const df zero{0.0f, 0.0f};
  df W[4] = {zero, zero, zero, zero};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    long long nb[4];
    neighbours(i, j, k, e, g, nb);
    const df r12 = d2df_bits(g.r12h[e]);
#pragma unroll
    for (int qv = 0; qv < 4; ++qv) {
      const long long b = (long long)(qv * 3 + e) * N;
      W[qv] = df_add_fast(W[qv], df_neg(d4_dfv(ld(b + nb[0]), ld(b + nb[1]), ld(b + nb[2]), ld(b + nb[3]), r12)));
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) W[m] = df_add_fast(W[m], ld((long long)(12 + m) * N + p));
  double Wb[4];
#pragma unroll
  for (int qv = 0; qv < 4; ++qv) Wb[qv] = (f2d_bits(W[qv].hi) + f2d_bits(W[qv].lo)) * up;
  const double rho = u[p], e = u[4 * N + p];
  const double rr = 1.0 / rho;
  const double V[3] = {u[N + p] * rr, u[2 * N + p] * rr, u[3 * N + p] * rr};
  const double gg = gamma * (gamma - 1.0);
  const double Tb = gg * Wb[3];
  double ub[5];
  ub[4] = Tb * rr;
  double v2 = 0.0, wv = 0.0;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    ub[1 + m] = fma(-Tb, V[m], Wb[m]) * rr;
    v2 = fma(V[m], V[m], v2);
    wv = fma(Wb[m], V[m], wv);
  }
  ub[0] = fma(Tb, v2 - e * rr, -wv) * rr;
  if (accumulate) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * N + p] += ub[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * N + p] = ub[v];
  }
}

// d(mean of rho |v|^2/2)/du: (-|V|^2/2, V) / N, 0 for the energy.
__global__ void __launch_bounds__(256) k_ke_seed(const Grid g, const double* __restrict__ u,
                                                 double* __restrict__ out) {
  const long long N = g.N;
  const double rn = 1.0 / (double)N;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const double rr = 1.0 / u[p];
    double v2 = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double V = u[(1 + m) * N + p] * rr;
      out[(1 + m) * N + p] = V * rn;
      v2 = fma(V, V, v2);
    }
    out[p] = -0.5 * v2 * rn;
    out[4 * N + p] = 0.0;
  }
}

// Enstrophy mean of rho |omega|^2/2: adjoint of the velocity gradients (rho omega / N on
// the antisymmetric pairs), zero velocity adjoint, direct density term |omega|^2/(2N).
__global__ void __launch_bounds__(256) k_ens_seed(const Grid g, const double* __restrict__ u,
                                                  const double* __restrict__ pm, double* __restrict__ sc) {
  const long long N = g.N;
  const double rn = 1.0 / (double)N;
  // one thread per point of a 32 x 8 block of an x-y plane; blockIdx.z = the plane
  const int i = blockIdx.x * 32 + threadIdx.x % 32, j = blockIdx.y * 8 + threadIdx.x / 32, k = blockIdx.z;
  if (i < g.n[0] && j < g.n[1]) {
    const long long p = flat3(i, j, k, g.n[0], g.n[1]);
    double G[4][3];
    point_gradients(g, pm, i, j, k, G);
    const double wx = G[2][1] - G[1][2], wy = G[0][2] - G[2][0], wz = G[1][0] - G[0][1];
    const double rw = u[p] * rn;
    double Gb[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    Gb[2][1] = rw * wx;
    Gb[1][2] = -rw * wx;
    Gb[0][2] = rw * wy;
    Gb[2][0] = -rw * wy;
    Gb[1][0] = rw * wz;
    Gb[0][1] = -rw * wz;
#pragma unroll
    for (int qv = 0; qv < 4; ++qv)
#pragma unroll
      for (int e = 0; e < 3; ++e) sc[(long long)(qv * 3 + e) * N + p] = Gb[qv][e];
#pragma unroll
    for (int m = 0; m < 3; ++m) sc[(long long)(12 + m) * N + p] = 0.0;
    sc[15 * N + p] = 0.5 * rn * fma(wx, wx, fma(wy, wy, wz * wz));
  }
}

int point_blocks(const Grid& g) {
  const long long b = (g.N + 255) / 256;
  return (int)(b < 152LL * 16 ? b : 152LL * 16);
}

// Launch geometry of the stencil point kernels: 32 x 8 x 1 blocks of 256 threads over (x, y, z).
dim3 plane_blocks(const Grid& g) { return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.n[2]); }

}  // namespace

cudaError_t prepare_adj_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_adj_dir<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, APL::BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adj_dir<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, APL::BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adj_dir<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, APL::BYTES);
  auto df_attr = [](auto* kernel) {
    cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, APF::BYTES);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return r;
  };
  if (e == cudaSuccess) e = df_attr(k_adj_dir_df<0>);
  if (e == cudaSuccess) e = df_attr(k_adj_dir_df<1>);
  if (e == cudaSuccess) e = df_attr(k_adj_dir_df<2>);
  return e;
}

cudaError_t launch_adj_dir(int d, const AdjArgs& a, cudaStream_t s) {
  const int AXd = (d == 0) ? 1 : 0;
  const int BXd = (d == 2) ? 1 : 2;
  if (a.mode == 1) {
    dim3 grid((a.g.n[d] + APF::TP - 1) / APF::TP, (a.g.n[AXd] + APF::W - 1) / APF::W, a.g.n[BXd]);
    switch (d) {
      case 0: k_adj_dir_df<0><<<grid, APF::THREADS, APF::BYTES, s>>>(a); break;
      case 1: k_adj_dir_df<1><<<grid, APF::THREADS, APF::BYTES, s>>>(a); break;
      default: k_adj_dir_df<2><<<grid, APF::THREADS, APF::BYTES, s>>>(a); break;
    }
    return cudaGetLastError();
  }
  dim3 grid((a.g.n[d] + APL::TP - 1) / APL::TP, (a.g.n[AXd] + APL::W - 1) / APL::W, a.g.n[BXd]);
  switch (d) {
    case 0: k_adj_dir<0><<<grid, APL::THREADS, APL::BYTES, s>>>(a); break;
    case 1: k_adj_dir<1><<<grid, APL::THREADS, APL::BYTES, s>>>(a); break;
    default: k_adj_dir<2><<<grid, APL::THREADS, APL::BYTES, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_visc_adj1(const Grid& g, const double* pm, const double* lam, double lam_scale, double* scratch,
                             double mu, double kappa, cudaStream_t s, int* expo) {
  if (expo) {
    cudaError_t e = cudaMemsetAsync(expo, 0x80, sizeof(int), s);  // 0x80808080: below every exponent
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((4 * g.N + 255) / 256, 4096);
    k_lam_expo<<<(int)blocks, 256, 0, s>>>(lam, g.N, lam_scale, expo);
    k_visc_adj1_df<<<plane_blocks(g), 256, 0, s>>>(g, pm, lam, lam_scale, scratch, mu, kappa, expo);
  } else
    k_visc_adj1<<<plane_blocks(g), 256, 0, s>>>(g, pm, lam, lam_scale, scratch, mu, kappa);
  return cudaGetLastError();
}

cudaError_t launch_visc_adj2(const Grid& g, const double* u, const double* scratch, double gamma, double* out,
                             int accumulate, int with_rho, cudaStream_t s, const int* expo) {
  if (expo && !with_rho)  // the double-float scratch of k_visc_adj1_df
    k_visc_adj2_df<<<plane_blocks(g), 256, 0, s>>>(g, u, scratch, gamma, out, accumulate, expo);
  else
    k_visc_adj2<<<plane_blocks(g), 256, 0, s>>>(g, u, scratch, gamma, out, accumulate, with_rho);
  return cudaGetLastError();
}

cudaError_t launch_ke_seed(const Grid& g, const double* u, double* grad, cudaStream_t s) {
  k_ke_seed<<<point_blocks(g), 256, 0, s>>>(g, u, grad);
  return cudaGetLastError();
}

cudaError_t launch_ens_seed(const Grid& g, const double* u, const double* pm, double* scratch, cudaStream_t s) {
  k_ens_seed<<<plane_blocks(g), 256, 0, s>>>(g, u, pm, scratch);
  return cudaGetLastError();
}

}  // namespace ns3d
