/*
 * FP64 CPU oracle of the thermal pseudopotential MRT lattice Boltzmann step
 * (Huang, Wang, He & Huang, arXiv 2206.00946).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py, never by the product path.  Plain per-cell loops in
 * FP64, the collision done literally as m = M f, m* = m - Lambda (m - m^eq) + ...,
 * f* = M^-1 m* with the matrices of the appendix (Eqs. 39-40) and inverses
 * computed here by Gauss-Jordan elimination.  No -ffast-math.
 *
 * One step t -> t+1 (the paper gives the equations, not a driver loop; the order
 * below is this project's reading and is the same one the CUDA path follows):
 *   1. rho = sum f, rho u^eq = sum c f (Eq. 3); T = sum g (m_0^eq = T, Eq. 25)
 *   2. p_EOS, (dp/dT)_rho (Eq. 37) and psi (Eq. 7)
 *   3. ghost psi beyond the faces (periodic wrap / wetting Eq. 36 / open copy)
 *   4. F = -G psi(x) sum w(|c|^2) psi(x+c) c (Eq. 6); du = F/rho (Eq. 4);
 *      u = u^eq + F/(2 rho) (Eq. 5); u^eq := 0 and u := 0 at wall nodes (Sec. 3.1)
 *   5. D3Q19 MRT collision in moment space with the exact-difference forcing (Eq. 8)
 *   6. streaming (Eq. 8b) with the modified bounce-back at wall faces (Eq. 34)
 *   7. Zou-He type constant-pressure boundary at open faces (Sec. 3.3)
 *   8. D3Q7 MRT collision with the source -w_i Fbar (Eqs. 13, 15); grad T from the
 *      local first moment (Eqs. 27-29), div u by the isotropic D3Q19 difference
 *   9. relaxed streaming rho c_v g_i(x+c_i,t+1) = g*_i(x,t) + (rho c_v - 1) g_i(x+c_i,t)
 *      (Eq. 13) with rho c_v taken at the destination node
 *  10. non-equilibrium extrapolation of g at every Dirichlet node (Eqs. 35-36)
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- tables -- */

/* Appendix, D3Q19 transformation matrix M-hat (rows = moments, columns = i). */
/* Built with -fopenmp (oracle/build.py, omp=True) the per-cell loops over z run on all
 * host cores; each iteration writes only its own cells (or, in the streaming loops, a
 * destination no other source writes), so the result is bit-identical to the serial
 * build.  Without OpenMP the pragma is empty. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_PAR_Z _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PAR_Z
#endif

static const int MHAT[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1}};

/* Appendix, D3Q7 transformation matrix M. */
static const int M7I[7][7] = {{1, 1, 1, 1, 1, 1, 1},   {0, 1, -1, 0, 0, 0, 0}, {0, 0, 0, 1, -1, 0, 0},
                              {0, 0, 0, 0, 0, 1, -1},  {0, 1, 1, 1, 1, 1, 1},  {0, 1, 1, -1, -1, 0, 0},
                              {0, 1, 1, 0, 0, -1, -1}};

static int T_ready = 0;
static int C19[19][3], OPP19[19];
static int C7[7][3];
static double W19[19], VARPI[19];
static double Mh[19][19], Mhi[19][19];
static double M7[7][7], M7i[7][7];

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix. */
static void gj_inverse(int n, const double* A, double* Ainv) {
  double a[19][38];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) a[r][c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    double d = a[col][col];
    for (int c = 0; c < 2 * n; ++c) a[col][c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double m = a[r][col];
      if (m != 0.0)
        for (int c = 0; c < 2 * n; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r][n + c];
}

static void init_tables(void) {
  if (T_ready) return;
  /* velocities read off rows 1-3 (c_x, c_y, c_z) of the transformation matrices */
  for (int i = 0; i < 19; ++i)
    for (int d = 0; d < 3; ++d) C19[i][d] = MHAT[1 + d][i];
  for (int i = 0; i < 7; ++i)
    for (int d = 0; d < 3; ++d) C7[i][d] = M7I[1 + d][i];
  for (int i = 0; i < 19; ++i) {
    int c2 = C19[i][0] * C19[i][0] + C19[i][1] * C19[i][1] + C19[i][2] * C19[i][2];
    W19[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0); /* Eq. 2 weights */
    VARPI[i] = (c2 == 0) ? 0.0 : (c2 == 1 ? 1.0 / 6.0 : 1.0 / 12.0);      /* Eq. 6 weights */
    for (int j = 0; j < 19; ++j)
      if (C19[j][0] == -C19[i][0] && C19[j][1] == -C19[i][1] && C19[j][2] == -C19[i][2]) OPP19[i] = j;
  }
  double A[19 * 19], Ai[19 * 19];
  for (int r = 0; r < 19; ++r)
    for (int c = 0; c < 19; ++c) A[r * 19 + c] = Mh[r][c] = MHAT[r][c];
  gj_inverse(19, A, Ai);
  for (int r = 0; r < 19; ++r)
    for (int c = 0; c < 19; ++c) Mhi[r][c] = Ai[r * 19 + c];
  double B[49], Bi[49];
  for (int r = 0; r < 7; ++r)
    for (int c = 0; c < 7; ++c) B[r * 7 + c] = M7[r][c] = M7I[r][c];
  gj_inverse(7, B, Bi);
  for (int r = 0; r < 7; ++r)
    for (int c = 0; c < 7; ++c) M7i[r][c] = Bi[r * 7 + c];
  T_ready = 1;
}

void orc_tables(int* c19, double* w19, int* c7, double* Mhat, double* Mhat_inv, double* M7o,
                double* M7_inv) {
  init_tables();
  for (int i = 0; i < 19; ++i) {
    for (int d = 0; d < 3; ++d)
      if (c19) c19[i * 3 + d] = C19[i][d];
    if (w19) w19[i] = W19[i];
  }
  for (int i = 0; i < 7; ++i)
    for (int d = 0; d < 3; ++d)
      if (c7) c7[i * 3 + d] = C7[i][d];
  for (int r = 0; r < 19; ++r)
    for (int c = 0; c < 19; ++c) {
      if (Mhat) Mhat[r * 19 + c] = Mh[r][c];
      if (Mhat_inv) Mhat_inv[r * 19 + c] = Mhi[r][c];
    }
  for (int r = 0; r < 7; ++r)
    for (int c = 0; c < 7; ++c) {
      if (M7o) M7o[r * 7 + c] = M7[r][c];
      if (M7_inv) M7_inv[r * 7 + c] = M7i[r][c];
    }
}

/* -------------------------------------------------------- thermodynamics -- */

/* Eq. 38: a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc, hence Tc. */
double orc_Tc(const orc_params* P) { return 0.0778 * P->a / (0.45724 * P->b * P->R); }

static double kappa_pr(const orc_params* P) {
  return 0.37464 + 1.54226 * P->omega - 0.26992 * P->omega * P->omega;
}

/* xi(T) of Eq. 37 and its T-derivative. */
static double xi_pr(const orc_params* P, double T) {
  double s = 1.0 + kappa_pr(P) * (1.0 - sqrt(T / orc_Tc(P)));
  return s * s;
}
static double dxi_pr(const orc_params* P, double T) {
  double Tc = orc_Tc(P), k = kappa_pr(P);
  double s = 1.0 + k * (1.0 - sqrt(T / Tc));
  return -k * s / sqrt(T * Tc);
}

/* Eq. 37 (Peng-Robinson); eos_kind 1 is the isothermal ideal gas p = c0 rho. */
double orc_p_eos(const orc_params* P, double rho, double T) {
  if (P->eos_kind == 1) return P->eos_c0 * rho;
  double b = P->b;
  return rho * P->R * T / (1.0 - b * rho) -
         P->a * xi_pr(P, T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* (dp_EOS/dT) at constant rho, the derivative of Eq. 37 used in Fbar (Eq. 15). */
double orc_dpdT(const orc_params* P, double rho, double T) {
  if (P->eos_kind == 1) return 0.0;
  double b = P->b;
  return rho * P->R / (1.0 - b * rho) -
         P->a * dxi_pr(P, T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

double orc_dpdrho(const orc_params* P, double rho, double T) {
  if (P->eos_kind == 1) return P->eos_c0;
  double b = P->b, den = 1.0 + 2.0 * b * rho - b * b * rho * rho;
  double a1 = P->R * T / ((1.0 - b * rho) * (1.0 - b * rho));
  double a2 = P->a * xi_pr(P, T) * (2.0 * rho * den - rho * rho * (2.0 * b - 2.0 * b * b * rho)) / (den * den);
  return a1 - a2;
}

/* Antiderivative of p(rho)/rho^2 in rho (closed form for Eq. 37). */
static double pr_A(const orc_params* P, double rho, double T) {
  double b = P->b, s2 = sqrt(2.0);
  double t1 = P->R * T * log(rho / (1.0 - b * rho));
  double t2 = P->a * xi_pr(P, T) / (2.0 * s2 * b) * log((s2 + b * rho - 1.0) / (s2 - b * rho + 1.0));
  return t1 - t2;
}

/* Roots of p(rho) = ps on [lo, hi] by bisection (p assumed monotone there). */
static double bisect_p(const orc_params* P, double T, double ps, double lo, double hi) {
  double flo = orc_p_eos(P, lo, T) - ps;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi), fm = orc_p_eos(P, mid, T) - ps;
    if ((fm < 0) == (flo < 0)) {
      lo = mid;
      flo = fm;
    } else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Maxwell equal-area construction (Sec. 4.2): p(rho_v) = p(rho_l) = p_sat and
 * int_{rho_v}^{rho_l} p/rho^2 drho = p_sat (1/rho_v - 1/rho_l).  Nested
 * bisection between the spinodal pressures.  Returns 0 on success. */
int orc_maxwell(const orc_params* P, double T, double* rho_v, double* rho_l, double* p_sat) {
  if (P->eos_kind != 0 || T >= orc_Tc(P)) return ORC_ERR_ARG;
  double rmax = 1.0 / P->b;
  /* spinodals: first local max and the following local min of p on (0, 1/b) */
  int n = 200000;
  double h = rmax / n, r_max = -1, r_min = -1;
  for (int k = 1; k < n - 1; ++k) {
    double r = k * h;
    double d0 = orc_dpdrho(P, r, T), d1 = orc_dpdrho(P, r + h, T);
    if (r_max < 0 && d0 > 0 && d1 <= 0) r_max = r;
    if (r_max > 0 && d0 < 0 && d1 >= 0) {
      r_min = r;
      break;
    }
  }
  if (r_max < 0 || r_min < 0) return ORC_ERR_ARG;
  double plo = fmax(orc_p_eos(P, r_min, T), 1e-14), phi = orc_p_eos(P, r_max, T);
  double rv = 0, rl = 0, ps = 0;
  for (int it = 0; it < 200; ++it) {
    ps = 0.5 * (plo + phi);
    rv = bisect_p(P, T, ps, 1e-12, r_max);
    rl = bisect_p(P, T, ps, r_min, rmax * (1.0 - 1e-12));
    double area = pr_A(P, rl, T) - pr_A(P, rv, T) - ps * (1.0 / rv - 1.0 / rl);
    /* area > 0 means the chosen p_sat is too low */
    if (area > 0)
      plo = ps;
    else
      phi = ps;
  }
  *rho_v = rv;
  *rho_l = rl;
  if (p_sat) *p_sat = ps;
  return ORC_OK;
}

/* ------------------------------------------------------ per-cell physics -- */

/* Eq. 2 with |u^eq|^2 in the last term. */
void orc_feq19(double rho, const double u[3], double feq[19]) {
  init_tables();
  double cs2 = 1.0 / 3.0, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 19; ++i) {
    double cu = C19[i][0] * u[0] + C19[i][1] * u[1] + C19[i][2] * u[2];
    feq[i] = W19[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
  }
}

/* m^eq = M-hat f^eq (the definition under Eq. 8); with meq_printed the rows
 * 16-18 are replaced by the expressions printed in Eq. 9. */
void orc_meq19(const orc_params* P, double rho, const double u[3], double meq[19]) {
  init_tables();
  double feq[19];
  orc_feq19(rho, u, feq);
  for (int r = 0; r < 19; ++r) {
    double s = 0.0;
    for (int i = 0; i < 19; ++i) s += Mh[r][i] * feq[i];
    meq[r] = s;
  }
  if (P && P->meq_printed) {
    double cs2 = 1.0 / 3.0, uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double base = rho * cs2 * cs2 * (1.0 - 1.5 * uu);
    meq[16] = base + rho * cs2 * (u[0] * u[0] + u[1] * u[1]);
    meq[17] = base + rho * cs2 * (u[0] * u[0] + u[2] * u[2]);
    meq[18] = base + rho * cs2 * (u[1] * u[1] + u[2] * u[2]);
  }
}

/* Eq. 8: m* = m - Lambda (m - m^eq|u^eq) + [m^eq|u^eq+du - m^eq|u^eq], f* = M^-1 m*,
 * with Lambda-hat of Eq. 10 and du = F / rho (Eq. 4). */
void orc_collide19(const orc_params* P, const double f[19], double rho, const double ueq[3],
                   const double F[3], double fstar[19]) {
  init_tables();
  double lam[19] = {1, 1, 1, 1, P->s_e, P->s_v, P->s_v, P->s_v, P->s_v, P->s_v,
                    P->s_q, P->s_q, P->s_q, P->s_q, P->s_q, P->s_q, P->s_pi, P->s_pi, P->s_pi};
  double m[19], meq[19], meq2[19], ms[19], u2[3];
  for (int r = 0; r < 19; ++r) {
    double s = 0.0;
    for (int i = 0; i < 19; ++i) s += Mh[r][i] * f[i];
    m[r] = s;
  }
  for (int d = 0; d < 3; ++d) u2[d] = ueq[d] + F[d] / rho;
  orc_meq19(P, rho, ueq, meq);
  orc_meq19(P, rho, u2, meq2);
  for (int r = 0; r < 19; ++r) ms[r] = m[r] - lam[r] * (m[r] - meq[r]) + (meq2[r] - meq[r]);
  for (int i = 0; i < 19; ++i) {
    double s = 0.0;
    for (int r = 0; r < 19; ++r) s += Mhi[i][r] * ms[r];
    fstar[i] = s;
  }
}

static double lambda_of_rho(const orc_params* P, double rho) {
  /* conductivity interpolated across the interface by the liquid fraction */
  if (P->lambda_l == P->lambda_v) return P->lambda_v;
  double phi = (rho - P->rho_v) / (P->rho_l - P->rho_v);
  if (phi < 0) phi = 0;
  if (phi > 1) phi = 1;
  return P->lambda_v + (P->lambda_l - P->lambda_v) * phi;
}

/* Eq. 13 collision part plus the source of Eq. 15:
 * g* = g - M^-1 Lambda M (g - g^eq) - w Fbar,  Fbar = rho c_v u.grad T + T (dp/dT) div u,
 * grad T = -varsigma sum c_i g_i / c_s^2 (Eqs. 27-29), lambda = (1/varsigma - 1/2) c_s^2. */
void orc_collide7(const orc_params* P, const double g[7], double rho, double T, const double u[3],
                  double divu, double dpdT, double d2T, double gstar[7]) {
  init_tables();
  double cs2 = P->wbar / 3.0;
  double w7[7];
  w7[0] = 1.0 - P->wbar;
  for (int i = 1; i < 7; ++i) w7[i] = P->wbar / 6.0;
  double vs = 1.0 / (lambda_of_rho(P, rho) / cs2 + 0.5);
  double lam[7] = {1.0, vs, vs, vs, 1.0, 1.0, 1.0};
  double gradT[3];
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int i = 0; i < 7; ++i) s += C7[i][d] * g[i];
    gradT[d] = -vs * s / cs2;
  }
  double Fbar = rho * P->cv * (u[0] * gradT[0] + u[1] * gradT[1] + u[2] * gradT[2]) + T * dpdT * divu;
  double geq[7], m[7], meq[7], ms[7];
  for (int i = 0; i < 7; ++i) geq[i] = w7[i] * T;
  for (int r = 0; r < 7; ++r) {
    double s = 0.0, se = 0.0;
    for (int i = 0; i < 7; ++i) {
      s += M7[r][i] * g[i];
      se += M7[r][i] * geq[i];
    }
    m[r] = s;
    meq[r] = se;
  }
  for (int r = 0; r < 7; ++r) ms[r] = m[r] - lam[r] * (m[r] - meq[r]);
  for (int i = 0; i < 7; ++i) {
    double s = 0.0;
    for (int r = 0; r < 7; ++r) s += M7i[i][r] * ms[r];
    /* Eq. 13: + dt F_i with F_i = -w_i Fbar (Eq. 15), + vartheta dt S_i with
       S_i = w_i rho c_v (dt/2) d^2T/dt^2 (Eq. 16), dt = 1 */
    gstar[i] = s - w7[i] * Fbar + P->vartheta * w7[i] * rho * P->cv * 0.5 * d2T;
  }
}

/* Sec. 3.3 constant-pressure boundary written for an arbitrary face with outward
 * normal n: with U = {c.n = -1} unknown, Z = {c.n = 0}, Pp = {c.n = +1},
 *   u_n = [sum_Z f + 2 sum_P f + F.n/2] / rho_b - 1            (Eq. 41 for n = +z)
 *   f_{-n} = f_{n} - rho_b u_n / 3                             (Eq. 42)
 *   f_i  = f_ibar - rho_b u_n/6 - (sig/2)[sum_Z c_a f + F_a/2] + F.n/8
 * for the diagonal unknowns c_i = -n + sig e_a (Eqs. 43-50 for n = +z). */
void orc_zouhe(const orc_params* P, int face, const double F[3], double f[19]) {
  init_tables();
  int ax = face / 2, sg = (face % 2) ? 1 : -1;
  double n[3] = {0, 0, 0};
  n[ax] = sg;
  double rb = P->face_rho[face];
  double SZ = 0, SP = 0, S_t[3] = {0, 0, 0};
  for (int i = 0; i < 19; ++i) {
    double cn = C19[i][0] * n[0] + C19[i][1] * n[1] + C19[i][2] * n[2];
    if (cn == 0) {
      SZ += f[i];
      for (int d = 0; d < 3; ++d) S_t[d] += C19[i][d] * f[i];
    } else if (cn > 0)
      SP += f[i];
  }
  double Fn = F[0] * n[0] + F[1] * n[1] + F[2] * n[2];
  double un = (SZ + 2.0 * SP + 0.5 * Fn) / rb - 1.0;
  for (int i = 0; i < 19; ++i) {
    double cn = C19[i][0] * n[0] + C19[i][1] * n[1] + C19[i][2] * n[2];
    if (cn != -1) continue;
    int ib = OPP19[i];
    double t[3];
    for (int d = 0; d < 3; ++d) t[d] = C19[i][d] + n[d];
    int alpha = -1;
    for (int d = 0; d < 3; ++d)
      if (t[d] != 0) alpha = d;
    if (alpha < 0)
      f[i] = f[ib] - rb * un / 3.0;
    else {
      double sig = t[alpha];
      f[i] = f[ib] - rb * un / 6.0 - 0.5 * sig * (S_t[alpha] + 0.5 * F[alpha]) + Fn / 8.0;
    }
  }
}

/* ------------------------------------------------------------ lattice ------ */

static int dims(const orc_params* P, int a) { return a == 0 ? P->nx : (a == 1 ? P->ny : P->nz); }

int orc_check(const orc_params* P) {
  if (P->nx < 1 || P->ny < 1 || P->nz < 1) return ORC_ERR_ARG;
  if (P->vartheta != 0 && P->vartheta != 1) return ORC_ERR_ARG;
  if (P->lambda_l != P->lambda_v && !(P->rho_l > P->rho_v)) return ORC_ERR_ARG;
  if (!(P->cv > 0) || !(P->wbar > 0 && P->wbar < 1) || !(P->lambda_l > 0) || !(P->lambda_v > 0)) return ORC_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    int k0 = P->face_kind[2 * a], k1 = P->face_kind[2 * a + 1];
    if ((k0 == ORC_PERIODIC) != (k1 == ORC_PERIODIC)) return ORC_ERR_ARG;
    if (k0 != ORC_PERIODIC && dims(P, a) < 3) return ORC_ERR_ARG;
  }
  /* a node layer held at a fixed temperature on a periodic axis needs an inward neighbour */
  for (int f = 0; f < 6; ++f)
    if (P->face_T_fixed[f] && P->face_kind[f] == ORC_PERIODIC && dims(P, f / 2) < 3) return ORC_ERR_ARG;
  /* a wall face may not share an edge with an open face */
  for (int f1 = 0; f1 < 6; ++f1)
    for (int f2 = 0; f2 < 6; ++f2)
      if (f1 / 2 != f2 / 2 && P->face_kind[f1] == ORC_WALL && P->face_kind[f2] == ORC_OPEN) return ORC_ERR_ARG;
  return ORC_OK;
}

/* bit f set <=> the node lies on non-periodic face f */
static int node_faces(const orc_params* P, int x, int y, int z) {
  int q[3] = {x, y, z}, m = 0;
  for (int a = 0; a < 3; ++a) {
    if (P->face_kind[2 * a] == ORC_PERIODIC) continue;
    if (q[a] == 0) m |= 1 << (2 * a);
    if (q[a] == dims(P, a) - 1) m |= 1 << (2 * a + 1);
  }
  return m;
}

/* bit f set <=> the node lies on face f and that face's node layer carries a Dirichlet
 * temperature: every non-periodic face, and a periodic face marked face_T_fixed */
static int node_tfaces(const orc_params* P, int x, int y, int z) {
  int q[3] = {x, y, z}, m = 0;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s) {
      const int f = 2 * a + s;
      if (P->face_kind[f] == ORC_PERIODIC && !P->face_T_fixed[f]) continue;
      if (q[a] == (s ? dims(P, a) - 1 : 0)) m |= 1 << f;
    }
  return m;
}

static int is_wall_node(const orc_params* P, int m) {
  for (int f = 0; f < 6; ++f)
    if ((m >> f & 1) && P->face_kind[f] == ORC_WALL) return 1;
  return 0;
}

int orc_node_class(const orc_params* P, unsigned char* cls) {
  if (orc_check(P)) return ORC_ERR_ARG;
  for (int z = 0; z < P->nz; ++z)
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x) cls[x + P->nx * (y + P->ny * z)] = (unsigned char)node_faces(P, x, y, z);
  return ORC_OK;
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* psi at a possibly out-of-domain lattice point: periodic faces wrap, open faces
 * copy the boundary node, wall faces use the ghost layer of Eq. 36. */
static double psi_at(const orc_params* P, const double* psi, int x, int y, int z) {
  int q[3] = {x, y, z}, out_axes = 0, wall_axis = -1, wall_face = -1;
  int r[3];
  for (int a = 0; a < 3; ++a) {
    int n = dims(P, a), v = q[a];
    if (v >= 0 && v < n) {
      r[a] = v;
      continue;
    }
    int face = 2 * a + (v >= n);
    if (P->face_kind[face] == ORC_PERIODIC) {
      r[a] = wrap(v, n);
      continue;
    }
    out_axes++; /* beyond a non-periodic face */
    if (P->face_kind[face] == ORC_OPEN)
      r[a] = (v < 0) ? 0 : n - 1;
    else {
      r[a] = (v < 0) ? -v : 2 * (n - 1) - v; /* mirror through the wall layer */
      wall_axis = a;
      wall_face = face;
    }
  }
  double val = psi[r[0] + P->nx * (r[1] + P->ny * r[2])];
  if (out_axes == 1 && wall_axis >= 0) {
    double th = P->face_theta_deg[wall_face] * M_PI / 180.0;
    double tn = tan(M_PI / 2.0 - th);
    if (tn != 0.0) {
      /* tangential differences of psi on the wall layer (Eq. 36) */
      int layer = (q[wall_axis] < 0) ? 0 : dims(P, wall_axis) - 1;
      double s2 = 0.0;
      for (int b = 0; b < 3; ++b) {
        if (b == wall_axis) continue;
        int nb = dims(P, b), pp[3], pm[3];
        for (int a = 0; a < 3; ++a) pp[a] = pm[a] = r[a];
        pp[wall_axis] = pm[wall_axis] = layer;
        int up = q[b] + 1, dn = q[b] - 1;
        if (P->face_kind[2 * b] == ORC_PERIODIC) {
          up = wrap(up, nb);
          dn = wrap(dn, nb);
        } else {
          up = up > nb - 1 ? nb - 1 : up;
          dn = dn < 0 ? 0 : dn;
        }
        pp[b] = up;
        pm[b] = dn;
        double d = psi[pp[0] + P->nx * (pp[1] + P->ny * pp[2])] - psi[pm[0] + P->nx * (pm[1] + P->ny * pm[2])];
        s2 += d * d;
      }
      val += sqrt(s2) * tn;
    }
  }
  return val;
}

/* velocity at a possibly out-of-domain point for the div u stencil:
 * zero beyond a wall, boundary copy beyond an open face, periodic wrap. */
static void u_at(const orc_params* P, const double* ux, const double* uy, const double* uz, int x, int y, int z,
                 double out[3]) {
  int q[3] = {x, y, z}, r[3];
  for (int a = 0; a < 3; ++a) {
    int n = dims(P, a), v = q[a];
    if (v >= 0 && v < n) {
      r[a] = v;
      continue;
    }
    int face = 2 * a + (v >= n);
    if (P->face_kind[face] == ORC_WALL) {
      out[0] = out[1] = out[2] = 0.0;
      return;
    }
  }
  for (int a = 0; a < 3; ++a) {
    int n = dims(P, a), v = q[a];
    if (v >= 0 && v < n)
      r[a] = v;
    else if (P->face_kind[2 * a + (v >= n)] == ORC_PERIODIC)
      r[a] = wrap(v, n);
    else
      r[a] = (v < 0) ? 0 : n - 1;
  }
  int c = r[0] + P->nx * (r[1] + P->ny * r[2]);
  out[0] = ux[c];
  out[1] = uy[c];
  out[2] = uz[c];
}

/* Destination of population i leaving cell (x,y,z): returns the flat slot
 * i'*N + c', or -1 if it leaves through an open face.  Bounce-back at a wall
 * face sends it to the opposite direction of the same cell (Eq. 34). */
static long dest19(const orc_params* P, int x, int y, int z, int i) {
  long N = (long)P->nx * P->ny * P->nz;
  int q[3] = {x + C19[i][0], y + C19[i][1], z + C19[i][2]};
  int bounce = 0, drop = 0;
  for (int a = 0; a < 3; ++a) {
    int n = dims(P, a);
    if (q[a] >= 0 && q[a] < n) continue;
    int k = P->face_kind[2 * a + (q[a] >= n)];
    if (k == ORC_PERIODIC)
      q[a] = wrap(q[a], n);
    else if (k == ORC_WALL)
      bounce = 1;
    else
      drop = 1;
  }
  if (bounce) return (long)OPP19[i] * N + x + (long)P->nx * (y + (long)P->ny * z);
  if (drop) return -1;
  return (long)i * N + q[0] + (long)P->nx * (q[1] + (long)P->ny * q[2]);
}

/* Destination of D3Q7 population i from cell (x,y,z), or -1 if it leaves the lattice. */
static long dest7(const orc_params* P, int x, int y, int z, int i) {
  long N = (long)P->nx * P->ny * P->nz;
  int q[3] = {x + C7[i][0], y + C7[i][1], z + C7[i][2]};
  for (int a = 0; a < 3; ++a) {
    int n = dims(P, a);
    if (q[a] >= 0 && q[a] < n) continue;
    if (P->face_kind[2 * a + (q[a] >= n)] != ORC_PERIODIC) return -1;
    q[a] = wrap(q[a], n);
  }
  return (long)i * N + q[0] + (long)P->nx * (q[1] + (long)P->ny * q[2]);
}

int orc_stream_map19(const orc_params* P, int* dst) {
  init_tables();
  if (orc_check(P)) return ORC_ERR_ARG;
  long N = (long)P->nx * P->ny * P->nz;
  for (int z = 0; z < P->nz; ++z)
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x)
        for (int i = 0; i < 19; ++i)
          dst[(long)i * N + x + (long)P->nx * (y + (long)P->ny * z)] = (int)dest19(P, x, y, z, i);
  return ORC_OK;
}

int orc_stream_map7(const orc_params* P, int* dst) {
  init_tables();
  if (orc_check(P)) return ORC_ERR_ARG;
  long N = (long)P->nx * P->ny * P->nz;
  for (int z = 0; z < P->nz; ++z)
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x)
        for (int i = 0; i < 7; ++i)
          dst[(long)i * N + x + (long)P->nx * (y + (long)P->ny * z)] = (int)dest7(P, x, y, z, i);
  return ORC_OK;
}

static double face_T_at(const orc_params* P, const double* const* Tface, int face, int x, int y, int z) {
  int a = face / 2, q[3] = {x, y, z}, t[2], k = 0;
  for (int b = 0; b < 3; ++b)
    if (b != a) t[k++] = b;
  if (Tface && Tface[face]) return Tface[face][q[t[0]] + dims(P, t[0]) * q[t[1]]];
  return P->face_T[face];
}

/* Steps 1-4: macroscopic fields at time t. */
static int fields_t(const orc_params* P, const double* f, const double* g, double* rho, double* jx, double* jy,
                    double* jz, double* T, double* pe, double* dpdT, double* psi, double* Fx, double* Fy,
                    double* Fz, double* ux, double* uy, double* uz) {
  long N = (long)P->nx * P->ny * P->nz;
  int nonfinite = 0, psi_bad = 0; /* a non-finite population outranks a psi-domain error */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : nonfinite, psi_bad)
#endif
  for (long c = 0; c < N; ++c) {
    double r = 0, j[3] = {0, 0, 0}, t = 0;
    for (int i = 0; i < 19; ++i) {
      double v = f[i * N + c];
      if (!isfinite(v)) nonfinite = 1;
      r += v;
      for (int d = 0; d < 3; ++d) j[d] += C19[i][d] * v;
    }
    for (int i = 0; i < 7; ++i) {
      if (!isfinite(g[i * N + c])) nonfinite = 1;
      t += g[i * N + c];
    }
    rho[c] = r;
    jx[c] = j[0];
    jy[c] = j[1];
    jz[c] = j[2];
    T[c] = t;
    pe[c] = orc_p_eos(P, r, t);
    dpdT[c] = orc_dpdT(P, r, t);
    double arg = 2.0 * (pe[c] - r / 3.0) / P->G; /* Eq. 7 with dx = dt = 1, c_s^2 = 1/3 */
    if (!(arg >= 0.0)) {
      psi_bad = 1;
      psi[c] = NAN;
    } else
      psi[c] = sqrt(arg);
  }
  const int st = nonfinite ? ORC_ERR_NONFINITE : (psi_bad ? ORC_ERR_PSI_DOMAIN : ORC_OK);
  ORC_PAR_Z
  for (int z = 0; z < P->nz; ++z)
    for (int y = 0; y < P->ny; ++y)
      for (int x = 0; x < P->nx; ++x) {
        long c = x + (long)P->nx * (y + (long)P->ny * z);
        double s[3] = {0, 0, 0};
        for (int i = 1; i < 19; ++i) {
          double pn = psi_at(P, psi, x + C19[i][0], y + C19[i][1], z + C19[i][2]);
          for (int d = 0; d < 3; ++d) s[d] += VARPI[i] * pn * C19[i][d];
        }
        Fx[c] = -P->G * psi[c] * s[0];
        Fy[c] = -P->G * psi[c] * s[1];
        Fz[c] = -P->G * psi[c] * s[2];
        if (is_wall_node(P, node_faces(P, x, y, z)))
          ux[c] = uy[c] = uz[c] = 0.0;
        else {
          ux[c] = (jx[c] + 0.5 * Fx[c]) / rho[c];
          uy[c] = (jy[c] + 0.5 * Fy[c]) / rho[c];
          uz[c] = (jz[c] + 0.5 * Fz[c]) / rho[c];
        }
      }
  return st;
}

typedef struct {
  double *rho, *jx, *jy, *jz, *T, *pe, *dpdT, *psi, *Fx, *Fy, *Fz, *ux, *uy, *uz;
  double* block;
} work_t;

static int work_alloc(work_t* w, long N) {
  w->block = (double*)malloc(sizeof(double) * 14 * N);
  if (!w->block) return -1;
  double** p[14] = {&w->rho, &w->jx, &w->jy, &w->jz, &w->T, &w->pe, &w->dpdT,
                    &w->psi, &w->Fx, &w->Fy, &w->Fz, &w->ux, &w->uy, &w->uz};
  for (int k = 0; k < 14; ++k) *p[k] = w->block + k * N;
  return 0;
}

static void copy_fields(const work_t* w, long N, orc_fields* o) {
  if (!o) return;
  double* src[11] = {w->rho, w->T, w->psi, w->pe, w->dpdT, w->ux, w->uy, w->uz, w->Fx, w->Fy, w->Fz};
  double* dst[11] = {o->rho, o->T, o->psi, o->p, o->dpdT, o->ux, o->uy, o->uz, o->Fx, o->Fy, o->Fz};
  for (int k = 0; k < 11; ++k)
    if (dst[k]) memcpy(dst[k], src[k], sizeof(double) * N);
}

int orc_macros(const orc_params* P, const double* f, const double* g, orc_fields* out) {
  init_tables();
  if (orc_check(P)) return ORC_ERR_ARG;
  long N = (long)P->nx * P->ny * P->nz;
  work_t w;
  if (work_alloc(&w, N)) return ORC_ERR_ARG;
  int st = fields_t(P, f, g, w.rho, w.jx, w.jy, w.jz, w.T, w.pe, w.dpdT, w.psi, w.Fx, w.Fy, w.Fz, w.ux, w.uy, w.uz);
  copy_fields(&w, N, out);
  free(w.block);
  return st;
}

/* One step.  Th (2N, NULL when vartheta = 0): T at t-1 and t-2; d^2T/dt^2 at t is the
 * backward second difference T(t) - 2 T(t-1) + T(t-2) (dt = 1).  Tho (2N): T at t and
 * t-1 for the next step. */
static int step_impl(const orc_params* P, const double* const* Tface, const double* f, const double* g,
                     const double* Th, double* fo, double* go, double* Tho, orc_fields* diag) {
  init_tables();
  if (orc_check(P)) return ORC_ERR_ARG;
  if (P->vartheta && (!Th || !Tho)) return ORC_ERR_ARG;
  const int nx = P->nx, ny = P->ny, nz = P->nz;
  const long N = (long)nx * ny * nz;
  work_t w;
  if (work_alloc(&w, N)) return ORC_ERR_ARG;
  double* fs = (double*)malloc(sizeof(double) * 19 * N);
  double* gs = (double*)malloc(sizeof(double) * 7 * N);

  /* steps 1-4 */
  int st = fields_t(P, f, g, w.rho, w.jx, w.jy, w.jz, w.T, w.pe, w.dpdT, w.psi, w.Fx, w.Fy, w.Fz, w.ux, w.uy, w.uz);
  copy_fields(&w, N, diag);

  /* step 5: D3Q19 collision at every node, wall and open-face nodes included */
  ORC_PAR_Z
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long c = x + (long)nx * (y + (long)ny * z);
        double fl[19], fsl[19], ueq[3], F[3] = {w.Fx[c], w.Fy[c], w.Fz[c]};
        for (int i = 0; i < 19; ++i) fl[i] = f[i * N + c];
        if (P->wall_ueq_zero && is_wall_node(P, node_faces(P, x, y, z)))
          ueq[0] = ueq[1] = ueq[2] = 0.0;
        else {
          ueq[0] = w.jx[c] / w.rho[c];
          ueq[1] = w.jy[c] / w.rho[c];
          ueq[2] = w.jz[c] / w.rho[c];
        }
        orc_collide19(P, fl, w.rho[c], ueq, F, fsl);
        for (int i = 0; i < 19; ++i) fs[i * N + c] = fsl[i];
      }

  /* step 6: streaming with bounce-back; slots nobody writes stay NaN */
  for (long k = 0; k < 19 * N; ++k) fo[k] = NAN;
  ORC_PAR_Z
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        for (int i = 0; i < 19; ++i) {
          long d = dest19(P, x, y, z, i);
          if (d >= 0) fo[d] = fs[i * N + x + (long)nx * (y + (long)ny * z)];
        }

  /* step 7: open faces */
  ORC_PAR_Z
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int m = node_faces(P, x, y, z);
        int nopen = 0, nnp = 0, face = -1;
        double rb = 0.0;
        for (int fc = 0; fc < 6; ++fc)
          if (m >> fc & 1) {
            nnp++;
            if (P->face_kind[fc] == ORC_OPEN) {
              nopen++;
              face = fc;
              rb += P->face_rho[fc];
            }
          }
        if (nopen == 0) continue;
        long c = x + (long)nx * (y + (long)ny * z);
        double fl[19];
        for (int i = 0; i < 19; ++i) fl[i] = fo[i * N + c];
        if (nnp == 1) {
          double F[3] = {w.Fx[c], w.Fy[c], w.Fz[c]};
          orc_zouhe(P, face, F, fl);
        } else {
          /* edge / corner of open faces: every unknown population := f^eq(rho_b, 0) */
          double feq[19], u0[3] = {0, 0, 0};
          orc_feq19(rb / nopen, u0, feq);
          int q[3] = {x, y, z};
          for (int i = 0; i < 19; ++i) {
            int unknown = 0;
            for (int a = 0; a < 3; ++a) {
              int s = q[a] - C19[i][a];
              if ((s < 0 || s >= dims(P, a)) && P->face_kind[2 * a] != ORC_PERIODIC) unknown = 1;
            }
            if (unknown) fl[i] = feq[i];
          }
        }
        for (int i = 0; i < 19; ++i) fo[i * N + c] = fl[i];
      }

  /* step 8: D3Q7 collision */
  ORC_PAR_Z
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long c = x + (long)nx * (y + (long)ny * z);
        double divu = 0.0;
        for (int i = 1; i < 19; ++i) {
          double un[3];
          u_at(P, w.ux, w.uy, w.uz, x + C19[i][0], y + C19[i][1], z + C19[i][2], un);
          divu += W19[i] * (C19[i][0] * un[0] + C19[i][1] * un[1] + C19[i][2] * un[2]);
        }
        divu *= 3.0; /* 1 / c_s-hat^2 */
        double gl[7], gsl[7], u[3] = {w.ux[c], w.uy[c], w.uz[c]};
        for (int i = 0; i < 7; ++i) gl[i] = g[i * N + c];
        const double d2T = Th ? w.T[c] - 2.0 * Th[c] + Th[N + c] : 0.0;
        orc_collide7(P, gl, w.rho[c], w.T[c], u, divu, w.dpdT[c], d2T, gsl);
        for (int i = 0; i < 7; ++i) gs[i * N + c] = gsl[i];
      }

  /* step 9: relaxed streaming, rho c_v at the destination */
  for (long k = 0; k < 7 * N; ++k) go[k] = g[k];
  ORC_PAR_Z
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        for (int i = 0; i < 7; ++i) {
          long d = dest7(P, x, y, z, i);
          if (d < 0) continue;
          long yc = d - (long)i * N;
          double gold = g[d];
          go[d] = gold + (gs[i * N + x + (long)nx * (y + (long)ny * z)] - gold) / (w.rho[yc] * P->cv);
        }

  /* step 10: non-equilibrium extrapolation at every Dirichlet node */
  {
    double w7[7];
    w7[0] = 1.0 - P->wbar;
    for (int i = 1; i < 7; ++i) w7[i] = P->wbar / 6.0;
    ORC_PAR_Z
  for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          int m = node_tfaces(P, x, y, z);
          if (!m) continue;
          int q[3] = {x, y, z}, nf = 0;
          double Tb = 0.0;
          for (int fc = 0; fc < 6; ++fc)
            if (m >> fc & 1) {
              q[fc / 2] += (fc % 2) ? -1 : 1; /* step inward */
              Tb += face_T_at(P, Tface, fc, x, y, z);
              nf++;
            }
          Tb /= nf;
          long cb = x + (long)nx * (y + (long)ny * z);
          long cf = q[0] + (long)nx * (q[1] + (long)ny * q[2]);
          double Tf = 0.0;
          for (int i = 0; i < 7; ++i) Tf += go[i * N + cf];
          for (int i = 0; i < 7; ++i) go[i * N + cb] = w7[i] * Tb + go[i * N + cf] - w7[i] * Tf;
        }
  }

  if (Tho)
    for (long c = 0; c < N; ++c) {
      Tho[N + c] = Th[c];
      Tho[c] = w.T[c];
    }

  free(fs);
  free(gs);
  free(w.block);
  return st;
}

int orc_step(const orc_params* P, const double* const* Tface, const double* f, const double* g, double* fo,
             double* go, orc_fields* diag) {
  return step_impl(P, Tface, f, g, NULL, fo, go, NULL, diag);
}

int orc_step_hist(const orc_params* P, const double* const* Tface, const double* f, const double* g,
                  const double* Th, double* fo, double* go, double* Tho) {
  return step_impl(P, Tface, f, g, Th, fo, go, Tho, NULL);
}

int orc_run_hist(const orc_params* P, const double* const* Tface, double* f, double* g, double* Th, int nsteps) {
  long N = (long)P->nx * P->ny * P->nz;
  double* f2 = (double*)malloc(sizeof(double) * 19 * N);
  double* g2 = (double*)malloc(sizeof(double) * 7 * N);
  double* T2 = (double*)malloc(sizeof(double) * 2 * N);
  int st = ORC_OK;
  for (int s = 0; s < nsteps; ++s) {
    int r = step_impl(P, Tface, f, g, Th, f2, g2, T2, NULL);
    memcpy(f, f2, sizeof(double) * 19 * N);
    memcpy(g, g2, sizeof(double) * 7 * N);
    memcpy(Th, T2, sizeof(double) * 2 * N);
    if (r != ORC_OK) {
      st = r;
      break;
    }
  }
  free(f2);
  free(g2);
  free(T2);
  return st;
}

int orc_run(const orc_params* P, const double* const* Tface, double* f, double* g, int nsteps) {
  long N = (long)P->nx * P->ny * P->nz;
  double* f2 = (double*)malloc(sizeof(double) * 19 * N);
  double* g2 = (double*)malloc(sizeof(double) * 7 * N);
  int st = ORC_OK;
  for (int s = 0; s < nsteps; ++s) {
    int r = orc_step(P, Tface, f, g, f2, g2, NULL);
    memcpy(f, f2, sizeof(double) * 19 * N);
    memcpy(g, g2, sizeof(double) * 7 * N);
    if (r != ORC_OK) {
      st = r;
      break;
    }
  }
  free(f2);
  free(g2);
  return st;
}

/* Initial populations (Sec. 4.2): f = f^eq(rho0, 0), g = w_i T0. */
void orc_init_state(const orc_params* P, const double* rho0, const double* T0, double* f, double* g) {
  init_tables();
  long N = (long)P->nx * P->ny * P->nz;
  double u0[3] = {0, 0, 0}, feq[19];
  for (long c = 0; c < N; ++c) {
    orc_feq19(rho0[c], u0, feq);
    for (int i = 0; i < 19; ++i) f[i * N + c] = feq[i];
    g[c] = (1.0 - P->wbar) * T0[c];
    for (int i = 1; i < 7; ++i) g[i * N + c] = P->wbar / 6.0 * T0[c];
  }
}

/* Threads the per-cell loops use: n > 0 sets it (OpenMP build only); returns the count in
 * effect (1 in the serial build). */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
