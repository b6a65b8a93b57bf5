// Host-side harness for the per-cell vector-Jacobian products of the adjoint
// (lbm_adjoint_cell.cuh), instantiated in double next to the double forward
// functions, so that CPU tests can compare each product with central
// differences of the forward.  Test infrastructure only.
#include "lbm_adjoint_cell.cuh"

using namespace lbm;

static Params make(const double* d, const int* k) {
  Params P = {};
  P.a = (float)d[0]; P.b = (float)d[1]; P.R = (float)d[2]; P.kappa = (float)d[3]; P.inv_Tc = (float)d[4];
  P.G = (float)d[5]; P.inv_G = (float)(1.0 / d[5]); P.eos_c0 = (float)d[6];
  P.s_e = (float)d[7]; P.s_v = (float)d[8]; P.s_q = (float)d[9]; P.s_pi = (float)d[10];
  P.cv = (float)d[11]; P.inv_cv = (float)(1.0 / d[11]); P.wbar = (float)d[12]; P.inv_cs2t = (float)(3.0 / d[12]);
  P.lambda_l = (float)d[13]; P.lambda_v = (float)d[14]; P.rho_l = (float)d[15]; P.rho_v = (float)d[16];
  P.inv_drho = d[15] > d[16] ? (float)(1.0 / (d[15] - d[16])) : 0.f;
  P.lam_uniform = d[13] == d[14];
  P.meq_printed = k[0]; P.eos_kind = k[1];
  return P;
}

extern "C" {
// forward: f (19), F (3) -> f* (19), with rho = sum f and u^eq = j/rho or 0
void a_collide19(const double* d, const int* k, const double* f, int ueq_from_f, const double* F, double* fs) {
  Params P = make(d, k);
  double rho = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < 19; ++i) {
    rho += f[i];
    j[0] += c19x(i) * f[i];
    j[1] += c19y(i) * f[i];
    j[2] += c19z(i) * f[i];
  }
  const double u[3] = {ueq_from_f ? j[0] / rho : 0.0, ueq_from_f ? j[1] / rho : 0.0, ueq_from_f ? j[2] / rho : 0.0};
  collide19(P, f, rho, u[0], u[1], u[2], F[0], F[1], F[2], fs);
}
// the closed-form collision of the rate-1 case, same inputs as a_collide19
void a_collide19_fast(const double* d, const int* k, const double* f, int ueq_from_f, const double* F, double* fs) {
  Params P = make(d, k);
  double rho = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < 19; ++i) {
    rho += f[i];
    j[0] += c19x(i) * f[i];
    j[1] += c19y(i) * f[i];
    j[2] += c19z(i) * f[i];
  }
  const double u[3] = {ueq_from_f ? j[0] / rho : 0.0, ueq_from_f ? j[1] / rho : 0.0, ueq_from_f ? j[2] / rho : 0.0};
  collide19_fast(P, f, rho, u[0], u[1], u[2], F[0], F[1], F[2], fs);
}
void a_collide19_vjp(const double* d, const int* k, const double* f, int ueq_from_f, const double* F,
                     const double* fsb, double* fb, double* Fb) {
  Params P = make(d, k);
  collide19_vjp(P, f, ueq_from_f != 0, F, fsb, fb, Fb);
}
void a_collide19_fast_vjp(const double* d, const int* k, const double* f, int ueq_from_f, const double* F,
                          const double* fsb, double* fb, double* Fb) {
  Params P = make(d, k);
  collide19_fast_vjp(P, f, ueq_from_f != 0, F, fsb, fb, Fb);
}
// forward: x = (g[7], rho, u[3], divu, dpdT) -> g* (7), T = sum g
void a_collide7(const double* d, const int* k, const double* x, double* gs) {
  Params P = make(d, k);
  double T = 0;
  for (int i = 0; i < 7; ++i) T += x[i];
  collide7(P, x, x[7], T, x[8], x[9], x[10], x[11], x[12], 0.0, gs);
}
void a_collide7_vjp(const double* d, const int* k, const double* x, const double* gsb, double* xb) {
  Params P = make(d, k);
  double T = 0;
  for (int i = 0; i < 7; ++i) T += x[i];
  double gb[7], rhob, Tb, ub[3], divub, dpdTb;
  collide7_vjp(P, x, x[7], T, x + 8, x[11], x[12], gsb, gb, rhob, Tb, ub, divub, dpdTb);
  for (int i = 0; i < 7; ++i) xb[i] = gb[i] + Tb;
  xb[7] = rhob;
  xb[8] = ub[0]; xb[9] = ub[1]; xb[10] = ub[2];
  xb[11] = divub;
  xb[12] = dpdTb;
}
// forward: x = (f[19], F[3]) -> f after the rule (19)
void a_zouhe(int face, double rho_b, const double* x, double* fo) {
  for (int i = 0; i < 19; ++i) fo[i] = x[i];
  zouhe(face, rho_b, x[19], x[20], x[21], fo);
}
void a_zouhe_vjp(int face, double rho_b, const double* fob, double* xb) {
  double fb[19], Fb[3] = {0, 0, 0};
  for (int i = 0; i < 19; ++i) fb[i] = fob[i];
  zouhe_vjp(face, rho_b, fb, Fb);
  for (int i = 0; i < 19; ++i) xb[i] = fb[i];
  xb[19] = Fb[0]; xb[20] = Fb[1]; xb[21] = Fb[2];
}
// forward: (rho, T) -> (psi, dp/dT)
void a_eos(const double* d, const int* k, double rho, double T, double* out) {
  Params P = make(d, k);
  double p, dpdT, psi;
  eos_pr(P, rho, T, p, dpdT);
  psi_of(P, rho, p, psi);
  out[0] = psi;
  out[1] = dpdT;
}
void a_eos_vjp(const double* d, const int* k, double rho, double T, double psib, double dpdTb, double* out) {
  Params P = make(d, k);
  double p, dpdT, psi;
  eos_pr(P, rho, T, p, dpdT);
  psi_of(P, rho, p, psi);
  double rb = 0, Tb = 0;
  psi_dpdT_vjp(P, rho, T, psi, psib, dpdTb, rb, Tb);
  out[0] = rb;
  out[1] = Tb;
}
}
