// Host-side harness: exposes the CUDA library's per-cell FP32 arithmetic
// (lbm_cell.cuh, compiled for the host) so that CPU tests can compare it with
// the FP64 oracle cell by cell.  Test infrastructure only.
#include "lbm_cell.cuh"

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
  P.meq_printed = k[0]; P.eos_kind = k[1]; P.vartheta = k[2];
  return P;
}

extern "C" {
void h_collide19(const double* d, const int* k, const float* f, float rho, const float* u, const float* F, float* fs) {
  Params P = make(d, k);
  collide19(P, f, rho, u[0], u[1], u[2], F[0], F[1], F[2], fs);
}
void h_collide7(const double* d, const int* k, const float* g, float rho, float T, const float* u, float divu,
                float dpdT, float d2T, float* gs) {
  Params P = make(d, k);
  collide7(P, g, rho, T, u[0], u[1], u[2], divu, dpdT, d2T, gs);
}
void h_zouhe(int face, float rho_b, const float* F, float* f) { zouhe(face, rho_b, F[0], F[1], F[2], f); }
void h_eos(const double* d, const int* k, float rho, float T, float* out) {
  Params P = make(d, k);
  float p, dpdT, psi;
  eos_pr(P, rho, T, p, dpdT);
  out[3] = psi_of(P, rho, p, psi) ? 1.f : 0.f;
  out[0] = p; out[1] = dpdT; out[2] = psi;
}
void h_feq19(float rho, const float* u, float* fe) { feq19(rho, u[0], u[1], u[2], fe); }
}

extern "C" unsigned h_fdiv_check(unsigned d, unsigned nmax, unsigned step) {
  unsigned mul, shr;
  fdiv_init(d, mul, shr);
  unsigned bad = 0;
  for (unsigned long long n = 0; n < nmax; n += step)
    if (fdiv((unsigned)n, mul, shr) != (unsigned)n / d) ++bad;
  if (fdiv(nmax - 1, mul, shr) != (nmax - 1) / d) ++bad;
  return bad;
}
