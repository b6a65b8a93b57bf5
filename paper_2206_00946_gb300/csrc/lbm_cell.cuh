// Per-cell arithmetic of the thermal pseudopotential MRT-LBM step
// (Huang, Wang, He & Huang, arXiv 2206.00946), FP32, written for registers:
// the D3Q19 transform M-hat and its inverse are expanded by hand into
// sparse sums, the equilibrium moments and the exact-difference forcing
// increments are evaluated in closed form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

// Device functions of the phase code (lbm_lattice.cuh, lbm_phases.cuh); host
// functions as well when LBM_HOST_PHASES is defined, for a CPU harness that runs
// the same per-cell code.
#if defined(LBM_HOST_PHASES)
#define LBM_DEV __host__ __device__ __forceinline__
#else
#define LBM_DEV __device__ __forceinline__
#endif

namespace lbm {

// ---------------------------------------------------------------- lattices --
// D3Q19 velocities in the order of the appendix matrix (rows 1-3 of M-hat).
LBM_HD constexpr int c19x(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
LBM_HD constexpr int c19y(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
LBM_HD constexpr int c19z(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
LBM_HD constexpr int opp19(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// D3Q19 weights (Eq. 2) and interaction weights varpi(|c|^2) (Eq. 6).
LBM_HD constexpr float w19(int i) { return i == 0 ? (1.f / 3.f) : (i < 7 ? (1.f / 18.f) : (1.f / 36.f)); }
LBM_HD constexpr float varpi19(int i) { return i == 0 ? 0.f : (i < 7 ? (1.f / 6.f) : (1.f / 12.f)); }
// D3Q7 velocities: 0 rest, 1/2 +-x, 3/4 +-y, 5/6 +-z.
LBM_HD constexpr int c7x(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
LBM_HD constexpr int c7y(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
LBM_HD constexpr int c7z(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }

enum { FACE_PERIODIC = 0, FACE_WALL = 1, FACE_OPEN = 2 };
enum { ERRF_NONFINITE = 1, ERRF_PSI = 2, ERRF_TIMEOUT = 4 };

// Reciprocal: CUDA's fast division intrinsic on the device (within 2 ulp for
// divisors of magnitude 2^-126 .. 2^126; every operand here is a density, a
// temperature or a sum of rates), IEEE division on the host.
LBM_HD float rcp(float x) {
#if defined(__CUDA_ARCH__)
  return __fdividef(1.f, x);
#else
  return 1.f / x;
#endif
}

LBM_HD double rcp(double x) { return 1.0 / x; }

// Division of a non-negative 32-bit value (< 2^31) by a runtime divisor d with a
// precomputed multiplier: q = umulhi(n, mul) >> shr (mul = 0 means d = 1).
LBM_HD unsigned fdiv(unsigned n, unsigned mul, unsigned shr) {
#if defined(__CUDA_ARCH__)
  return mul ? (__umulhi(n, mul) >> shr) : n;
#else
  return mul ? ((unsigned)(((unsigned long long)n * mul) >> 32) >> shr) : n;
#endif
}

inline void fdiv_init(unsigned d, unsigned& mul, unsigned& shr) {
  if (d <= 1) {
    mul = 0;
    shr = 0;
    return;
  }
  unsigned l = 0;
  while ((1ull << l) < d) ++l;  // ceil(log2 d)
  const unsigned long long p = 31ull + l;
  mul = (unsigned)(((1ull << p) + d - 1) / d);
  shr = (unsigned)(p - 32);
}

struct Params {
  int nx, ny, nz;
  long long N;
  unsigned dnx_mul, dnx_shr, dny_mul, dny_shr;
  // boundary nodes, enumerated plane by plane (see boundary_candidate)
  int bd_zplanes, bd_perim;
  unsigned dpl_mul, dpl_shr, dper_mul, dper_shr;
  long long bd_total;
  int meq_printed, wall_ueq_zero, eos_kind;
  int vartheta;  // 1: the correction S_i of Eqs. 13 and 16 (needs the T history of Aux)
  float a, b, R, kappa, inv_Tc, G, inv_G, eos_c0;
  float s_e, s_v, s_q, s_pi;
  float cv, inv_cv, wbar, inv_cs2t;  // c_s^2 of D3Q7 = wbar/3
  float lambda_l, lambda_v, rho_l, rho_v, inv_drho;
  float rho_ref, T_ref;  // shifts of the 16-bit population storage
  int lam_uniform;
  int fast19;  // s_q = s_pi = 1 and m^eq = M-hat f^eq: collide19_fast is exact
  int face_kind[6];
  float face_rho[6];
  float tan_wet[6];  // tan(pi/2 - theta) of each wall face (Eq. 36)
  const float* Tface[6];  // per-node Dirichlet temperature of each face that holds one (tface)
  int any_nonperiodic;
  int tface[6];  // 1: the node layer of face f holds a Dirichlet T (non-periodic, or held)
};

// --------------------------------------------------------------- thermo ----
// Peng-Robinson EOS (Eq. 37) with xi(T) = [1 + kappa (1 - sqrt(T/Tc))]^2, its
// T-derivative at constant rho, and psi of Eq. 7 (dx = dt = 1, c_s-hat^2 = 1/3).
template <typename R>
LBM_HD void eos_pr(const Params& P, R rho, R T, R& p, R& dpdT) {
  if (P.eos_kind == 1) {
    p = P.eos_c0 * rho;
    dpdT = R(0);
    return;
  }
  const R sr = sqrt(T * P.inv_Tc);
  const R s = R(1) + P.kappa * (R(1) - sr);
  const R xi = s * s;
  // d xi / dT = -kappa s / sqrt(T Tc) = -kappa s sr / T
  const R dxi = -P.kappa * s * sr * rcp(T);
  const R br = P.b * rho;
  const R inv1 = rcp(R(1) - br);
  const R den = R(1) + br * (R(2) - br);
  const R att = P.a * rho * rho * rcp(den);
  p = rho * P.R * T * inv1 - xi * att;
  dpdT = rho * P.R * inv1 - dxi * att;
}

// psi^2 = 2 (p - rho/3) / G.  Returns false when the argument is negative.
template <typename R>
LBM_HD bool psi_of(const Params& P, R rho, R p, R& psi) {
  const R arg = R(2) * (p - rho * (R(1) / R(3))) * P.inv_G;
  if (!(arg >= R(0))) {
    psi = R(0);
    return false;
  }
  psi = sqrt(arg);
  return true;
}

// ----------------------------------------------------------- D3Q19 MRT -----
// Collision of Eq. 8 for one cell: m = M-hat f; m* = m - Lambda (m - m^eq(u)) +
// [m^eq(u + F/rho) - m^eq(u)]; f* = M-hat^-1 m*.  m^eq is M-hat f^eq in closed form
// (rows 16-18 optionally as printed in Eq. 9).  u is u^eq (zero at wall nodes).
template <typename R>
LBM_HD void collide19(const Params& P, const R* f, R rho, R ux, R uy, R uz, R Fx,
                      R Fy, R Fz, R* fs) {
  // raw moments, rows 4..18 of M-hat
  const R s7_10 = f[7] + f[8] + f[9] + f[10];
  const R s11_14 = f[11] + f[12] + f[13] + f[14];
  const R s15_18 = f[15] + f[16] + f[17] + f[18];
  const R a12 = f[1] + f[2], a34 = f[3] + f[4], a56 = f[5] + f[6];
  const R m4 = a12 + a34 + a56 + R(2) * (s7_10 + s11_14 + s15_18);
  const R m5 = R(2) * a12 - a34 - a56 + s7_10 + s11_14 - R(2) * s15_18;
  const R m6 = a34 - a56 + s7_10 - s11_14;
  const R m7 = f[7] + f[8] - f[9] - f[10];
  const R m8 = f[11] + f[12] - f[13] - f[14];
  const R m9 = f[15] + f[16] - f[17] - f[18];
  const R m10 = f[7] - f[8] - f[9] + f[10];
  const R m11 = f[7] - f[8] + f[9] - f[10];
  const R m12 = f[11] - f[12] - f[13] + f[14];
  const R m13 = f[11] - f[12] + f[13] - f[14];
  const R m14 = f[15] - f[16] - f[17] + f[18];
  const R m15 = f[15] - f[16] + f[17] - f[18];
  const R m16 = s7_10, m17 = s11_14, m18 = s15_18;

  const R ir = rcp(rho);
  const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
  // rho (u'_a^2 - u_a^2) with u' = u + F/rho
  const R qx = R(2) * ux * Fx + Fx * Fx * ir;
  const R qy = R(2) * uy * Fy + Fy * Fy * ir;
  const R qz = R(2) * uz * Fz + Fz * Fz * ir;
  const R third = R(1) / R(3), ninth = R(1) / R(9), sixth = R(1) / R(6);

  const R e4 = rho * (R(1) + uxx + uyy + uzz), d4 = qx + qy + qz;
  const R e5 = rho * (R(2) * uxx - uyy - uzz), d5 = R(2) * qx - qy - qz;
  const R e6 = rho * (uyy - uzz), d6 = qy - qz;
  const R e7 = rho * ux * uy, d7 = ux * Fy + Fx * uy + Fx * Fy * ir;
  const R e8 = rho * ux * uz, d8 = ux * Fz + Fx * uz + Fx * Fz * ir;
  const R e9 = rho * uy * uz, d9 = uy * Fz + Fy * uz + Fy * Fz * ir;
  const R e10 = third * rho * uy, e11 = third * rho * ux, e12 = third * rho * uz;
  R e16, e17, e18, d16, d17, d18;
  if (P.meq_printed) {
    const R base = ninth * rho - sixth * rho * (uxx + uyy + uzz), db = -sixth * d4;
    e16 = base + third * rho * (uxx + uyy);
    e17 = base + third * rho * (uxx + uzz);
    e18 = base + third * rho * (uyy + uzz);
    d16 = db + third * (qx + qy);
    d17 = db + third * (qx + qz);
    d18 = db + third * (qy + qz);
  } else {
    e16 = ninth * rho - sixth * rho * uzz + third * rho * (uxx + uyy);
    e17 = ninth * rho - sixth * rho * uyy + third * rho * (uxx + uzz);
    e18 = ninth * rho - sixth * rho * uxx + third * rho * (uyy + uzz);
    d16 = -sixth * qz + third * (qx + qy);
    d17 = -sixth * qy + third * (qx + qz);
    d18 = -sixth * qx + third * (qy + qz);
  }
  const R se = P.s_e, sv = P.s_v, sq = P.s_q, sp = P.s_pi;
  // post-collision moments
  const R n0 = rho;
  const R n1 = rho * ux + Fx, n2 = rho * uy + Fy, n3 = rho * uz + Fz;
  const R n4 = m4 - se * (m4 - e4) + d4;
  const R n5 = m5 - sv * (m5 - e5) + d5;
  const R n6 = m6 - sv * (m6 - e6) + d6;
  const R n7 = m7 - sv * (m7 - e7) + d7;
  const R n8 = m8 - sv * (m8 - e8) + d8;
  const R n9 = m9 - sv * (m9 - e9) + d9;
  const R n10 = m10 - sq * (m10 - e10) + third * Fy;
  const R n11 = m11 - sq * (m11 - e11) + third * Fx;
  const R n12 = m12 - sq * (m12 - e12) + third * Fz;
  const R n13 = m13 - sq * (m13 - e11) + third * Fx;
  const R n14 = m14 - sq * (m14 - e12) + third * Fz;
  const R n15 = m15 - sq * (m15 - e10) + third * Fy;
  const R n16 = m16 - sp * (m16 - e16) + d16;
  const R n17 = m17 - sp * (m17 - e17) + d17;
  const R n18 = m18 - sp * (m18 - e18) + d18;

  // f* = M-hat^-1 m*, solved by hand from the block structure of M-hat
  const R D = n16 + n17 + n18;
  const R S = n4 - R(2) * D;            // (f1+f2) + (f3+f4) + (f5+f6)
  const R A = (n5 - n16 - n17 + R(2) * n18 + S) * third;  // f1 + f2
  const R P6 = n6 - n16 + n17;          // (f3+f4) - (f5+f6)
  const R B = R(0.5) * (S - A + P6);      // f3 + f4
  const R C = R(0.5) * (S - A - P6);      // f5 + f6
  const R dx = n1 - n11 - n13, dy = n2 - n10 - n15, dz = n3 - n12 - n14;
  fs[0] = n0 - n4 + D;
  fs[1] = R(0.5) * (A + dx);
  fs[2] = R(0.5) * (A - dx);
  fs[3] = R(0.5) * (B + dy);
  fs[4] = R(0.5) * (B - dy);
  fs[5] = R(0.5) * (C + dz);
  fs[6] = R(0.5) * (C - dz);
  fs[7] = R(0.25) * (n16 + n7 + n10 + n11);
  fs[8] = R(0.25) * (n16 + n7 - n10 - n11);
  fs[9] = R(0.25) * (n16 - n7 - n10 + n11);
  fs[10] = R(0.25) * (n16 - n7 + n10 - n11);
  fs[11] = R(0.25) * (n17 + n8 + n12 + n13);
  fs[12] = R(0.25) * (n17 + n8 - n12 - n13);
  fs[13] = R(0.25) * (n17 - n8 - n12 + n13);
  fs[14] = R(0.25) * (n17 - n8 + n12 - n13);
  fs[15] = R(0.25) * (n18 + n9 + n14 + n15);
  fs[16] = R(0.25) * (n18 + n9 - n14 - n15);
  fs[17] = R(0.25) * (n18 - n9 - n14 + n15);
  fs[18] = R(0.25) * (n18 - n9 + n14 - n15);
}

template <typename R>
LBM_HD void feq19(R rho, R ux, R uy, R uz, R* fe) {
  const R uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const R cu = c19x(i) * ux + c19y(i) * uy + c19z(i) * uz;
    fe[i] = w19(i) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
  }
}

// The same collision when s_q = s_pi = 1 and m^eq = M-hat f^eq (the default
// reading): every moment of rate 1, the conserved ones included, leaves the
// collision as m^eq(rho, u + F/rho), so f* = f^eq(rho, u + F/rho) plus the
// relaxed non-equilibrium parts (1 - s_k)(m_k - m^eq_k(u)) of the six second-
// order moments, mapped back through their columns of M-hat^-1: the rest and
// axis populations for e and the normal stresses, one diagonal pair per
// shear component.  An exact identity, cheaper than the general transform.
template <typename R>
LBM_HD void collide19_fast(const Params& P, const R* f, R rho, R ux, R uy, R uz, R Fx, R Fy, R Fz, R* fs) {
  const R s7_10 = f[7] + f[8] + f[9] + f[10];
  const R s11_14 = f[11] + f[12] + f[13] + f[14];
  const R s15_18 = f[15] + f[16] + f[17] + f[18];
  const R Sxx = (f[1] + f[2]) + s7_10 + s11_14;
  const R Syy = (f[3] + f[4]) + s7_10 + s15_18;
  const R Szz = (f[5] + f[6]) + s11_14 + s15_18;
  const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
  const R ce = R(1) - R(P.s_e), cv = R(1) - R(P.s_v);
  // relaxed non-equilibrium moments (1 - s_k)(m_k - rho e_k(u))
  const R A4 = ce * (Sxx + Syy + Szz - rho * (R(1) + uxx + uyy + uzz));
  const R A5 = cv * (R(2) * Sxx - Syy - Szz - rho * (R(2) * uxx - uyy - uzz));
  const R A6 = cv * (Syy - Szz - rho * (uyy - uzz));
  const R A7 = cv * ((f[7] + f[8]) - (f[9] + f[10]) - rho * ux * uy);
  const R A8 = cv * ((f[11] + f[12]) - (f[13] + f[14]) - rho * ux * uz);
  const R A9 = cv * ((f[15] + f[16]) - (f[17] + f[18]) - rho * uy * uz);
  // f^eq(rho, u') with u' = u + F/rho, pair by pair: w rho (1 + 4.5 cu^2 - 1.5 u'^2) +- 3 w rho cu
  const R ir = rcp(rho);
  const R vx = ux + Fx * ir, vy = uy + Fy * ir, vz = uz + Fz * ir;
  const R base = rho * (R(1) - R(1.5) * (vx * vx + vy * vy + vz * vz));
  const R r45 = R(4.5) * rho, r3 = R(3) * rho;
  const R w0 = R(1) / R(3), w1 = R(1) / R(18), w2 = R(1) / R(36);
  fs[0] = w0 * base - A4;
  {
    const R e = w1 * (base + r45 * vx * vx) + (A4 + A5) * (R(1) / R(6)), o = w1 * r3 * vx;
    fs[1] = e + o;
    fs[2] = e - o;
  }
  {
    const R e = w1 * (base + r45 * vy * vy) + A4 * (R(1) / R(6)) - A5 * (R(1) / R(12)) + A6 * R(0.25),
            o = w1 * r3 * vy;
    fs[3] = e + o;
    fs[4] = e - o;
  }
  {
    const R e = w1 * (base + r45 * vz * vz) + A4 * (R(1) / R(6)) - A5 * (R(1) / R(12)) - A6 * R(0.25),
            o = w1 * r3 * vz;
    fs[5] = e + o;
    fs[6] = e - o;
  }
  // diagonal pairs (c, -c): c = (1,1,0), (1,-1,0), (1,0,1), (1,0,-1), (0,1,1), (0,1,-1)
  const R p7 = vx + vy, p9 = vx - vy, p11 = vx + vz, p13 = vx - vz, p15 = vy + vz, p17 = vy - vz;
  {
    const R e = w2 * (base + r45 * p7 * p7) + A7 * R(0.25), o = w2 * r3 * p7;
    fs[7] = e + o;
    fs[8] = e - o;
  }
  {
    const R e = w2 * (base + r45 * p9 * p9) - A7 * R(0.25), o = w2 * r3 * p9;
    fs[9] = e + o;
    fs[10] = e - o;
  }
  {
    const R e = w2 * (base + r45 * p11 * p11) + A8 * R(0.25), o = w2 * r3 * p11;
    fs[11] = e + o;
    fs[12] = e - o;
  }
  {
    const R e = w2 * (base + r45 * p13 * p13) - A8 * R(0.25), o = w2 * r3 * p13;
    fs[13] = e + o;
    fs[14] = e - o;
  }
  {
    const R e = w2 * (base + r45 * p15 * p15) + A9 * R(0.25), o = w2 * r3 * p15;
    fs[15] = e + o;
    fs[16] = e - o;
  }
  {
    const R e = w2 * (base + r45 * p17 * p17) - A9 * R(0.25), o = w2 * r3 * p17;
    fs[17] = e + o;
    fs[18] = e - o;
  }
}

// ------------------------------------------------------------ D3Q7 MRT ------
template <typename R>
LBM_HD R lambda_of(const Params& P, R rho) {
  if (P.lam_uniform) return P.lambda_v;
  R phi = (rho - P.rho_v) * P.inv_drho;
  phi = fmin(fmax(phi, R(0)), R(1));
  return P.lambda_v + (P.lambda_l - P.lambda_v) * phi;
}

// Eq. 13 collision with the source of Eq. 15: g* = g - M^-1 Lambda M (g - w T) - w Fbar
// (+ vartheta w rho c_v d2T / 2, the S_i of Eq. 16 with dt = 1; d2T = d^2T/dt^2),
// Lambda = diag(1, vs, vs, vs, 1, 1, 1), vs from lambda, grad T = -vs m_alpha / c_s^2.
// VT: vartheta known at compile time (0 or 1), or -1 to read it from P.
template <typename R, int VT = -1>
LBM_HD void collide7(const Params& P, const R* g, R rho, R T, R ux, R uy, R uz, R divu,
                     R dpdT, R d2T, R* gs) {
  const R m1 = g[1] - g[2], m2 = g[3] - g[4], m3 = g[5] - g[6];
  const R vs = rcp(lambda_of(P, rho) * P.inv_cs2t + R(0.5));
  const R k = -vs * P.inv_cs2t;
  const R ugT = k * (ux * m1 + uy * m2 + uz * m3);
  const R Fbar = rho * P.cv * ugT + T * dpdT * divu;
  R h = T - Fbar;
  if (VT < 0 ? P.vartheta != 0 : VT != 0) h += R(0.5) * rho * P.cv * d2T;
  const R w0 = R(1) - P.wbar, w1 = P.wbar * (R(1) / R(6));
  const R r = R(0.5) * (R(1) - vs);
  gs[0] = w0 * h;
  gs[1] = w1 * h + r * m1;
  gs[2] = w1 * h - r * m1;
  gs[3] = w1 * h + r * m2;
  gs[4] = w1 * h - r * m2;
  gs[5] = w1 * h + r * m3;
  gs[6] = w1 * h - r * m3;
}

// ------------------------------------------------------ open-face boundary --
// Constant-pressure boundary of Sec. 3.3 on face `face` (outward normal n):
// u_n = [sum_{c.n=0} f + 2 sum_{c.n=1} f + F.n/2]/rho_b - 1; f_{-n} = f_n - rho_b u_n / 3;
// diagonal unknowns c = -n + sig e_a: f = f_opp - rho_b u_n/6 - sig/2 (sum_{c.n=0} c_a f + F_a/2) + F.n/8.
template <typename R>
LBM_HD void zouhe(int face, R rho_b, R Fx, R Fy, R Fz, R* f) {
  const int ax = face >> 1;
  const int sg = (face & 1) ? 1 : -1;
  R SZ = R(0), SP = R(0), tx = R(0), ty = R(0), tz = R(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int cn = sg * (ax == 0 ? c19x(i) : (ax == 1 ? c19y(i) : c19z(i)));
    if (cn == 0) {
      SZ += f[i];
      tx += c19x(i) * f[i];
      ty += c19y(i) * f[i];
      tz += c19z(i) * f[i];
    } else if (cn > 0) {
      SP += f[i];
    }
  }
  const R Fn = sg * (ax == 0 ? Fx : (ax == 1 ? Fy : Fz));
  const R un = (SZ + R(2) * SP + R(0.5) * Fn) * rcp(rho_b) - R(1);
  const R base6 = -rho_b * un * (R(1) / R(6)) + R(0.125) * Fn;
  const R hx = R(0.5) * (tx + R(0.5) * Fx), hy = R(0.5) * (ty + R(0.5) * Fy), hz = R(0.5) * (tz + R(0.5) * Fz);
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
    const int cn = sg * (ax == 0 ? cx : (ax == 1 ? cy : cz));
    if (cn != -1) continue;
    const int tx_ = ax == 0 ? 0 : cx, ty_ = ax == 1 ? 0 : cy, tz_ = ax == 2 ? 0 : cz;
    if (tx_ == 0 && ty_ == 0 && tz_ == 0) {
      f[i] = f[opp19(i)] - rho_b * un * (R(1) / R(3));
    } else {
      const R t = tx_ * hx + ty_ * hy + tz_ * hz;  // sig/2 (S_a + F_a/2)
      f[i] = f[opp19(i)] + base6 - t;
    }
  }
}

}  // namespace lbm
