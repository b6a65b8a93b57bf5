// Per-cell vector-Jacobian products of the step (the transposed derivatives of
// lbm_cell.cuh), for the discrete adjoint.  Each function takes the forward
// inputs of one cell and the adjoint (cotangent) of the forward outputs and
// returns the adjoints of the inputs; templated on the real type so that the
// same code is checked against double-precision differences on the host.
#pragma once

#include "lbm_cell.cuh"

namespace lbm {

// -------------------------------------------------- D3Q19 collision (Eq. 8) --
// Normalised equilibrium moments e_k(u) = m^eq_k(rho, u) / rho and their
// u-gradients, contracted with weights v[19]: returns sum v_k e_k(u) and
// adds sum v_k d e_k / d u to g[3].
template <typename R>
LBM_HD R meq_contract(const Params& P, const R* v, R ux, R uy, R uz, R* g) {
  const R t = R(1) / R(3), s6 = R(1) / R(6), n9 = R(1) / R(9);
  const R xx = ux * ux, yy = uy * uy, zz = uz * uz;
  R e = v[0] + v[1] * ux + v[2] * uy + v[3] * uz + v[4] * (R(1) + xx + yy + zz) + v[5] * (R(2) * xx - yy - zz) +
        v[6] * (yy - zz) + v[7] * ux * uy + v[8] * ux * uz + v[9] * uy * uz +
        t * (v[10] * uy + v[11] * ux + v[12] * uz + v[13] * ux + v[14] * uz + v[15] * uy);
  R gx = v[1] + R(2) * ux * v[4] + R(4) * ux * v[5] + uy * v[7] + uz * v[8] + t * (v[11] + v[13]);
  R gy = v[2] + R(2) * uy * v[4] - R(2) * uy * v[5] + R(2) * uy * v[6] + ux * v[7] + uz * v[9] + t * (v[10] + v[15]);
  R gz = v[3] + R(2) * uz * v[4] - R(2) * uz * v[5] - R(2) * uz * v[6] + ux * v[8] + uy * v[9] + t * (v[12] + v[14]);
  if (P.meq_printed) {  // rows 16-18 as printed: 1/9 - |u|^2/6 + (u_a^2 + u_b^2)/3
    const R uu = xx + yy + zz;
    e += v[16] * (n9 - s6 * uu + t * (xx + yy)) + v[17] * (n9 - s6 * uu + t * (xx + zz)) +
         v[18] * (n9 - s6 * uu + t * (yy + zz));
    gx += t * ux * (v[16] + v[17] - v[18]);
    gy += t * uy * (v[16] - v[17] + v[18]);
    gz += t * uz * (-v[16] + v[17] + v[18]);
  } else {  // M-hat f^eq: 1/9 - u_c^2/6 + (u_a^2 + u_b^2)/3, c the excluded axis
    e += v[16] * (n9 - s6 * zz + t * (xx + yy)) + v[17] * (n9 - s6 * yy + t * (xx + zz)) +
         v[18] * (n9 - s6 * xx + t * (yy + zz));
    gx += R(2) * t * ux * (v[16] + v[17]) - t * ux * v[18];
    gy += R(2) * t * uy * (v[16] + v[18]) - t * uy * v[17];
    gz += R(2) * t * uz * (v[17] + v[18]) - t * uz * v[16];
  }
  g[0] += gx;
  g[1] += gy;
  g[2] += gz;
  return e;
}

// Transpose of the hand-solved f* = M-hat^-1 n of collide19: nb = M-hat^-T b.
template <typename R>
LBM_HD void minv19_T(const R* b, R* nb) {
#pragma unroll
  for (int k = 0; k < 19; ++k) nb[k] = R(0);
  const R q = R(1) / R(4);
  nb[0] = b[0];
  nb[4] = -b[0];
  R Db = b[0];
  R Ab = R(0.5) * (b[1] + b[2]), dxb = R(0.5) * (b[1] - b[2]);
  const R Bb = R(0.5) * (b[3] + b[4]), dyb = R(0.5) * (b[3] - b[4]);
  const R Cb = R(0.5) * (b[5] + b[6]), dzb = R(0.5) * (b[5] - b[6]);
  nb[16] += q * (b[7] + b[8] + b[9] + b[10]);
  nb[7] = q * (b[7] + b[8] - b[9] - b[10]);
  nb[10] += q * (b[7] - b[8] - b[9] + b[10]);
  nb[11] += q * (b[7] - b[8] + b[9] - b[10]);
  nb[17] += q * (b[11] + b[12] + b[13] + b[14]);
  nb[8] = q * (b[11] + b[12] - b[13] - b[14]);
  nb[12] += q * (b[11] - b[12] - b[13] + b[14]);
  nb[13] += q * (b[11] - b[12] + b[13] - b[14]);
  nb[18] += q * (b[15] + b[16] + b[17] + b[18]);
  nb[9] = q * (b[15] + b[16] - b[17] - b[18]);
  nb[14] += q * (b[15] - b[16] - b[17] + b[18]);
  nb[15] += q * (b[15] - b[16] + b[17] - b[18]);
  // dx = n1 - n11 - n13, dy = n2 - n10 - n15, dz = n3 - n12 - n14
  nb[1] = dxb;
  nb[11] -= dxb;
  nb[13] -= dxb;
  nb[2] = dyb;
  nb[10] -= dyb;
  nb[15] -= dyb;
  nb[3] = dzb;
  nb[12] -= dzb;
  nb[14] -= dzb;
  // B = (S - A + P6)/2, C = (S - A - P6)/2
  R Sb = R(0.5) * (Bb + Cb);
  Ab -= R(0.5) * (Bb + Cb);
  const R P6b = R(0.5) * (Bb - Cb);
  // P6 = n6 - n16 + n17
  nb[6] = P6b;
  nb[16] -= P6b;
  nb[17] += P6b;
  // A = (n5 - n16 - n17 + 2 n18 + S)/3
  const R a3 = Ab / R(3);
  nb[5] = a3;
  nb[16] -= a3;
  nb[17] -= a3;
  nb[18] += R(2) * a3;
  Sb += a3;
  // S = n4 - 2D, D = n16 + n17 + n18
  nb[4] += Sb;
  Db -= R(2) * Sb;
  nb[16] += Db;
  nb[17] += Db;
  nb[18] += Db;
}

// M-hat^T nb for rows 4..18 added to fb (rows = raw moments of c_i).
template <typename R>
LBM_HD void mhat_T_add(const R* nb, R* fb) {
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const R x = R(c19x(i)), y = R(c19y(i)), z = R(c19z(i));
    const R xx = x * x, yy = y * y, zz = z * z;
    fb[i] += nb[4] * (xx + yy + zz) + nb[5] * (R(2) * xx - yy - zz) + nb[6] * (yy - zz) + nb[7] * x * y +
             nb[8] * x * z + nb[9] * y * z + nb[10] * xx * y + nb[11] * x * yy + nb[12] * xx * z + nb[13] * x * zz +
             nb[14] * yy * z + nb[15] * y * zz + nb[16] * xx * yy + nb[17] * xx * zz + nb[18] * yy * zz;
  }
}

// Adjoint of f* = collide19(f, rho = sum f, u^eq, F): fsb = d L / d f*.
// u^eq = j / rho when ueq_from_f, else 0 (wall nodes).  Sets fb = d L / d f
// (through m = M-hat f, rho and u^eq) and Fb = d L / d F.
template <typename R>
LBM_HD void collide19_vjp(const Params& P, const R* f, bool ueq_from_f, const R* F, const R* fsb, R* fb, R* Fb) {
  R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    rho += f[i];
    jx += R(c19x(i)) * f[i];
    jy += R(c19y(i)) * f[i];
    jz += R(c19z(i)) * f[i];
  }
  const R ir = rcp(rho);
  const R ux = ueq_from_f ? jx * ir : R(0), uy = ueq_from_f ? jy * ir : R(0), uz = ueq_from_f ? jz * ir : R(0);
  const R vx = ux + F[0] * ir, vy = uy + F[1] * ir, vz = uz + F[2] * ir;  // u' = u + F/rho
  R nb[19];
  minv19_T(fsb, nb);
  R s[19];
  s[0] = s[1] = s[2] = s[3] = R(1);
  s[4] = R(P.s_e);
#pragma unroll
  for (int k = 5; k <= 9; ++k) s[k] = R(P.s_v);
#pragma unroll
  for (int k = 10; k <= 15; ++k) s[k] = R(P.s_q);
#pragma unroll
  for (int k = 16; k <= 18; ++k) s[k] = R(P.s_pi);
  // n_k = (1 - s_k) m_k + (s_k - 1) rho e_k(u) + rho e_k(u')
  R v0[19], mb[19];
#pragma unroll
  for (int k = 0; k < 19; ++k) {
    v0[k] = (s[k] - R(1)) * nb[k];
    mb[k] = (R(1) - s[k]) * nb[k];
  }
  R g0[3] = {R(0), R(0), R(0)}, g1[3] = {R(0), R(0), R(0)};
  const R e0 = meq_contract(P, v0, ux, uy, uz, g0);
  const R e1 = meq_contract(P, nb, vx, vy, vz, g1);
  // F enters through u' = u + F/rho
  Fb[0] = g1[0];
  Fb[1] = g1[1];
  Fb[2] = g1[2];
  R rhob = e0 + e1 - (g1[0] * F[0] + g1[1] * F[1] + g1[2] * F[2]) * ir;
  const R ubx = rho * (g0[0] + g1[0]), uby = rho * (g0[1] + g1[1]), ubz = rho * (g0[2] + g1[2]);
  R jbx = R(0), jby = R(0), jbz = R(0);
  if (ueq_from_f) {  // u = j / rho
    jbx = ubx * ir;
    jby = uby * ir;
    jbz = ubz * ir;
    rhob -= (ubx * ux + uby * uy + ubz * uz) * ir;
  }
#pragma unroll
  for (int i = 0; i < 19; ++i) fb[i] = rhob + R(c19x(i)) * jbx + R(c19y(i)) * jby + R(c19z(i)) * jbz;
  mhat_T_add(mb, fb);
}

// The same product for the closed form of the rate-1 case (collide19_fast):
// f* = f^eq(rho, u') + sum_k A_k col_k, u' = u + F/rho, A_k = (1 - s_k)(m_k - rho e_k(u))
// for the six second-order moments k = 4..9 and their M-hat^-1 columns col_k.
// acc += m k for an integer k known at compile time (a velocity component or a
// product of them): skipped when k = 0, since m * 0 is not folded away.
template <typename R>
LBM_HD void add_k(R& acc, R m, int k) {
  if (k) acc += m * R(k);
}

template <typename R>
LBM_HD void collide19_fast_vjp(const Params& P, const R* f, bool ueq_from_f, const R* F, const R* b, R* fb,
                               R* Fb) {
  R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    rho += f[i];
    add_k(jx, f[i], c19x(i));
    add_k(jy, f[i], c19y(i));
    add_k(jz, f[i], c19z(i));
  }
  const R ir = rcp(rho);
  const R ux = ueq_from_f ? jx * ir : R(0), uy = ueq_from_f ? jy * ir : R(0), uz = ueq_from_f ? jz * ir : R(0);
  const R vx = ux + F[0] * ir, vy = uy + F[1] * ir, vz = uz + F[2] * ir;
  const R vv = vx * vx + vy * vy + vz * vz;
  // f^eq(rho, u'): d/d rho = f^eq / rho; d/d u' = w rho (3 c + 9 (c.u') c - 3 u')
  R rhob = R(0), swb = R(0), s1x = R(0), s1y = R(0), s1z = R(0), s2x = R(0), s2y = R(0), s2z = R(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
    R cu = R(0);
    add_k(cu, vx, cx);
    add_k(cu, vy, cy);
    add_k(cu, vz, cz);
    const R wi = i == 0 ? R(1) / R(3) : (i < 7 ? R(1) / R(18) : R(1) / R(36));  // as in collide19_fast
    const R wb = wi * b[i];
    rhob += wb * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * vv);
    swb += wb;
    add_k(s1x, wb, cx);
    add_k(s1y, wb, cy);
    add_k(s1z, wb, cz);
    add_k(s2x, wb * cu, cx);
    add_k(s2y, wb * cu, cy);
    add_k(s2z, wb * cu, cz);
  }
  const R vbx = rho * (R(3) * s1x + R(9) * s2x - R(3) * vx * swb);
  const R vby = rho * (R(3) * s1y + R(9) * s2y - R(3) * vy * swb);
  const R vbz = rho * (R(3) * s1z + R(9) * s2z - R(3) * vz * swb);
  // u' = u + F/rho
  Fb[0] = vbx * ir;
  Fb[1] = vby * ir;
  Fb[2] = vbz * ir;
  rhob -= (vbx * F[0] + vby * F[1] + vbz * F[2]) * ir * ir;
  R ubx = vbx, uby = vby, ubz = vbz;
  // the columns of the relaxed moments (transposed): dL/dA_k
  const R s6 = R(1) / R(6), s12 = R(1) / R(12), q = R(0.25);
  const R A4b = -b[0] + s6 * (b[1] + b[2] + b[3] + b[4] + b[5] + b[6]);
  const R A5b = s6 * (b[1] + b[2]) - s12 * (b[3] + b[4] + b[5] + b[6]);
  const R A6b = q * (b[3] + b[4] - b[5] - b[6]);
  const R A7b = q * (b[7] + b[8] - b[9] - b[10]);
  const R A8b = q * (b[11] + b[12] - b[13] - b[14]);
  const R A9b = q * (b[15] + b[16] - b[17] - b[18]);
  const R ce = R(1) - R(P.s_e), cv = R(1) - R(P.s_v);
  const R m4 = ce * A4b, m5 = cv * A5b, m6 = cv * A6b, m7 = cv * A7b, m8 = cv * A8b, m9 = cv * A9b;
  // A_k = c_k (m_k - rho e_k(u)): e4 = 1 + |u|^2, e5 = 2ux^2 - uy^2 - uz^2, e6 = uy^2 - uz^2,
  // e7 = ux uy, e8 = ux uz, e9 = uy uz
  const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
  rhob -= m4 * (R(1) + uxx + uyy + uzz) + m5 * (R(2) * uxx - uyy - uzz) + m6 * (uyy - uzz) + m7 * ux * uy +
          m8 * ux * uz + m9 * uy * uz;
  ubx -= rho * (R(2) * ux * m4 + R(4) * ux * m5 + uy * m7 + uz * m8);
  uby -= rho * (R(2) * uy * m4 - R(2) * uy * m5 + R(2) * uy * m6 + ux * m7 + uz * m9);
  ubz -= rho * (R(2) * uz * m4 - R(2) * uz * m5 - R(2) * uz * m6 + ux * m8 + uy * m9);
  R jbx = R(0), jby = R(0), jbz = R(0);
  if (ueq_from_f) {  // u = j / rho
    jbx = ubx * ir;
    jby = uby * ir;
    jbz = ubz * ir;
    rhob -= (ubx * ux + uby * uy + ubz * uz) * ir;
  }
  // m_k = rows 4..9 of M-hat applied to f
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int x = c19x(i), y = c19y(i), z = c19z(i);
    R v = rhob;
    add_k(v, jbx, x);
    add_k(v, jby, y);
    add_k(v, jbz, z);
    add_k(v, m4, x * x + y * y + z * z);
    add_k(v, m5, 2 * x * x - y * y - z * z);
    add_k(v, m6, y * y - z * z);
    add_k(v, m7, x * y);
    add_k(v, m8, x * z);
    add_k(v, m9, y * z);
    fb[i] = v;
  }
}

// ------------------------------------------ D3Q7 collision + source (Eq. 13) --
// Adjoint of g* = collide7(g, rho, T, u, div u, dp/dT) with gsb = d L / d g*.
// T is an input of its own here (the caller adds Tb to every d L / d g_i).
template <typename R>
LBM_HD void collide7_vjp(const Params& P, const R* g, R rho, R T, const R* u, R divu, R dpdT, const R* gsb, R* gb,
                         R& rhob, R& Tb, R* ub, R& divub, R& dpdTb) {
  const R m1 = g[1] - g[2], m2 = g[3] - g[4], m3 = g[5] - g[6];
  const R lam = lambda_of(P, rho);
  const R vs = rcp(lam * R(P.inv_cs2t) + R(0.5));
  const R k = -vs * R(P.inv_cs2t);
  const R um = u[0] * m1 + u[1] * m2 + u[2] * m3;
  const R ugT = k * um;
  const R w0 = R(1) - R(P.wbar), w1 = R(P.wbar) / R(6);
  const R r = R(0.5) * (R(1) - vs);
  // gs0 = w0 h, gs_{2a-1,2a} = w1 h +- r m_a, h = T - Fbar
  const R hb = w0 * gsb[0] + w1 * (gsb[1] + gsb[2] + gsb[3] + gsb[4] + gsb[5] + gsb[6]);
  const R d1 = gsb[1] - gsb[2], d2 = gsb[3] - gsb[4], d3 = gsb[5] - gsb[6];
  const R rb = m1 * d1 + m2 * d2 + m3 * d3;
  R mb1 = r * d1, mb2 = r * d2, mb3 = r * d3;
  Tb = hb;
  const R Fbb = -hb;
  // Fbar = rho cv ugT + T dpdT divu
  rhob = R(P.cv) * ugT * Fbb;
  const R ugTb = rho * R(P.cv) * Fbb;
  Tb += dpdT * divu * Fbb;
  dpdTb = T * divu * Fbb;
  divub = T * dpdT * Fbb;
  // ugT = k (u . m)
  const R kb = um * ugTb;
  ub[0] = k * m1 * ugTb;
  ub[1] = k * m2 * ugTb;
  ub[2] = k * m3 * ugTb;
  mb1 += k * u[0] * ugTb;
  mb2 += k * u[1] * ugTb;
  mb3 += k * u[2] * ugTb;
  // k = -vs / c_s^2, r = (1 - vs)/2, vs = 1 / (lambda / c_s^2 + 1/2)
  const R vsb = -R(P.inv_cs2t) * kb - R(0.5) * rb;
  const R lamb = -vs * vs * R(P.inv_cs2t) * vsb;
  if (!P.lam_uniform) {
    const R phi = (rho - R(P.rho_v)) * R(P.inv_drho);
    if (phi > R(0) && phi < R(1)) rhob += lamb * (R(P.lambda_l) - R(P.lambda_v)) * R(P.inv_drho);
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) gb[i] = R(0);
  gb[1] = mb1;
  gb[2] = -mb1;
  gb[3] = mb2;
  gb[4] = -mb2;
  gb[5] = mb3;
  gb[6] = -mb3;
}

// ------------------------------------------------ open faces (Sec. 3.3) -----
// Adjoint of zouhe(face, rho_b, F, f): on entry fb holds d L / d f after the
// rule (unknowns included); on exit the unknowns' adjoints are folded into the
// known populations and Fb (added), and the unknown entries are zero.
template <typename R>
LBM_HD void zouhe_vjp(int face, R rho_b, R* fb, R* Fb) {
  const int ax = face >> 1;
  const int sg = (face & 1) ? 1 : -1;
  R unb = R(0), Fnb = R(0), Sb[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
    const int cn = sg * (ax == 0 ? cx : (ax == 1 ? cy : cz));
    if (cn != -1) continue;
    const R b = fb[i];
    fb[i] = R(0);
    fb[opp19(i)] += b;
    const int t[3] = {ax == 0 ? 0 : cx, ax == 1 ? 0 : cy, ax == 2 ? 0 : cz};
    if (t[0] == 0 && t[1] == 0 && t[2] == 0) {
      unb -= rho_b * b / R(3);
    } else {
      unb -= rho_b * b / R(6);
      Fnb += b / R(8);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (t[a]) {  // - (sig/2) (S_a + F_a / 2)
          Sb[a] -= R(0.5) * R(t[a]) * b;
          Fb[a] -= R(0.25) * R(t[a]) * b;
        }
    }
  }
  // u_n = (sum_Z f + 2 sum_P f + F_n/2) / rho_b - 1; S_a = sum_Z c_a f
  const R ir = rcp(rho_b);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int c[3] = {c19x(i), c19y(i), c19z(i)};
    const int cn = sg * c[ax];
    if (cn == 0) fb[i] += unb * ir + R(c[0]) * Sb[0] + R(c[1]) * Sb[1] + R(c[2]) * Sb[2];
    else if (cn == 1) fb[i] += R(2) * unb * ir;
  }
  Fnb += R(0.5) * unb * ir;
  Fb[ax] += R(sg) * Fnb;
}

// ------------------------------------------------------- EOS and psi (Eq. 7, 37) --
// Partial derivatives of p_EOS: p_rho, p_T, p_rhoT, p_TT.
template <typename R>
LBM_HD void eos_derivs(const Params& P, R rho, R T, R& pr, R& pT, R& prT, R& pTT) {
  if (P.eos_kind == 1) {
    pr = R(P.eos_c0);
    pT = prT = pTT = R(0);
    return;
  }
  const R Tc = R(1) / R(P.inv_Tc), kap = R(P.kappa), a = R(P.a), b = R(P.b), Rg = R(P.R);
  const R sq = sqrt(T * Tc);
  const R s = R(1) + kap * (R(1) - sqrt(T * R(P.inv_Tc)));
  const R xi = s * s;
  const R isq = rcp(sq), ihT = rcp(R(2) * T);
  const R dxi = -kap * s * isq;
  const R d2xi = ihT * (kap * kap * R(P.inv_Tc) + kap * s * isq);
  const R om = R(1) - b * rho;
  const R den = R(1) + R(2) * b * rho - b * b * rho * rho;
  const R dden = R(2) * b - R(2) * b * b * rho;
  const R iom = rcp(om), iden = rcp(den);
  const R q = (R(2) * rho * den - rho * rho * dden) * iden * iden;  // d/drho (rho^2 / den)
  pr = Rg * T * iom * iom - a * xi * q;
  pT = rho * Rg * iom - a * dxi * rho * rho * iden;
  prT = Rg * iom * iom - a * dxi * q;
  pTT = -a * d2xi * rho * rho * iden;
}

// Adjoint of psi(rho, T) = sqrt(2 (p - rho/3) / G) and of dp/dT(rho, T):
// adds to rhob, Tb.
template <typename R>
LBM_HD void psi_dpdT_vjp(const Params& P, R rho, R T, R psi, R psib, R dpdTb, R& rhob, R& Tb) {
  R pr, pT, prT, pTT;
  eos_derivs(P, rho, T, pr, pT, prT, pTT);
  if (psi > R(0)) {
    const R c = psib * R(P.inv_G) * rcp(psi);  // psi_b / (G psi)
    rhob += c * (pr - R(1) / R(3));
    Tb += c * pT;
  }
  rhob += dpdTb * prT;
  Tb += dpdTb * pTT;
}

}  // namespace lbm
