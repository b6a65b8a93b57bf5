// The z-marching schedule: one time step in two stencil kernels (plus the face rules of
// phase D), each reading the populations once.
//
// A CTA owns a tile of 32 x 8 cells of the xy-plane and marches up through a range of
// z-planes.  Shared memory holds a ring of four planes of a scalar field on the tile and a
// one-cell halo around it (34 x 10 positions), filled one plane ahead of the plane being
// updated; ghost positions beyond a face take the per-axis rules of the step (periodic
// wrap, copy of the boundary node at an open face, mirror through the wall layer at a wall
// with contact angle 90 degrees), so the stencil sums read the ring without any face logic.
//
//   k_march19  phases A, B and the D3Q19 part of C: the populations f and g of plane z+1
//              (tile and halo) give rho, T and psi (Eqs. 3, 7, 37) into the psi ring;
//              plane z then takes the force of Eq. 6 from the ring, the real velocity of
//              Eq. 5, the MRT collision with the exact-difference forcing (Eq. 8) and the
//              push with bounce-back at walls.  It stores rho and u (and F at open-face
//              nodes) for the D3Q7 kernel and the face rules.
//   k_march7   the D3Q7 part of C: u and rho of plane z+1 (tile and halo) into rings;
//              plane z takes div u by the isotropic difference (18 neighbours, from the
//              ring), grad T from its own moments, the collision with the source of Eq. 15
//              and the relaxed streaming of Eq. 13, pushed to the six neighbours with
//              rho c_v of the destination.
//
// Each CTA's halo rows and columns belong to the neighbouring tiles, whose CTAs march at
// the same pace, so those reads are served mostly from L2.  A wall with a contact angle
// other than 90 degrees needs the wetting term of Eq. 36 at ghost positions two cells
// away; contexts with such walls use the other schedules.
#pragma once

#include "lbm_phases.cuh"

namespace lbm {

constexpr int kMarchTX = 32, kMarchTY = 8, kMarchThreads = kMarchTX * kMarchTY;
constexpr int kRingW = kMarchTX + 2, kRingH = kMarchTY + 2, kRingN = kRingW * kRingH;
constexpr int kMarchHalo = 2 * kRingW + 2 * kMarchTY;  // halo positions of the ring

// Source coordinate of ring coordinate v (at most one cell beyond the axis) under the psi
// rules: periodic wrap, open: the boundary node, wall: mirror through the wall layer.
LBM_DEV int march_map(int v, int n, int klo, int khi) {
  if (v < 0) return klo == FACE_PERIODIC ? v + n : (klo == FACE_OPEN ? 0 : -v);
  if (v >= n) return khi == FACE_PERIODIC ? v - n : (khi == FACE_OPEN ? n - 1 : 2 * (n - 1) - v);
  return v;
}

// 1 when v lies beyond a wall face of its axis
LBM_DEV bool march_beyond_wall(int v, int n, int klo, int khi) {
  return (v < 0 && klo == FACE_WALL) || (v >= n && khi == FACE_WALL);
}

// Halo position k (< kMarchHalo) of the ring, tile coordinates (-1 .. 32, -1 .. 8):
// the rows below and above the tile, then the columns left and right of it.
LBM_DEV void march_halo_pos(int k, int& hx, int& hy) {
  if (k < kRingW) {
    hx = k - 1;
    hy = -1;
  } else if (k < 2 * kRingW) {
    hx = k - kRingW - 1;
    hy = kMarchTY;
  } else if (k < 2 * kRingW + kMarchTY) {
    hx = -1;
    hy = k - 2 * kRingW;
  } else {
    hx = kMarchTX;
    hy = k - 2 * kRingW - kMarchTY;
  }
}

// Neighbour offsets of a coordinate along one axis: for a step s (0: -1, 1: +1) the
// cell-index offset (periodic faces wrap; 0 beyond a non-periodic face) and the kind of
// face crossed (0 inside or periodic).
struct MarchAxis {
  int off[2], kind[2];
};

LBM_DEV MarchAxis march_axis(int v, int n, int stride, int klo, int khi) {
  MarchAxis a;
  const bool per = klo == FACE_PERIODIC, lo = v == 0, hi = v == n - 1;
  a.off[0] = !lo ? -stride : (per ? (n - 1) * stride : 0);
  a.kind[0] = (!lo || per) ? 0 : klo;
  a.off[1] = !hi ? stride : (per ? -(n - 1) * stride : 0);
  a.kind[1] = (!hi || per) ? 0 : khi;
  return a;
}

// The populations of cell c decoded (the per-cell references of the state read, if the
// storage has them) and its macroscopic fields rho, j and T.
template <typename ST>
LBM_DEV void march_cell(const Params& P, unsigned c, const ST* __restrict__ fA, const ST* __restrict__ gA,
                        const AuxFor<ST>& X, const Hint& h, float* fl, float& rho, float& jx, float& jy,
                        float& jz, float& T) {
  const unsigned Nu = (unsigned)P.N;
  const float2 rin = ref_in_at<ST>(X, c);
  float gl[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) fl[i] = PopStore<ST>::ld(fA + (i * Nu + c), fbase_at<ST>(P, i, rin.x), h);
#pragma unroll
  for (int i = 0; i < 7; ++i) gl[i] = PopStore<ST>::ld(gA + (i * Nu + c), gbase_at<ST>(P, i, rin.y), h);
  sum19(fl, rho, jx, jy, jz);
  T = sum7(gl);
}

// psi of Eq. 7 at (rho, T); the error flags of a cell whose state is out of range
LBM_DEV float march_psi(const Params& P, float rho, float T, float jsum, int& err) {
  if (!isfinite(rho) || !isfinite(T) || !isfinite(jsum)) err |= ERRF_NONFINITE;
  float p, dpdT, psi;
  eos_pr(P, rho, T, p, dpdT);
  if (!psi_of(P, rho, p, psi)) err |= ERRF_PSI;
  return psi;
}

// ------------------------------------------------------------ k_march19 ----
template <typename ST>
__global__ void __launch_bounds__(kMarchThreads, 2)
    k_march19(Params P, const ST* __restrict__ fA, const ST* __restrict__ gA, ST* __restrict__ fB, AuxFor<ST> X,
              int* err_out, int zchunk) {
  constexpr bool LR = LocalRef<ST>::on;
  __shared__ float s_psi[4][kRingN];
  __shared__ float s_rho[LR ? 4 : 1][LR ? kRingN : 1];  // this step's rho, for the per-cell references
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int x0 = blockIdx.x * kMarchTX, y0 = blockIdx.y * kMarchTY;
  const int z0 = blockIdx.z * zchunk, z1 = min(nz, z0 + zchunk);
  if (z0 >= z1) return;  // the same for every thread of the CTA
  const unsigned Nu = (unsigned)P.N, plane = (unsigned)(nx * ny);
  const int xl = min(kMarchTX, nx - x0), yl = min(kMarchTY, ny - y0);  // valid own cells: tx < xl, ty < yl
  const int* fk = P.face_kind;
  const Hint h = make_hint();
  // ring positions this thread fills: its own and (tid < kMarchHalo) one halo position; only
  // those within one cell of a valid cell are needed
  const bool own = tx < xl && ty < yl;
  const bool own_pos = tx <= xl && ty <= yl;
  int hx = 0, hy = 0;
  bool halo = false;
  if (tid < kMarchHalo) {
    march_halo_pos(tid, hx, hy);
    halo = hx <= xl && hy <= yl;
  }
  const int ocol = march_map(x0 + tx, nx, fk[0], fk[1]) + nx * march_map(y0 + ty, ny, fk[2], fk[3]);
  const int hcol = halo ? march_map(x0 + hx, nx, fk[0], fk[1]) + nx * march_map(y0 + hy, ny, fk[2], fk[3]) : 0;
  const int orp = (ty + 1) * kRingW + tx + 1, hrp = (hy + 1) * kRingW + hx + 1;
  // push offsets along x and y (fixed through the march)
  const MarchAxis ax = march_axis(x0 + tx, nx, 1, fk[0], fk[1]);
  const MarchAxis ay = march_axis(y0 + ty, ny, nx, fk[2], fk[3]);
  int err = 0;

  float fc[19], rho_c = 1.f, jx_c = 0.f, jy_c = 0.f, jz_c = 0.f;
  // fills ring plane zl (psi; rho with per-cell references); keeps the own populations of a
  // real plane zl in fc (used as plane zc on the next pass)
  auto fill = [&](int zl, bool keep) {
    const int zs = march_map(zl, nz, fk[4], fk[5]);
    const unsigned pz = plane * (unsigned)zs;
    float* ring = s_psi[zl & 3];
    if (own_pos) {
      float fl[19], r, jx, jy, jz, T;
      const unsigned c = (unsigned)ocol + pz;
      march_cell<ST>(P, c, fA, gA, X, h, fl, r, jx, jy, jz, T);
      const bool real = own && zl >= z0 && zl < z1;  // counted once, by the plane's owner
      int e = 0;
      ring[orp] = march_psi(P, r, T, jx + jy + jz, e);
      if (real) err |= e;
      if constexpr (LR) {
        s_rho[zl & 3][orp] = r;
        if (real) X.ref_out[c] = make_float2(r, T);
      }
      if (keep) {
#pragma unroll
        for (int i = 0; i < 19; ++i) fc[i] = fl[i];
        rho_c = r;
        jx_c = jx;
        jy_c = jy;
        jz_c = jz;
      }
    }
    if (halo) {
      float fl[19], r, jx, jy, jz, T;
      march_cell<ST>(P, (unsigned)hcol + pz, fA, gA, X, h, fl, r, jx, jy, jz, T);
      int e = 0;
      ring[hrp] = march_psi(P, r, T, jx + jy + jz, e);
      if constexpr (LR) s_rho[zl & 3][hrp] = r;
    }
  };

  fill(z0 - 1, false);
  fill(z0, own);
  for (int zc = z0; zc < z1; ++zc) {
    // plane zc's populations move out of fc before the next plane's overwrite them
    float f0[19];
    const float r0 = rho_c, jx0 = jx_c, jy0 = jy_c, jz0 = jz_c;
#pragma unroll
    for (int i = 0; i < 19; ++i) f0[i] = fc[i];
    fill(zc + 1, own && zc + 1 < z1);
    __syncthreads();  // ring plane zc + 1 complete; planes zc - 1 and zc were completed before
    if (own) {
      const float* Rm = s_psi[(zc - 1) & 3];
      const float* R0 = s_psi[zc & 3];
      const float* Rp = s_psi[(zc + 1) & 3];
      // F = -G psi(x) sum_i varpi_i psi(x + c_i) c_i (Eq. 6), ghost psi in the ring
      float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
      for (int i = 1; i < 19; ++i) {
        const float* R = c19z(i) < 0 ? Rm : (c19z(i) > 0 ? Rp : R0);
        const float v = varpi19(i) * R[orp + c19x(i) + kRingW * c19y(i)];
        if (c19x(i)) sx += c19x(i) * v;  // zero components skipped (0 * v is not folded away)
        if (c19y(i)) sy += c19y(i) * v;
        if (c19z(i)) sz += c19z(i) * v;
      }
      const float kf = -P.G * R0[orp];
      const float Fx = kf * sx, Fy = kf * sy, Fz = kf * sz;
      const MarchAxis az = march_axis(zc, nz, (int)plane, fk[4], fk[5]);
      // faces of this node: bit f set when the node lies on non-periodic face f
      int faces = 0;
      if (fk[0] != FACE_PERIODIC) faces |= (x0 + tx == 0 ? 1 : 0) | (x0 + tx == nx - 1 ? 2 : 0);
      if (fk[2] != FACE_PERIODIC) faces |= (y0 + ty == 0 ? 4 : 0) | (y0 + ty == ny - 1 ? 8 : 0);
      if (fk[4] != FACE_PERIODIC) faces |= (zc == 0 ? 16 : 0) | (zc == nz - 1 ? 32 : 0);
      const bool wall = faces && on_wall(P, faces);
      const unsigned c = (unsigned)(x0 + tx) + (unsigned)nx * (unsigned)(y0 + ty) + plane * (unsigned)zc;
      const float ir = rcp(r0);
      float vx = 0.f, vy = 0.f, vz = 0.f;
      if (!wall) {
        vx = (jx0 + 0.5f * Fx) * ir;
        vy = (jy0 + 0.5f * Fy) * ir;
        vz = (jz0 + 0.5f * Fz) * ir;
      }
      st_aux(X.rho + c, r0, h);
      st_aux(X.ux + c, vx, h);
      st_aux(X.uy + c, vy, h);
      st_aux(X.uz + c, vz, h);
      if (faces && on_open(P, faces)) {  // the open-face rule of phase D reads F there
        X.Fx[c] = Fx;
        X.Fy[c] = Fy;
        X.Fz[c] = Fz;
      }
      float ux = jx0 * ir, uy = jy0 * ir, uz = jz0 * ir;
      if (wall && P.wall_ueq_zero) ux = uy = uz = 0.f;
      float fs[19];
      if (P.fast19)
        collide19_fast(P, f0, r0, ux, uy, uz, Fx, Fy, Fz, fs);
      else
        collide19(P, f0, r0, ux, uy, uz, Fx, Fy, Fz, fs);
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
        const int k = (cx ? ax.kind[cx > 0] : 0) | (cy ? ay.kind[cy > 0] : 0) | (cz ? az.kind[cz > 0] : 0);
        if (k == 0) {
          const int off = (cx ? ax.off[cx > 0] : 0) + (cy ? ay.off[cy > 0] : 0) + (cz ? az.off[cz > 0] : 0);
          // per-cell references: the destination's rho of this step
          const float r = LR ? s_rho[LR ? ((zc + cz) & 3) : 0][LR ? orp + cx + kRingW * cy : 0] : 0.f;
          PopStore<ST>::st(fB + (i * Nu + (unsigned)((int)c + off)), fs[i], fbase_at<ST>(P, i, r));
        } else if (k & FACE_WALL) {  // modified bounce-back
          PopStore<ST>::st(fB + (opp19(i) * Nu + c), fs[i], fbase_at<ST>(P, opp19(i), r0));
        }
        // else: leaves through an open face
      }
    }
  }
  if (err) atomicOr(err_out, err);
}

// ------------------------------------------------------------- k_march7 ----
// VT: vartheta (0 or 1) at compile time.
template <typename ST, int VT>
__global__ void __launch_bounds__(kMarchThreads, 3)
    k_march7(Params P, const ST* __restrict__ gA, ST* __restrict__ gB, AuxFor<ST> X, int zchunk) {
  constexpr bool LR = LocalRef<ST>::on;
  __shared__ float s_u[4][3][kRingN];
  __shared__ float s_r[4][kRingN];
  __shared__ float s_g[2][4][kMarchThreads];  // populations 1..4 of the own cells of plane zc, by parity of zc
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int x0 = blockIdx.x * kMarchTX, y0 = blockIdx.y * kMarchTY;
  const int z0 = blockIdx.z * zchunk, z1 = min(nz, z0 + zchunk);
  if (z0 >= z1) return;
  const unsigned Nu = (unsigned)P.N, plane = (unsigned)(nx * ny);
  const int xl = min(kMarchTX, nx - x0), yl = min(kMarchTY, ny - y0);
  const int* fk = P.face_kind;
  const Hint h = make_hint();
  const bool own = tx < xl && ty < yl;
  const bool own_pos = tx <= xl && ty <= yl;
  int hx = 0, hy = 0;
  bool halo = false;
  if (tid < kMarchHalo) {
    march_halo_pos(tid, hx, hy);
    halo = hx <= xl && hy <= yl;
  }
  const int ox = x0 + tx, oy = y0 + ty;
  const int ocol = march_map(ox, nx, fk[0], fk[1]) + nx * march_map(oy, ny, fk[2], fk[3]);
  const bool owall = march_beyond_wall(ox, nx, fk[0], fk[1]) || march_beyond_wall(oy, ny, fk[2], fk[3]);
  const int hcol = halo ? march_map(x0 + hx, nx, fk[0], fk[1]) + nx * march_map(y0 + hy, ny, fk[2], fk[3]) : 0;
  const bool hwall = march_beyond_wall(x0 + hx, nx, fk[0], fk[1]) || march_beyond_wall(y0 + hy, ny, fk[2], fk[3]);
  const int orp = (ty + 1) * kRingW + tx + 1, hrp = (hy + 1) * kRingW + hx + 1;
  const MarchAxis ax = march_axis(ox, nx, 1, fk[0], fk[1]);
  const MarchAxis ay = march_axis(oy, ny, nx, fk[2], fk[3]);

  // ring plane zl: u (zero beyond a wall) and rho (any value beyond a non-periodic face:
  // nothing is pushed there)
  auto fill = [&](int zl) {
    const int zs = march_map(zl, nz, fk[4], fk[5]);
    const bool zwall = march_beyond_wall(zl, nz, fk[4], fk[5]);
    const unsigned pz = plane * (unsigned)zs;
    const int s = zl & 3;
    if (own_pos) {
      const unsigned c = (unsigned)ocol + pz;
      const bool w = owall || zwall;
      s_u[s][0][orp] = w ? 0.f : ld_aux(X.ux + c, h);
      s_u[s][1][orp] = w ? 0.f : ld_aux(X.uy + c, h);
      s_u[s][2][orp] = w ? 0.f : ld_aux(X.uz + c, h);
      s_r[s][orp] = ld_aux(X.rho + c, h);
    }
    if (halo) {
      const unsigned c = (unsigned)hcol + pz;
      const bool w = hwall || zwall;
      s_u[s][0][hrp] = w ? 0.f : ld_aux(X.ux + c, h);
      s_u[s][1][hrp] = w ? 0.f : ld_aux(X.uy + c, h);
      s_u[s][2][hrp] = w ? 0.f : ld_aux(X.uz + c, h);
      s_r[s][hrp] = ld_aux(X.rho + c, h);
    }
  };
  // the own cell's populations of plane zl (zl mapped into the domain), decoded
  auto load_g = [&](int zl, float* gl) {
    const unsigned c = (unsigned)ocol + plane * (unsigned)march_map(zl, nz, fk[4], fk[5]);
    const float tin = ref_in_at<ST>(X, c).y;
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = PopStore<ST>::ld(gA + (i * Nu + c), gbase_at<ST>(P, i, tin), h);
  };

  float gp[7], gc[7], gn[7];
  fill(z0 - 1);
  fill(z0);
  if (own) {
    load_g(z0 - 1, gp);
    load_g(z0, gc);
  }
  for (int zc = z0; zc < z1; ++zc) {
    fill(zc + 1);
    if (own) {
      load_g(zc + 1, gn);
#pragma unroll
      for (int i = 1; i < 5; ++i) s_g[zc & 1][i - 1][tid] = gc[i];
    }
    __syncthreads();
    if (own) {
      const int sm = (zc - 1) & 3, s0 = zc & 3, sp = (zc + 1) & 3;
      // div u = 3 sum_i w_i c_i . u(x + c_i), the ghost rules in the ring
      float du = 0.f;
#pragma unroll
      for (int i = 1; i < 19; ++i) {
        const int s = c19z(i) < 0 ? sm : (c19z(i) > 0 ? sp : s0);
        const int q = orp + c19x(i) + kRingW * c19y(i);
        float v = 0.f;
        if (c19x(i)) v += c19x(i) * s_u[s][0][q];
        if (c19y(i)) v += c19y(i) * s_u[s][1][q];
        if (c19z(i)) v += c19z(i) * s_u[s][2][q];
        du += w19(i) * v;
      }
      du *= 3.f;
      const unsigned c = (unsigned)ox + (unsigned)nx * (unsigned)oy + plane * (unsigned)zc;
      const float rho = s_r[s0][orp];
      const float T = sum7(gc);
      float d2T = 0.f, T1 = 0.f;
      if (VT) {
        T1 = X.T1[c];
        d2T = T - 2.f * T1 + X.T2[c];
      }
      float p, dpdT;
      eos_pr(P, rho, T, p, dpdT);
      float gs[7];
      collide7<float, VT>(P, gc, rho, T, s_u[s0][0][orp], s_u[s0][1][orp], s_u[s0][2][orp], du, dpdT, d2T, gs);
      // relaxed streaming: g_i(y) += (g*_i(x) - g_i(y)) / (rho(y) c_v), y = x + c_i
      const float t_out = LR ? ref_out_at<ST>(X, c).y : 0.f;
      PopStore<ST>::st(gB + c, gc[0] + (gs[0] - gc[0]) * rcp(rho * P.cv), gbase_at<ST>(P, 0, t_out));
      const MarchAxis az = march_axis(zc, nz, (int)plane, fk[4], fk[5]);
#pragma unroll
      for (int i = 1; i < 7; ++i) {
        const int cx = c7x(i), cy = c7y(i), cz = c7z(i);
        const MarchAxis& a = cx ? ax : (cy ? ay : az);
        const int sgn = (cx + cy + cz) > 0;
        if (a.kind[sgn]) continue;  // beyond a non-periodic face: the boundary rule sets it
        const unsigned d = (unsigned)((int)c + a.off[sgn]);
        float gold;
        if (cz > 0) {
          gold = gn[i];
        } else if (cz < 0) {
          gold = gp[i];
        } else {
          const int qx = tx + cx, qy = ty + cy;
          const bool inside = qx >= 0 && qx < xl && qy >= 0 && qy < yl && a.off[sgn] == (cx ? cx : cy * nx);
          if (inside)
            gold = s_g[zc & 1][i - 1][qy * kMarchTX + qx];
          else
            gold = PopStore<ST>::ld(gA + (i * Nu + d), gbase_at<ST>(P, i, ref_in_at<ST>(X, d).y), h);
        }
        const float ry = s_r[cz < 0 ? sm : (cz > 0 ? sp : s0)][orp + cx + kRingW * cy];
        const float ty_ = LR ? ref_out_at<ST>(X, d).y : 0.f;
        PopStore<ST>::st(gB + (i * Nu + d), gold + (gs[i] - gold) * rcp(ry * P.cv), gbase_at<ST>(P, i, ty_));
      }
      if (VT) {
        X.T2[c] = T1;
        X.T1[c] = T;
      }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      gp[i] = gc[i];
      gc[i] = gn[i];
    }
  }
}

}  // namespace lbm
