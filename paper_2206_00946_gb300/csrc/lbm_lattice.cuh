// Lattice indexing shared by all step kernels: node classes, streaming
// destinations, and the out-of-domain rules for psi and u (periodic wrap,
// wetting ghost layer of Eq. 36 at walls, zero-gradient copy at open faces).
#pragma once

#include "lbm_cell.cuh"

namespace lbm {

LBM_HD int dim_of(const Params& P, int a) { return a == 0 ? P.nx : (a == 1 ? P.ny : P.nz); }

LBM_HD int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// bit f set <=> (x,y,z) lies on non-periodic face f
LBM_HD int node_faces(const Params& P, int x, int y, int z) {
  int m = 0;
  if (P.face_kind[0] != FACE_PERIODIC) {
    m |= (x == 0) ? 1 : 0;
    m |= (x == P.nx - 1) ? 2 : 0;
  }
  if (P.face_kind[2] != FACE_PERIODIC) {
    m |= (y == 0) ? 4 : 0;
    m |= (y == P.ny - 1) ? 8 : 0;
  }
  if (P.face_kind[4] != FACE_PERIODIC) {
    m |= (z == 0) ? 16 : 0;
    m |= (z == P.nz - 1) ? 32 : 0;
  }
  return m;
}

// bit f set <=> (x,y,z) lies on face f and that face's node layer holds a Dirichlet
// temperature (every non-periodic face; a periodic face when held, Sec. 4.2)
LBM_HD int node_tfaces(const Params& P, int x, int y, int z) {
  int m = 0;
  if (P.tface[0]) m |= (x == 0) ? 1 : 0;
  if (P.tface[1]) m |= (x == P.nx - 1) ? 2 : 0;
  if (P.tface[2]) m |= (y == 0) ? 4 : 0;
  if (P.tface[3]) m |= (y == P.ny - 1) ? 8 : 0;
  if (P.tface[4]) m |= (z == 0) ? 16 : 0;
  if (P.tface[5]) m |= (z == P.nz - 1) ? 32 : 0;
  return m;
}

LBM_HD bool on_open(const Params& P, int m) {
  bool o = false;
#pragma unroll
  for (int f = 0; f < 6; ++f) o |= ((m >> f) & 1) && P.face_kind[f] == FACE_OPEN;
  return o;
}

LBM_HD bool on_wall(const Params& P, int m) {
  bool w = false;
#pragma unroll
  for (int f = 0; f < 6; ++f) w |= ((m >> f) & 1) && P.face_kind[f] == FACE_WALL;
  return w;
}

// Flat destination slot (i' * N + c') of population i leaving (x,y,z), or -1
// when it leaves through an open face.  Wall faces bounce it back into the
// opposite direction of the same node (modified bounce-back, Sec. 3.1).
LBM_HD int cell_of(const Params& P, int x, int y, int z) { return x + P.nx * (y + P.ny * z); }

LBM_HD long long dest19(const Params& P, int x, int y, int z, int i) {
  int q[3] = {x + c19x(i), y + c19y(i), z + c19z(i)};
  bool bounce = false, drop = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = dim_of(P, a);
    if (q[a] >= 0 && q[a] < n) continue;
    const int k = P.face_kind[2 * a + (q[a] >= n ? 1 : 0)];
    if (k == FACE_PERIODIC)
      q[a] = wrapi(q[a], n);
    else if (k == FACE_WALL)
      bounce = true;
    else
      drop = true;
  }
  if (bounce) return (long long)opp19(i) * P.N + cell_of(P, x, y, z);
  if (drop) return -1;
  return (long long)i * P.N + cell_of(P, q[0], q[1], q[2]);
}

// D3Q7: destination cell of population i leaving (x,y,z), or -1 beyond a non-periodic face.
LBM_HD int dest7_cell(const Params& P, int x, int y, int z, int i) {
  int q[3] = {x + c7x(i), y + c7y(i), z + c7z(i)};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = dim_of(P, a);
    if (q[a] >= 0 && q[a] < n) continue;
    if (P.face_kind[2 * a + (q[a] >= n ? 1 : 0)] != FACE_PERIODIC) return -1;
    q[a] = wrapi(q[a], n);
  }
  return cell_of(P, q[0], q[1], q[2]);
}

// Neighbours of one cell, per axis a and step k (0: -1, 1: +1): the cell-index
// offset (periodic faces wrap; 0 beyond a non-periodic face) and the kind of
// face crossed (0 inside or periodic, FACE_WALL, FACE_OPEN).  The push, psi and
// velocity rules of the step all derive from this table without branching on
// the cell's position.
struct Nb {
  int off[3][2];
  int kind[3][2];
};

LBM_HD void make_nb(const Params& P, int x, int y, int z, Nb& nb) {
  const int q[3] = {x, y, z};
  const int n[3] = {P.nx, P.ny, P.nz};
  const int st[3] = {1, P.nx, P.nx * P.ny};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool per = P.face_kind[2 * a] == FACE_PERIODIC;
    const bool lo = q[a] == 0, hi = q[a] == n[a] - 1;
    nb.off[a][0] = !lo ? -st[a] : (per ? (n[a] - 1) * st[a] : 0);
    nb.kind[a][0] = (!lo || per) ? 0 : P.face_kind[2 * a];
    nb.off[a][1] = !hi ? st[a] : (per ? -(n[a] - 1) * st[a] : 0);
    nb.kind[a][1] = (!hi || per) ? 0 : P.face_kind[2 * a + 1];
  }
}

// The table of a cell whose moves cross no wall or open face and no y or z face: plain
// strides, wrapped across periodic x faces, kind 0 everywhere (INNER).
LBM_HD void make_nb_inner(const Params& P, int x, Nb& nb) {
  const int st[3] = {1, P.nx, P.nx * P.ny};
  nb.off[0][0] = x == 0 ? P.nx - 1 : -1;
  nb.off[0][1] = x == P.nx - 1 ? 1 - P.nx : 1;
#pragma unroll
  for (int a = 1; a < 3; ++a) {
    nb.off[a][0] = -st[a];
    nb.off[a][1] = st[a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) nb.kind[a][0] = nb.kind[a][1] = 0;
}

// true when the cell lies away from the y and z faces and, unless x is periodic, from
// the x faces: the cells that make_nb_inner describes
LBM_HD bool inner_cell(const Params& P, int x, int y, int z) {
  return (P.face_kind[0] == FACE_PERIODIC || (x >= 1 && x <= P.nx - 2)) && y >= 1 && y <= P.ny - 2 && z >= 1 &&
         z <= P.nz - 2;
}

// kinds crossed by a move (cx, cy, cz), OR-ed (FACE_WALL = 1, FACE_OPEN = 2)
LBM_HD int nb_kind(const Nb& nb, int cx, int cy, int cz) {
  return (cx ? nb.kind[0][cx > 0] : 0) | (cy ? nb.kind[1][cy > 0] : 0) | (cz ? nb.kind[2][cz > 0] : 0);
}
LBM_HD int nb_off(const Nb& nb, int cx, int cy, int cz) {
  return (cx ? nb.off[0][cx > 0] : 0) + (cy ? nb.off[1][cy > 0] : 0) + (cz ? nb.off[2][cz > 0] : 0);
}
// psi rule: a wall mirrors through the wall layer (Eq. 36 at 90 degrees), an
// open face copies the boundary node, periodic faces wrap.
LBM_HD int nb_off_psi(const Nb& nb, int cx, int cy, int cz) {
  int o = 0;
  if (cx) o += nb.kind[0][cx > 0] == FACE_WALL ? nb.off[0][cx < 0] : nb.off[0][cx > 0];
  if (cy) o += nb.kind[1][cy > 0] == FACE_WALL ? nb.off[1][cy < 0] : nb.off[1][cy > 0];
  if (cz) o += nb.kind[2][cz > 0] == FACE_WALL ? nb.off[2][cz < 0] : nb.off[2][cz > 0];
  return o;
}

// The lookups of a table known at compile time to belong to a cell that crosses no wall
// or open face (INNER): the kind is 0 and the psi rule is the (wrapped) offset.
template <bool INNER>
LBM_HD int nbk(const Nb& nb, int cx, int cy, int cz) {
  if constexpr (INNER)
    return 0;
  else
    return nb_kind(nb, cx, cy, cz);
}
template <bool INNER>
LBM_HD int nbo_psi(const Nb& nb, int cx, int cy, int cz) {
  if constexpr (INNER)
    return nb_off(nb, cx, cy, cz);
  else
    return nb_off_psi(nb, cx, cy, cz);
}

// v on every active lane of the warp (device); the lane's own v on the host
LBM_DEV bool warp_all(bool v) {
#if defined(__CUDA_ARCH__)
  return __all_sync(__activemask(), v);
#else
  return v;
#endif
}

// load through L2 only (cache-global); a plain load on the host
LBM_DEV float ld_cg(const float* p) {
#if defined(__CUDA_ARCH__)
  return __ldcg(p);
#else
  return *p;
#endif
}

// psi at lattice point (x,y,z) that may lie outside the domain: periodic faces
// wrap; open faces copy the boundary node; wall faces mirror through the wall
// layer and add the wetting term sqrt(|grad_t psi|^2) tan(pi/2 - theta) of
// Eq. 36 when exactly one non-periodic axis is crossed.
LBM_DEV float psi_ext(const Params& P, const float* psi, int x, int y, int z) {
  int q[3] = {x, y, z}, r[3];
  int nout = 0, wax = -1, wface = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = dim_of(P, a), v = q[a];
    if (v >= 0 && v < n) {
      r[a] = v;
      continue;
    }
    const int face = 2 * a + (v >= n ? 1 : 0);
    const int k = P.face_kind[face];
    if (k == FACE_PERIODIC) {
      r[a] = wrapi(v, n);
      continue;
    }
    ++nout;
    if (k == FACE_OPEN) {
      r[a] = v < 0 ? 0 : n - 1;
    } else {
      r[a] = v < 0 ? -v : 2 * (n - 1) - v;
      wax = a;
      wface = face;
    }
  }
  float val = ld_cg(psi + cell_of(P, r[0], r[1], r[2]));
  if (nout == 1 && wax >= 0) {
    const float tn = P.tan_wet[wface];
    if (tn != 0.f) {
      const int layer = q[wax] < 0 ? 0 : dim_of(P, wax) - 1;
      float s2 = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (b == wax) continue;
        const int nb = dim_of(P, b);
        int up = q[b] + 1, dn = q[b] - 1;
        if (P.face_kind[2 * b] == FACE_PERIODIC) {
          up = wrapi(up, nb);
          dn = wrapi(dn, nb);
        } else {
          up = up > nb - 1 ? nb - 1 : up;
          dn = dn < 0 ? 0 : dn;
        }
        int pp[3] = {r[0], r[1], r[2]}, pm[3] = {r[0], r[1], r[2]};
        pp[wax] = pm[wax] = layer;
        pp[b] = up;
        pm[b] = dn;
        const float d = ld_cg(psi + cell_of(P, pp[0], pp[1], pp[2])) - ld_cg(psi + cell_of(P, pm[0], pm[1], pm[2]));
        s2 += d * d;
      }
      val += sqrtf(s2) * tn;
    }
  }
  return val;
}

// Real velocity at a point that may lie outside: zero beyond a wall, the
// boundary node's value beyond an open face, periodic wrap otherwise.
LBM_DEV void u_ext(const Params& P, const float* ux, const float* uy, const float* uz, int x, int y, int z, float& ox, float& oy, float& oz) {
  int q[3] = {x, y, z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = dim_of(P, a), v = q[a];
    if (v >= 0 && v < n) continue;
    const int k = P.face_kind[2 * a + (v >= n ? 1 : 0)];
    if (k == FACE_WALL) {
      ox = oy = oz = 0.f;
      return;
    }
    q[a] = (k == FACE_PERIODIC) ? wrapi(v, n) : (v < 0 ? 0 : n - 1);
  }
  const int c = cell_of(P, q[0], q[1], q[2]);
  ox = ld_cg(ux + c);
  oy = ld_cg(uy + c);
  oz = ld_cg(uz + c);
}

}  // namespace lbm
