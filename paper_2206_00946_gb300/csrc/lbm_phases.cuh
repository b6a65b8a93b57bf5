// The four phases of one time step, written per cell so that the one-launch-
// per-phase schedule and the fused pipelined kernel run the same code.
//   A  macro: rho, j = sum c f, T = sum g, p_EOS, psi          (Eqs. 3, 7, 37)
//   B  force: F = -G psi sum varpi psi(x+c) c, u = (j + F/2)/rho (Eqs. 5, 6, 36)
//   C  collide + stream: D3Q19 MRT-EDM collision pushed to x+c (bounce-back at
//      walls), D3Q7 collision with the source pushed with the relaxed streaming
//      (Eqs. 8, 13-15, 27-29, 34)
//   D  boundary: constant-pressure open faces (Sec. 3.3) and non-equilibrium
//      extrapolation of g at Dirichlet nodes (Sec. 3.1), on the new state
#pragma once

#include "lbm_lattice.cuh"

namespace lbm {

struct Aux {
  float *rho, *jx, *jy, *jz, *psi;  // phase A
  float *Fx, *Fy, *Fz, *ux, *uy, *uz;  // phase B
};

__device__ __forceinline__ void sum19(const float* f, float& rho, float& jx, float& jy, float& jz) {
  rho = ((f[0] + (f[1] + f[2])) + ((f[3] + f[4]) + (f[5] + f[6]))) +
        (((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14]))) + ((f[15] + f[16]) + (f[17] + f[18]));
  jx = ((f[1] - f[2]) + (f[7] - f[8])) + ((f[9] - f[10]) + (f[11] - f[12])) + (f[13] - f[14]);
  jy = ((f[3] - f[4]) + (f[7] - f[8])) + ((f[10] - f[9]) + (f[15] - f[16])) + (f[17] - f[18]);
  jz = ((f[5] - f[6]) + (f[11] - f[12])) + ((f[14] - f[13]) + (f[15] - f[16])) + (f[18] - f[17]);
}

__device__ __forceinline__ float sum7(const float* g) {
  return (g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]));
}

__device__ __forceinline__ void cell_xyz(const Params& P, int c, int& x, int& y, int& z) {
  const int row = (int)fdiv((unsigned)c, P.dnx_mul, P.dnx_shr);
  x = c - row * P.nx;
  z = (int)fdiv((unsigned)row, P.dny_mul, P.dny_shr);
  y = row - z * P.ny;
}

// Boundary nodes of plane z are enumerated as candidates k = 0..count-1: the
// whole plane when z lies on a non-periodic z face, otherwise its perimeter
// rows/columns on non-periodic x or y faces.
__device__ __forceinline__ int boundary_count(const Params& P, int z) {
  const bool xnp = P.face_kind[0] != FACE_PERIODIC, ynp = P.face_kind[2] != FACE_PERIODIC;
  if (P.face_kind[4] != FACE_PERIODIC && (z == 0 || z == P.nz - 1)) return P.nx * P.ny;
  if (xnp && ynp) return 2 * P.nx + 2 * (P.ny - 2);
  if (xnp) return 2 * P.ny;
  if (ynp) return 2 * P.nx;
  return 0;
}

__device__ __forceinline__ void boundary_xy(const Params& P, int z, int k, int& x, int& y) {
  const bool xnp = P.face_kind[0] != FACE_PERIODIC, ynp = P.face_kind[2] != FACE_PERIODIC;
  if (P.face_kind[4] != FACE_PERIODIC && (z == 0 || z == P.nz - 1)) {
    y = (int)fdiv((unsigned)k, P.dnx_mul, P.dnx_shr);
    x = k - y * P.nx;
  } else if (xnp && ynp) {
    if (k < 2 * P.nx) {
      y = k < P.nx ? 0 : P.ny - 1;
      x = k < P.nx ? k : k - P.nx;
    } else {
      const int k2 = k - 2 * P.nx;
      y = 1 + (k2 >> 1);
      x = (k2 & 1) ? P.nx - 1 : 0;
    }
  } else if (xnp) {
    y = k >> 1;
    x = (k & 1) ? P.nx - 1 : 0;
  } else {
    y = k < P.nx ? 0 : P.ny - 1;
    x = k < P.nx ? k : k - P.nx;
  }
}

__device__ __forceinline__ bool interior1(const Params& P, int x, int y, int z) {
  return x >= 1 && x <= P.nx - 2 && y >= 1 && y <= P.ny - 2 && z >= 1 && z <= P.nz - 2;
}

// ------------------------------------------------------------------- A -----
__device__ __forceinline__ void phaseA(const Params& P, int c, const float* __restrict__ f,
                                       const float* __restrict__ g, const Aux& X, float* __restrict__ Tout,
                                       int& err) {
  float fl[19], gl[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) fl[i] = __ldg(f + i * P.N + c);
#pragma unroll
  for (int i = 0; i < 7; ++i) gl[i] = __ldg(g + i * P.N + c);
  float rho, jx, jy, jz;
  sum19(fl, rho, jx, jy, jz);
  const float T = sum7(gl);
  if (!isfinite(rho) || !isfinite(T) || !isfinite(jx + jy + jz)) err |= ERRF_NONFINITE;
  float p, dpdT, psi;
  eos_pr(P, rho, T, p, dpdT);
  if (!psi_of(P, rho, p, psi)) err |= ERRF_PSI;
  X.rho[c] = rho;
  X.jx[c] = jx;
  X.jy[c] = jy;
  X.jz[c] = jz;
  X.psi[c] = psi;
  if (Tout) Tout[c] = T;
}

// ------------------------------------------------------------------- B -----
__device__ __forceinline__ void phaseB(const Params& P, int c, const Aux& X) {
  int x, y, z;
  cell_xyz(P, c, x, y, z);
  const float* psi = X.psi;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  if (interior1(P, x, y, z)) {
    const int sY = P.nx, sZ = P.nx * P.ny;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const float v = varpi19(i) * __ldcg(psi + c + c19x(i) + c19y(i) * sY + c19z(i) * sZ);
      sx += c19x(i) * v;
      sy += c19y(i) * v;
      sz += c19z(i) * v;
    }
  } else {
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const float v = varpi19(i) * psi_ext(P, psi, x + c19x(i), y + c19y(i), z + c19z(i));
      sx += c19x(i) * v;
      sy += c19y(i) * v;
      sz += c19z(i) * v;
    }
  }
  const float k = -P.G * __ldcg(psi + c);
  const float Fx = k * sx, Fy = k * sy, Fz = k * sz;
  X.Fx[c] = Fx;
  X.Fy[c] = Fy;
  X.Fz[c] = Fz;
  const int m = P.any_nonperiodic ? node_faces(P, x, y, z) : 0;
  if (m && on_wall(P, m)) {
    X.ux[c] = X.uy[c] = X.uz[c] = 0.f;
  } else {
    const float ir = 1.f / __ldcg(X.rho + c);
    X.ux[c] = (__ldcg(X.jx + c) + 0.5f * Fx) * ir;
    X.uy[c] = (__ldcg(X.jy + c) + 0.5f * Fy) * ir;
    X.uz[c] = (__ldcg(X.jz + c) + 0.5f * Fz) * ir;
  }
}

// ------------------------------------------------------------------- C -----
__device__ __forceinline__ void phaseC(const Params& P, int c, const float* __restrict__ fA,
                                       const float* __restrict__ gA, float* __restrict__ fB,
                                       float* __restrict__ gB, const Aux& X) {
  int x, y, z;
  cell_xyz(P, c, x, y, z);
  const long long N = P.N;
  float fl[19], gl[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) fl[i] = __ldg(fA + i * N + c);
#pragma unroll
  for (int i = 0; i < 7; ++i) gl[i] = __ldg(gA + i * N + c);
  float rho, jx, jy, jz;
  sum19(fl, rho, jx, jy, jz);
  const float T = sum7(gl);
  const int m = P.any_nonperiodic ? node_faces(P, x, y, z) : 0;
  const bool wall = m && on_wall(P, m);
  const float Fx = __ldcg(X.Fx + c), Fy = __ldcg(X.Fy + c), Fz = __ldcg(X.Fz + c);
  float ux, uy, uz;
  if (wall && P.wall_ueq_zero) {
    ux = uy = uz = 0.f;
  } else {
    const float ir = 1.f / rho;
    ux = jx * ir;
    uy = jy * ir;
    uz = jz * ir;
  }
  float fs[19];
  collide19(P, fl, rho, ux, uy, uz, Fx, Fy, Fz, fs);

  const bool in1 = interior1(P, x, y, z);
  const int sY = P.nx, sZ = P.nx * P.ny;
  if (in1) {
#pragma unroll
    for (int i = 0; i < 19; ++i) fB[i * N + (c + c19x(i) + c19y(i) * sY + c19z(i) * sZ)] = fs[i];
  } else {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const long long d = dest19(P, x, y, z, i);
      if (d >= 0) fB[d] = fs[i];
    }
  }

  // D3Q7: div u by the isotropic D3Q19 difference, grad T from the local moments
  float du = 0.f;
  if (in1) {
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const int n = c + c19x(i) + c19y(i) * sY + c19z(i) * sZ;
      float s = 0.f;
      if (c19x(i)) s += c19x(i) * __ldcg(X.ux + n);
      if (c19y(i)) s += c19y(i) * __ldcg(X.uy + n);
      if (c19z(i)) s += c19z(i) * __ldcg(X.uz + n);
      du += w19(i) * s;
    }
  } else {
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      float vx, vy, vz;
      u_ext(P, X.ux, X.uy, X.uz, x + c19x(i), y + c19y(i), z + c19z(i), vx, vy, vz);
      du += w19(i) * (c19x(i) * vx + c19y(i) * vy + c19z(i) * vz);
    }
  }
  du *= 3.f;
  float p, dpdT;
  eos_pr(P, rho, T, p, dpdT);
  const float uxr = __ldcg(X.ux + c), uyr = __ldcg(X.uy + c), uzr = __ldcg(X.uz + c);
  float gs[7];
  collide7(P, gl, rho, T, uxr, uyr, uzr, du, dpdT, gs);
  const float icv = P.inv_cv;
  // relaxed streaming: g_i(y) += (g*_i(y - c_i) - g_i(y)) / (rho(y) c_v)
  gB[c] = gl[0] + (gs[0] - gl[0]) / (rho * P.cv);
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    int yc;
    if (in1)
      yc = c + c7x(i) + c7y(i) * sY + c7z(i) * sZ;
    else
      yc = dest7_cell(P, x, y, z, i);
    if (yc < 0) continue;
    const float gold = __ldg(gA + i * N + yc);
    const float ry = __ldcg(X.rho + yc);
    gB[i * N + yc] = gold + (gs[i] - gold) / ry * icv;
  }
}

// ------------------------------------------------------------------- D -----
__device__ __forceinline__ float face_T_at(const Params& P, int face, int x, int y, int z) {
  const int a = face >> 1;
  const float* t = P.Tface[face];
  if (a == 0) return t[y + P.ny * z];
  if (a == 1) return t[x + P.nx * z];
  return t[x + P.nx * y];
}

__device__ __forceinline__ void phaseD(const Params& P, int c, int x, int y, int z, int m,
                                       float* __restrict__ fB, float* __restrict__ gB, const Aux& X) {
  const long long N = P.N;
  int nnp = 0, nopen = 0, oface = -1;
  float rb = 0.f, Tb = 0.f;
  int q[3] = {x, y, z};
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    if (!((m >> f) & 1)) continue;
    ++nnp;
    if (P.face_kind[f] == FACE_OPEN) {
      ++nopen;
      oface = f;
      rb += P.face_rho[f];
    }
    Tb += face_T_at(P, f, x, y, z);
    q[f >> 1] += (f & 1) ? -1 : 1;
  }
  if (nopen) {
    float fl[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = __ldcg(fB + i * N + c);
    if (nnp == 1) {
      zouhe(oface, P.face_rho[oface], __ldcg(X.Fx + c), __ldcg(X.Fy + c), __ldcg(X.Fz + c), fl);
    } else {
      float fe[19];
      feq19(rb / (float)nopen, 0.f, 0.f, 0.f, fe);
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const int sx = x - c19x(i), sy = y - c19y(i), sz = z - c19z(i);
        const bool unk = ((sx < 0 || sx >= P.nx) && P.face_kind[0] != FACE_PERIODIC) ||
                         ((sy < 0 || sy >= P.ny) && P.face_kind[2] != FACE_PERIODIC) ||
                         ((sz < 0 || sz >= P.nz) && P.face_kind[4] != FACE_PERIODIC);
        if (unk) fl[i] = fe[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) fB[i * N + c] = fl[i];
  }
  Tb /= (float)nnp;
  const int cf = cell_of(P, q[0], q[1], q[2]);
  float gf[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) gf[i] = __ldcg(gB + i * N + cf);
  const float Tf = sum7(gf);
  const float w0 = 1.f - P.wbar, w1 = P.wbar * (1.f / 6.f);
  gB[c] = w0 * Tb + gf[0] - w0 * Tf;
#pragma unroll
  for (int i = 1; i < 7; ++i) gB[i * N + c] = w1 * Tb + gf[i] - w1 * Tf;
}

}  // namespace lbm
