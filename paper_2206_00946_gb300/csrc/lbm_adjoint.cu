// Discrete adjoint of the time step: lbm_record keeps checkpoints of a forward
// run, lbm_adjoint_step runs the transposed step backwards through it,
// recomputing each segment between checkpoints, and accumulates in FP64 the
// gradients of a loss of the final rho and T fields with respect to the
// per-node Dirichlet face temperatures (every step) and the initial
// temperature field.  The step is differentiated exactly as the forward
// kernels compute it (FP32): open-face rules, extrapolation, relaxed
// streaming, D3Q7 and D3Q19 collisions, force stencil, velocity and the
// EOS / psi chain rule, with the ghost rules of the stencils transposed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_adjoint_cell.cuh"
#include "lbm_ctx.cuh"

namespace {

constexpr int kT = 256;

int blocks_for(long long n) {
  long long b = (n + kT - 1) / kT;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)(b < 1 ? 1 : b);
}

// Programmatic dependent launch: a kernel launched after another on the same
// stream with launch_pdl may start while that kernel finishes.  It reads the
// earlier kernel's results only after griddep_wait, which returns once that grid
// has completed and its writes are visible (at once for an ordinary launch).
// griddep_launch lets the next such kernel be scheduled.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... K, typename... A>
cudaError_t launch_pdl(bool pdl, void (*kern)(K...), int grid, int block, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// adjoint scratch fields, N floats each unless noted
struct AdjAux {
  float *Fb;     // 3N: d L / d F
  float *Rb;     // d L / d rho (partial)
  float *Ub;     // 3N: d L / d u from the D3Q7 collision at the cell itself
  float *Divb;   // d L / d (div u)
  float *Dpb;    // d L / d (dp/dT)
};

// Segment slot: the state of one step and the scratch the forward step
// computed from it: f (19N), g (7N), rho, psi, F (3N), u (3N), div u and the
// post-collision D3Q7 populations g* (7N) = 42 N floats.
constexpr int kSlot = 42;

Aux slot_aux(float* s, long long N, const Aux& ctxX) {
  Aux X = ctxX;  // j is not needed by the adjoint (the step does not store it)
  X.rho = s + 26 * N;
  X.psi = s + 27 * N;
  X.Fx = s + 28 * N;
  X.Fy = s + 29 * N;
  X.Fz = s + 30 * N;
  X.ux = s + 31 * N;
  X.uy = s + 32 * N;
  X.uz = s + 33 * N;
  X.divu = s + 34 * N;
  X.gstar = s + 35 * N;
  return X;
}

// ---------------------------------------------------------------- forward --
__global__ void k_adj_seed(Params P, const float* rhob, const float* Tb, float* fb, float* gb) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    const float r = rhob ? rhob[c] : 0.f, t = Tb ? Tb[c] : 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) fb[i * P.N + c] = r;
#pragma unroll
    for (int i = 0; i < 7; ++i) gb[i * P.N + c] = t;
  }
}

// --------------------------------------------------------- face nodes -------
// Transposes of the rules applied last in the forward step, in place on the
// adjoint of the new state: the extrapolation of g at every face node (the
// face temperature gradient is accumulated in FP64; the inward neighbours
// x_f are shared by edge and face nodes, hence the atomics) and the open-face
// rule (unknown populations folded into the known ones and into d L / d F).
struct DT6 {
  double* p[6];
};

// PART 0: the extrapolation of g (touches only the g adjoint and the face
// gradients); PART 1: the open-face rule (only the f adjoint and d L / d F).  The
// two parts run on different streams, each ahead of its lattice's transpose.
template <int PART>
__global__ void k_adj_faces(Params P, float* fb, float* gb, Aux X, float* Fb, DT6 dTf) {
  const long long N = P.N;
  const float w0 = 1.f - P.wbar, w1 = P.wbar * (1.f / 6.f);
  griddep_launch();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)P.bd_total; k += gridDim.x * blockDim.x) {
    int x, y, z;
    boundary_candidate(P, k, x, y, z);
    const int m = node_faces(P, x, y, z);
    if (!m) continue;
    const int c = cell_of(P, x, y, z);
    int nnp = 0, nopen = 0, oface = -1, q[3] = {x, y, z};
#pragma unroll
    for (int fc = 0; fc < 6; ++fc) {
      if (!((m >> fc) & 1)) continue;
      ++nnp;
      if (P.face_kind[fc] == FACE_OPEN) {
        ++nopen;
        oface = fc;
      }
      q[fc >> 1] += (fc & 1) ? -1 : 1;
    }
    if (PART == 0) {
      // extrapolation: g_k(x_b) = w_k T_b + g_k(x_f) - w_k sum_j g_j(x_f)
      float a[7], Tb = 0.f;
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        a[i] = gb[i * N + c];
        Tb += (i == 0 ? w0 : w1) * a[i];
      }
      const int cf = cell_of(P, q[0], q[1], q[2]);
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        gb[i * N + c] = 0.f;
        atomicAdd(gb + i * N + cf, a[i] - Tb);
      }
#pragma unroll
      for (int fc = 0; fc < 6; ++fc) {
        if (!((m >> fc) & 1)) continue;
        const int ax = fc >> 1;
        const int idx = ax == 0 ? y + P.ny * z : (ax == 1 ? x + P.nx * z : x + P.nx * y);
        dTf.p[fc][idx] += (double)Tb / nnp;  // one (face, node) entry per thread
      }
      continue;
    }
    if (nopen) {
      float fl[19];
#pragma unroll
      for (int i = 0; i < 19; ++i) fl[i] = fb[i * N + c];
      if (nnp == 1) {
        float F3[3] = {0.f, 0.f, 0.f};
        zouhe_vjp(oface, P.face_rho[oface], fl, F3);
        Fb[c] = F3[0];  // the first term of d L / d F at this node (k_adj_c19 adds its own)
        Fb[N + c] = F3[1];
        Fb[2 * N + c] = F3[2];
      } else {
        const unsigned unk = unknown19(P, x, y, z);
#pragma unroll
        for (int i = 1; i < 19; ++i)
          if ((unk >> i) & 1u) fl[i] = 0.f;  // f^eq(rho_b, 0): constant
      }
#pragma unroll
      for (int i = 0; i < 19; ++i) fb[i * N + c] = fl[i];
    }
  }
}

// ------------------------------------------------------- D3Q19 transpose ----
// d L / d f*(x) gathered from the slots the push wrote (bounce-back included),
// then the collision's vector-Jacobian product.
__global__ void __launch_bounds__(256, 2) k_adj_c19(Params P, const float* f, const float* fb1, float* fb0, Aux X,
                                                     float* Fb) {
  const long long N = P.N;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    Nb nb;
    make_nb(P, x, y, z, nb);
    float fl[19], fsb[19], fbo[19], F3[3] = {X.Fx[c], X.Fy[c], X.Fz[c]}, Fo[3];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = f[i * N + c];
    griddep_wait();  // the open-face transpose before this kernel wrote fb1 and Fb
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const int k = nb_kind(nb, c19x(i), c19y(i), c19z(i));
      fsb[i] = k == 0 ? fb1[i * N + c + nb_off(nb, c19x(i), c19y(i), c19z(i))]
                      : ((k & FACE_WALL) ? fb1[opp19(i) * N + c] : 0.f);
    }
    const int m = P.any_nonperiodic ? node_faces(P, x, y, z) : 0;
    const bool wall = m && on_wall(P, m);
    if (P.fast19)  // the closed form of the rate-1 case, as in the forward step
      collide19_fast_vjp(P, fl, !(wall && P.wall_ueq_zero), F3, fsb, fbo, Fo);
    else
      collide19_vjp(P, fl, !(wall && P.wall_ueq_zero), F3, fsb, fbo, Fo);
#pragma unroll
    for (int i = 0; i < 19; ++i) fb0[i * N + c] = fbo[i];
    // d L / d F starts here, except at nodes of a single open face, where the
    // open-face rule's transpose (same stream, launched before) stored its term
    if (m && __popc(m) == 1 && on_open(P, m)) {
      Fo[0] += Fb[c];
      Fo[1] += Fb[N + c];
      Fo[2] += Fb[2 * N + c];
    }
    Fb[c] = Fo[0];
    Fb[N + c] = Fo[1];
    Fb[2 * N + c] = Fo[2];
  }
}

// -------------------------------------------------------- D3Q7 transpose ----
// Relaxed streaming g'_i(y) = g_i(y) + (g*_i(y - c_i) - g_i(y)) / (rho(y) c_v)
// transposed at x both as a source (d L / d g*) and as a destination (the
// retained g_i(x) and rho(x) c_v), then the D3Q7 collision's product.
__global__ void k_adj_c7(Params P, const float* g, const float* gb1, float* gb0, Aux X, AdjAux A) {
  const long long N = P.N;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    Nb nb;
    make_nb(P, x, y, z, nb);
    float gl[7], gsb[7], gout[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = g[i * N + c];
    const float rho = X.rho[c], T = sum7(gl);
    const float beta = rcp(rho * P.cv), ir = rcp(rho);
    griddep_wait();  // the extrapolation transpose before this kernel wrote gb1
    // rest population: source and destination are the cell itself
    float a = gb1[c];
    gsb[0] = a * beta;
    gout[0] = (1.f - beta) * a;
    float rhob = -a * (X.gstar[c] - gl[0]) * beta * ir;
#pragma unroll
    for (int i = 1; i < 7; ++i) {
      const int ax = (i - 1) >> 1, s = (i & 1) ? 1 : 0;  // s: 1 for +c, 0 for -c
      a = gb1[i * N + c];
      // as a source: population i goes to y = x + c_i
      if (nb.kind[ax][s] == 0) {
        const int yd = c + nb.off[ax][s];
        gsb[i] = gb1[i * N + yd] * rcp(X.rho[yd] * P.cv);
      } else {
        gsb[i] = 0.f;
      }
      // as a destination: the source x - c_i
      if (nb.kind[ax][1 - s] == 0) {
        const int sc = c + nb.off[ax][1 - s];
        gout[i] = (1.f - beta) * a;
        rhob -= a * (X.gstar[i * N + sc] - gl[i]) * beta * ir;
      } else {
        gout[i] = a;
      }
    }
    const float du = X.divu[c];
    float p, dpdT;
    eos_pr(P, rho, T, p, dpdT);
    const float u3[3] = {X.ux[c], X.uy[c], X.uz[c]};
    float gbv[7], rb7, Tb, ub[3], divb, dpb;
    collide7_vjp(P, gl, rho, T, u3, du, dpdT, gsb, gbv, rb7, Tb, ub, divb, dpb);
#pragma unroll
    for (int i = 0; i < 7; ++i) gb0[i * N + c] = gout[i] + gbv[i] + Tb;
    A.Rb[c] = rhob + rb7;
    A.Ub[c] = ub[0];
    A.Ub[N + c] = ub[1];
    A.Ub[2 * N + c] = ub[2];
    A.Divb[c] = divb;
    A.Dpb[c] = dpb;
  }
}

// ------------------------------------------------- stencil transposes -------
// A stencil read of the forward step at x in direction c (the psi force, the
// div u difference) lands on the cell y = x + c, or, beyond a non-periodic
// face, on the ghost rule's image (open face: the boundary node itself; wall,
// psi only: the mirror node; wall, velocity: nothing).  Its transpose at y
// gathers from every such x.  The main source x = y - c exists exactly when
// the move from y by -c crosses no non-periodic face; the other sources (an
// "extra" coordinate on some axis) exist only for y on or next to a face.
// Extra source coordinate of ya on axis a for a move of sign sg (-1: none).
__device__ __forceinline__ int extra_coord(const Params& P, int a, int ya, int sg, int mode) {
  if (P.face_kind[2 * a] == FACE_PERIODIC) return -1;
  const int n = dim_of(P, a);
  const int b = sg > 0 ? n - 1 : 0;
  const int kind = P.face_kind[2 * a + (sg > 0 ? 1 : 0)];
  if (kind == FACE_OPEN && ya == b) return b;
  if (kind == FACE_WALL && mode == 0 && ya == b - sg) return b;
  return -1;
}

// Extra coordinates of a cell for the six (axis, sign) pairs; bit 2a+(sg>0) of
// the returned mask is set where one exists.
__device__ __forceinline__ unsigned extra_table(const Params& P, const int* q, int mode, int (*ec)[2]) {
  unsigned m = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      ec[a][s] = extra_coord(P, a, q[a], s ? 1 : -1, mode);
      m |= (ec[a][s] >= 0 ? 1u : 0u) << (2 * a + s);
    }
  return m;
}

// main source coordinate of ya for a move by c (-1: none)
__device__ __forceinline__ int main_coord(const Params& P, int a, int ya, int c) {
  if (c == 0) return ya;
  const int n = dim_of(P, a), s = ya - c;
  if (s >= 0 && s < n) return s;
  return P.face_kind[2 * a] == FACE_PERIODIC ? wrapi(s, n) : -1;
}

// sum of val(x) over the sources of a move (cx, cy, cz) with at least one
// extra coordinate
template <typename V>
__device__ __forceinline__ float extra_sources(const Params& P, const int* q, int cx, int cy, int cz,
                                               const int (*ec)[2], V val) {
  const int c3[3] = {cx, cy, cz};
  int mc[3], e3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mc[a] = main_coord(P, a, q[a], c3[a]);
    e3[a] = c3[a] ? ec[a][c3[a] > 0] : -1;
  }
  float s = 0.f;
#pragma unroll
  for (int msk = 1; msk < 8; ++msk) {
    int r[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      r[a] = ((msk >> a) & 1) ? e3[a] : mc[a];
      ok = ok && r[a] >= 0;
    }
    if (ok) s += val(cell_of(P, r[0], r[1], r[2]));
  }
  return s;
}

// does the move (cx, cy, cz) have an extra source at a cell with mask m
__device__ __forceinline__ bool has_extra(unsigned m, int cx, int cy, int cz) {
  return (cx && ((m >> (0 + (cx > 0))) & 1)) || (cy && ((m >> (2 + (cy > 0))) & 1)) ||
         (cz && ((m >> (4 + (cz > 0))) & 1));
}

// d L / d u(y) = the D3Q7 collision's own term + the div u stencil transposed,
// then u = (j + F/2) / rho (zero at walls): d L / d j, d L / d F, d L / d rho.
__global__ void k_adj_u(Params P, Aux X, AdjAux A, float* Jb) {
  const long long N = P.N;
  griddep_launch();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int q[3];
    cell_xyz(P, c, q[0], q[1], q[2]);
    Nb nb;
    make_nb(P, q[0], q[1], q[2], nb);
    float ub[3] = {A.Ub[c], A.Ub[N + c], A.Ub[2 * N + c]};
    int ec[3][2];
    const unsigned em = P.any_nonperiodic ? extra_table(P, q, 1, ec) : 0u;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
      float s = nb_kind(nb, -cx, -cy, -cz) == 0 ? A.Divb[c + nb_off(nb, -cx, -cy, -cz)] : 0.f;
      if (has_extra(em, cx, cy, cz)) s += extra_sources(P, q, cx, cy, cz, ec, [&](int x) { return A.Divb[x]; });
      const float k = 3.f * w19(i) * s;
      if (cx) ub[0] += cx * k;
      if (cy) ub[1] += cy * k;
      if (cz) ub[2] += cz * k;
    }
    const int m = P.any_nonperiodic ? node_faces(P, q[0], q[1], q[2]) : 0;
    float j3[3] = {0.f, 0.f, 0.f};
    if (!(m && on_wall(P, m))) {
      const float ir = rcp(X.rho[c]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        j3[a] = ub[a] * ir;
        A.Fb[a * N + c] += 0.5f * ub[a] * ir;
      }
      A.Rb[c] -= (ub[0] * X.ux[c] + ub[1] * X.uy[c] + ub[2] * X.uz[c]) * ir;
    }
    Jb[c] = j3[0];
    Jb[N + c] = j3[1];
    Jb[2 * N + c] = j3[2];
  }
}

// d L / d psi(y) from F(x) = -G psi(x) sum_i varpi_i psi(x + c_i) c_i (the
// cell's own factor and the transposed stencil), then through the EOS to the
// cell's complete d L / d rho (Rb) and d L / d T (Tbar).
__global__ void k_adj_psi(Params P, const float* g, Aux X, AdjAux A, float* Tbar) {
  const long long N = P.N;
  const Hint h = make_hint();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int q[3];
    cell_xyz(P, c, q[0], q[1], q[2]);
    Nb nb;
    make_nb(P, q[0], q[1], q[2], nb);
    int ec[3][2];
    const unsigned em = P.any_nonperiodic ? extra_table(P, q, 0, ec) : 0u;
    float S[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
      const float v = varpi19(i) * ld_aux(X.psi + c + nb_off_psi(nb, cx, cy, cz), h);
      if (cx) S[0] += cx * v;
      if (cy) S[1] += cy * v;
      if (cz) S[2] += cz * v;
    }
    float T = 0.f;
#pragma unroll
    for (int i = 0; i < 7; ++i) T += g[i * N + c];
    griddep_wait();  // d L / d F, rho and dp/dT of the kernels before
    griddep_launch();
    float psib = 0.f;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const int cx = c19x(i), cy = c19y(i), cz = c19z(i);
      // only the components the move has are loaded (0 * Fb is not folded away)
      auto term = [&](int x) {
        float s = 0.f;
        if (cx) s += cx * A.Fb[x];
        if (cy) s += cy * A.Fb[N + x];
        if (cz) s += cz * A.Fb[2 * N + x];
        return X.psi[x] * s;
      };
      float t = nb_kind(nb, -cx, -cy, -cz) == 0 ? term(c + nb_off(nb, -cx, -cy, -cz)) : 0.f;
      if (has_extra(em, cx, cy, cz)) t += extra_sources(P, q, cx, cy, cz, ec, term);
      psib += varpi19(i) * t;
    }
    psib = -P.G * (psib + A.Fb[c] * S[0] + A.Fb[N + c] * S[1] + A.Fb[2 * N + c] * S[2]);
    // the EOS chain rule of psi and dp/dT: the cell's complete d L / d rho and d L / d T
    float rhob = A.Rb[c], Tb = 0.f;
    psi_dpdT_vjp(P, X.rho[c], T, X.psi[c], psib, A.Dpb[c], rhob, Tb);
    A.Rb[c] = rhob;
    Tbar[c] = Tb;
  }
}

// The macroscopic fields rho = sum f, j = sum c f, T = sum g folded into the
// adjoint of the populations at time t (a streaming update).  The lattice
// transposes wrote fb0 and gb0 before d L / d u was taken, so they are loaded
// while the psi transpose finishes.
__global__ void k_adj_fold(Params P, AdjAux A, const float* Jb, const float* Tbar, float* fb0, float* gb0) {
  const long long N = P.N;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    float fv[19], gv[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) fv[i] = fb0[i * N + c];
#pragma unroll
    for (int i = 0; i < 7; ++i) gv[i] = gb0[i * N + c];
    griddep_wait();  // Rb and Tbar of the psi transpose
    const float rhob = A.Rb[c], Tb = Tbar[c];
    const float jx = Jb[c], jy = Jb[N + c], jz = Jb[2 * N + c];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      float s = fv[i] + rhob;
      if (c19x(i)) s += c19x(i) * jx;
      if (c19y(i)) s += c19y(i) * jy;
      if (c19z(i)) s += c19z(i) * jz;
      fb0[i * N + c] = s;
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) gb0[i * N + c] = gv[i] + Tb;
  }
}

// d L / d T0 = sum_i w_i d L / d g_i(0) for g_i(0) = w_i T0 (FP64)
__global__ void k_adj_T0(Params P, const float* gb, double* out) {
  const float w0 = 1.f - P.wbar, w1 = P.wbar * (1.f / 6.f);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    double s = (double)w0 * gb[c];
    for (int i = 1; i < 7; ++i) s += (double)w1 * gb[i * P.N + c];
    out[c] = s;
  }
}

}  // namespace

// ------------------------------------------------------------------- host --
struct AdjRec {
  int K = 0, nrec = 0, cur = 0;
  bool last_kept = false;    // seg holds the last segment, computed by lbm_record
  long long N = 0;
  std::vector<float*> ckpt;  // f (19N) + g (7N) at steps 0, K, 2K, ...
  float* fin = nullptr;      // the recorded final state (f, g)
  float* seg[2] = {nullptr, nullptr};  // K + 1 slots of kSlot * N floats each: the segment being
                                       // reversed and (when memory allows) the next one, recomputed
                                       // meanwhile on the side stream
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_adj[2] = {nullptr, nullptr}, ev_fork = nullptr,
              ev_c19 = nullptr;
  float* fb[2] = {nullptr, nullptr};
  float* gb[2] = {nullptr, nullptr};
  float* scr = nullptr;      // AdjAux fields + d L / d j
  double* dTf = nullptr;     // per-face accumulators, faces concatenated
  long long face_off[7] = {0, 0, 0, 0, 0, 0, 0};
  bool pdl = true;  // programmatic dependent launches within an adjoint step
  // K-step segments replayed from CUDA graphs, captured on first use from the
  // parameters below: the adjoint of a segment per (segment buffer, which of the
  // two adjoint buffers holds the newest adjoint), its recomputation per buffer
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gx[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t gr[2] = {nullptr, nullptr};
  Params gP{};
  Aux gX{};
  bool gpdl = true;
};

void adj_drop_graphs(AdjRec* r) {
  for (int b = 0; b < 2; ++b) {
    for (int k = 0; k < 2; ++k)
      if (r->gx[b][k]) {
        cudaGraphExecDestroy(r->gx[b][k]);
        r->gx[b][k] = nullptr;
      }
    if (r->gr[b]) {
      cudaGraphExecDestroy(r->gr[b]);
      r->gr[b] = nullptr;
    }
  }
}

// The graphs hold the parameters and scratch pointers they were captured with.
void adj_graph_key(lbm_ctx* c, AdjRec* r) {
  if (std::memcmp(&r->gP, &c->P, sizeof(Params)) || std::memcmp(&r->gX, &c->X, sizeof(Aux)) || r->gpdl != r->pdl) {
    adj_drop_graphs(r);
    std::memcpy(&r->gP, &c->P, sizeof(Params));
    std::memcpy(&r->gX, &c->X, sizeof(Aux));
    r->gpdl = r->pdl;
  }
}

// Captures the launches that `issue` makes on the private capture stream (the
// context stream may be the legacy default stream, which cannot be captured)
// into *gx.  Returns false, with nothing launched, when that fails.
template <typename F>
bool adj_capture(AdjRec* r, cudaGraphExec_t* gx, F issue) {
  if (!r->cap && cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int e = issue(r->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(r->cap, &g);
  bool ok = !e && ce == cudaSuccess && g;
  if (ok) ok = cudaGraphInstantiate(gx, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    *gx = nullptr;
    cudaGetLastError();
  }
  return ok;
}

void adj_free(lbm_ctx* c) {
  if (!c || !c->adj) return;
  AdjRec* r = c->adj;
  for (float* p : r->ckpt) cudaFree(p);
  cudaFree(r->fin);
  for (int k = 0; k < 2; ++k) {
    cudaFree(r->seg[k]);
    if (r->ev_rec[k]) cudaEventDestroy(r->ev_rec[k]);
    if (r->ev_adj[k]) cudaEventDestroy(r->ev_adj[k]);
  }
  if (r->ev_fork) cudaEventDestroy(r->ev_fork);
  if (r->ev_c19) cudaEventDestroy(r->ev_c19);
  if (r->side) {
    cudaStreamSynchronize(r->side);
    cudaStreamDestroy(r->side);
  }
  if (r->side2) {
    cudaStreamSynchronize(r->side2);
    cudaStreamDestroy(r->side2);
  }
  for (int k = 0; k < 2; ++k) {
    cudaFree(r->fb[k]);
    cudaFree(r->gb[k]);
  }
  cudaFree(r->scr);
  cudaFree(r->dTf);
  adj_drop_graphs(r);
  if (r->cap) cudaStreamDestroy(r->cap);
  delete r;
  c->adj = nullptr;
}

namespace {

int cst(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

long long face_nodes(const lbm_params& p, int face) {
  if (p.face_kind[face] == LBM_FACE_PERIODIC) return 0;
  const int n[3] = {p.nx, p.ny, p.nz};
  long long L = 1;
  for (int b = 0; b < 3; ++b)
    if (b != face / 2) L *= n[b];
  return L;
}

// state of the context (f, g of the current buffer, FP32) to / from a flat copy
int save_state(lbm_ctx* c, float* dst) {
  const size_t fb = 19ull * c->N * sizeof(float), gb = 7ull * c->N * sizeof(float);
  int st = cst(cudaMemcpyAsync(dst, c->f[c->cur], fb, cudaMemcpyDeviceToDevice, c->stream));
  if (!st) st = cst(cudaMemcpyAsync(dst + 19 * c->N, c->g[c->cur], gb, cudaMemcpyDeviceToDevice, c->stream));
  return st;
}

int load_state(lbm_ctx* c, const float* src) {
  const size_t fb = 19ull * c->N * sizeof(float), gb = 7ull * c->N * sizeof(float);
  int st = cst(cudaMemcpyAsync(c->f[c->cur], src, fb, cudaMemcpyDeviceToDevice, c->stream));
  if (!st) st = cst(cudaMemcpyAsync(c->g[c->cur], src + 19 * c->N, gb, cudaMemcpyDeviceToDevice, c->stream));
  return st;
}

int flags(lbm_ctx* c) {
  int e = 0;
  if (cudaMemcpyAsync(&e, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (e & ERRF_TIMEOUT) return LBM_ERR_TIMEOUT;
  if (e & ERRF_NONFINITE) return LBM_ERR_NONFINITE;
  if (e & ERRF_PSI) return LBM_ERR_PSI_DOMAIN;
  return LBM_OK;
}

// Recomputes len steps from the checkpoint ck: slot t receives state t and the
// scratch (rho, psi, F, u) the step computed from it.  The phase kernels write
// straight into the slots (the context's buffers are pointed at them).
// The launches go to `stream` (the context's stream is swapped for it meanwhile).
int recompute_steps(lbm_ctx* c, float* seg, int len, cudaStream_t stream) {
  const long long N = c->N;
  int st = LBM_OK;
  void* f0[2] = {c->f[0], c->f[1]};
  void* g0[2] = {c->g[0], c->g[1]};
  const Aux X0 = c->X;
  const int cur0 = c->cur;
  cudaStream_t s0 = c->stream;
  c->stream = stream;
  for (int t = 0; t < len && !st; ++t) {
    float* s = seg + (size_t)kSlot * N * t;
    float* s1 = s + (size_t)kSlot * N;
    c->f[c->cur] = s;
    c->g[c->cur] = s + 19 * N;
    c->f[1 - c->cur] = s1;
    c->g[1 - c->cur] = s1 + 19 * N;
    c->X = slot_aux(s, N, X0);
    st = lbm_step_phases_internal(c);
  }
  c->f[0] = f0[0];
  c->f[1] = f0[1];
  c->g[0] = g0[0];
  c->g[1] = g0[1];
  c->X = X0;
  c->cur = cur0;
  c->stream = s0;
  return st;
}

// With gx (full segments of the adjoint), the steps after the copy of the
// checkpoint are replayed from a graph, captured on first use.
int recompute(lbm_ctx* c, float* seg, const float* ck, int len, cudaStream_t stream, AdjRec* r = nullptr,
              cudaGraphExec_t* gx = nullptr) {
  int st = cst(cudaMemcpyAsync(seg, ck, 26ull * c->N * sizeof(float), cudaMemcpyDeviceToDevice, stream));
  if (st) return st;
  if (gx && !c->profiling &&
      (*gx || adj_capture(r, gx, [&](cudaStream_t cs) { return recompute_steps(c, seg, len, cs); })) &&
      cudaGraphLaunch(*gx, stream) == cudaSuccess)
    return LBM_OK;
  return recompute_steps(c, seg, len, stream);
}

// One adjoint step through the step from slot s:
// (fb1, gb1) = d L / d state(t+1) -> (fb0, gb0) = d L / d state(t).
int adjoint_one(lbm_ctx* c, AdjRec* r, float* s, float* fb1, float* gb1, float* fb0, float* gb0) {
  const Params& P = c->P;
  const long long N = c->N;
  const float* f = s;
  const float* g = s + 19 * N;
  const Aux X = slot_aux(s, N, c->X);
  cudaStream_t st = c->stream;
  const int B = blocks_for(N);
  float* q = r->scr;
  AdjAux A;
  A.Fb = q;
  A.Rb = q + 3 * N;
  A.Ub = q + 4 * N;
  A.Divb = q + 7 * N;
  A.Dpb = q + 8 * N;
  float* Jb = q + 9 * N;
  float* Tbar = q + 12 * N;  // d L / d T of the EOS chain
  // transposes, last forward operation first
  // the two lattices' transposes are independent: the D3Q19 chain (open-face
  // rule, collision) on a second stream, the D3Q7 chain (extrapolation,
  // relaxed streaming, collision) on the context stream
  cudaEventRecord(r->ev_fork, st);
  cudaStreamWaitEvent(r->side2, r->ev_fork, 0);
  DT6 d;
  for (int k = 0; k < 6; ++k) d.p[k] = r->face_off[k + 1] > r->face_off[k] ? r->dTf + r->face_off[k] : nullptr;
  if (P.bd_total > 0) {
    const int FB = (int)((P.bd_total + 63) / 64);
    k_adj_faces<1><<<FB, 64, 0, r->side2>>>(P, fb1, gb1, X, A.Fb, d);
    k_adj_faces<0><<<FB, 64, 0, st>>>(P, fb1, gb1, X, A.Fb, d);
  }
  // each lattice transpose overlaps the end of its face transpose
  const bool pf = r->pdl && P.bd_total > 0;
  cudaError_t e = launch_pdl(pf, k_adj_c19, B, kT, r->side2, P, f, (const float*)fb1, fb0, X, A.Fb);
  cudaEventRecord(r->ev_c19, r->side2);
  if (e == cudaSuccess) e = launch_pdl(pf, k_adj_c7, B, kT, st, P, g, (const float*)gb1, gb0, X, A);
  cudaStreamWaitEvent(st, r->ev_c19, 0);
  k_adj_u<<<B, kT, 0, st>>>(P, X, A, Jb);
  if (e == cudaSuccess) e = launch_pdl(r->pdl, k_adj_psi, B, kT, st, P, g, X, A, Tbar);
  if (e == cudaSuccess) e = launch_pdl(r->pdl, k_adj_fold, B, kT, st, P, A, (const float*)Jb, (const float*)Tbar, fb0, gb0);
  if (e != cudaSuccess) return LBM_ERR_CUDA;
  return cst(cudaGetLastError());
}

// Steps t = len-1 .. 0 of the segment in buffer seg, the newest adjoint in
// buffers cur, launched one by one on the context stream.
int adjoint_segment_eager(lbm_ctx* c, AdjRec* r, float* seg, int len, int cur) {
  int s = LBM_OK;
  for (int t = len - 1; t >= 0 && !s; --t) {
    s = adjoint_one(c, r, seg + (size_t)kSlot * c->N * t, r->fb[cur], r->gb[cur], r->fb[1 - cur], r->gb[1 - cur]);
    cur = 1 - cur;
  }
  return s;
}

// A full K-step segment from segment buffer b as one graph launch.  Returns
// false when the graph cannot be made; nothing has been launched then.
bool adjoint_segment_graph(lbm_ctx* c, AdjRec* r, int b, int cur) {
  if (!r->gx[b][cur] && !adj_capture(r, &r->gx[b][cur], [&](cudaStream_t cs) {
        cudaStream_t s0 = c->stream;
        c->stream = cs;
        const int e = adjoint_segment_eager(c, r, r->seg[b], r->K, cur);
        c->stream = s0;
        return e;
      }))
    return false;
  return cudaGraphLaunch(r->gx[b][cur], c->stream) == cudaSuccess;
}

}  // namespace

extern "C" int lbm_record(lbm_ctx* c, int n, int K) {
  if (!c || n < 0 || K < 1) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  if (c->hp.storage != LBM_STORE_F32 || c->hp.vartheta) return LBM_ERR_ARG;
  for (int f = 0; f < 6; ++f)
    if ((c->hp.face_kind[f] == LBM_FACE_WALL && c->hp.face_theta_deg[f] != 90.0) ||
        (c->hp.face_kind[f] == LBM_FACE_PERIODIC && c->hp.face_T_fixed[f]))
      return LBM_ERR_ARG;
  adj_free(c);
  AdjRec* r = new (std::nothrow) AdjRec();
  if (!r) return LBM_ERR_ARG;
  c->adj = r;
  r->K = K;
  r->N = c->N;
  const long long N = c->N;
  const int nck = n / K + 1;
  int st = LBM_OK;
  for (int k = 0; k < nck && !st; ++k) {
    float* p = nullptr;
    st = cst(cudaMalloc(&p, 26ull * N * sizeof(float)));
    if (!st) r->ckpt.push_back(p);
  }
  for (int k = 0; k < 6; ++k) r->face_off[k + 1] = r->face_off[k] + face_nodes(c->hp, k);
  const size_t slots = (size_t)std::min(K, std::max(n, 1)) + 1;
  if (!st) st = cst(cudaMalloc(&r->seg[0], (size_t)kSlot * N * sizeof(float) * slots));
  if (!st && n > K) {  // second segment buffer for the overlapped recompute, if it fits
    if (cudaMalloc(&r->seg[1], (size_t)kSlot * N * sizeof(float) * slots) != cudaSuccess) {
      r->seg[1] = nullptr;
      cudaGetLastError();
    }
  }
  if (!st) st = cst(cudaStreamCreateWithFlags(&r->side, cudaStreamNonBlocking));
  if (!st) st = cst(cudaStreamCreateWithFlags(&r->side2, cudaStreamNonBlocking));
  for (int k = 0; k < 2 && !st; ++k) {
    st = cst(cudaEventCreateWithFlags(&r->ev_rec[k], cudaEventDisableTiming));
    if (!st) st = cst(cudaEventCreateWithFlags(&r->ev_adj[k], cudaEventDisableTiming));
  }
  if (!st) st = cst(cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming));
  if (!st) st = cst(cudaEventCreateWithFlags(&r->ev_c19, cudaEventDisableTiming));
  for (int k = 0; k < 2 && !st; ++k) {
    st = cst(cudaMalloc(&r->fb[k], 19ull * N * sizeof(float)));
    if (!st) st = cst(cudaMalloc(&r->gb[k], 7ull * N * sizeof(float)));
  }
  if (!st) st = cst(cudaMalloc(&r->scr, 13ull * N * sizeof(float)));
  if (!st) st = cst(cudaMalloc(&r->fin, 26ull * N * sizeof(float)));
  if (!st) st = cst(cudaMalloc(&r->dTf, sizeof(double) * std::max(1LL, r->face_off[6])));
  // forward run, a checkpoint every K steps; the last segment's steps are
  // computed into the recompute slots, where the adjoint starts
  const int nseg = (n + K - 1) / K;
  const int tlast = nseg > 0 ? (nseg - 1) * K : 0;
  int done = 0;
  if (!st) st = save_state(c, r->ckpt[0]);
  while (!st && done < tlast) {
    st = lbm_step(c, K);
    done += K;
    if (!st && done / K < nck) st = save_state(c, r->ckpt[done / K]);
  }
  if (!st && n > tlast) {
    const int len = n - tlast;
    st = recompute(c, r->seg[0], r->ckpt[tlast / K], len, c->stream);
    // the state after the last step is slot len: make it current
    if (!st) st = load_state(c, r->seg[0] + (size_t)kSlot * N * len);
    if (!st && n % K == 0 && n / K < nck) st = save_state(c, r->ckpt[n / K]);
    r->last_kept = !st;
  }
  if (!st) st = save_state(c, r->fin);
  if (!st) st = flags(c);
  if (st) {
    adj_free(c);
    return st;
  }
  r->nrec = n;
  return LBM_OK;
}

extern "C" int lbm_adjoint_step(lbm_ctx* c, int n, const float* dL_drho, const float* dL_dT, double* dL_dTface,
                                double* dL_dT0) {
  if (!c) return LBM_ERR_ARG;
  AdjRec* r = c->adj;
  if (!r || n != r->nrec) return LBM_ERR_STATE;
  const long long N = c->N;
  cudaStream_t st = c->stream;
  int s = cst(cudaMemsetAsync(r->dTf, 0, sizeof(double) * std::max(1LL, r->face_off[6]), st));
  int cur = 0;  // adjoint of the newest state in fb[cur], gb[cur]
  k_adj_seed<<<blocks_for(N), kT, 0, st>>>(c->P, dL_drho, dL_dT, r->fb[0], r->gb[0]);
  const int K = r->K;
  const int nseg = (n + K - 1) / K;
  // Segment k is reversed from buffer set[k]; while it is, segment k-1 is
  // recomputed into the other buffer on the side stream (when there is one).
  const bool two = r->seg[1] != nullptr;
  // for comparison: LBM_ADJ_EAGER launches every step on its own, LBM_ADJ_NOPDL
  // launches the kernels of a step without programmatic dependencies
  const bool graphs = std::getenv("LBM_ADJ_EAGER") == nullptr;
  r->pdl = std::getenv("LBM_ADJ_NOPDL") == nullptr;
  if (graphs) adj_graph_key(c, r);
  auto set_of = [&](int k) { return two ? (nseg - 1 - k) & 1 : 0; };
  auto launch_recompute = [&](int k) {
    const int b = set_of(k);
    if (two) cudaStreamWaitEvent(r->side, r->ev_adj[b], 0);  // its previous user is done
    else cudaStreamWaitEvent(r->side, r->ev_adj[0], 0);
    const int len = std::min(K, n - k * K);
    int e = recompute(c, r->seg[b], r->ckpt[k], len, r->side, r, graphs && len == K ? &r->gr[b] : nullptr);
    if (!e) e = cst(cudaEventRecord(r->ev_rec[b], r->side));
    return e;
  };
  for (int b = 0; b < 2 && !s; ++b) s = cst(cudaEventRecord(r->ev_adj[b], st));
  if (nseg > 0 && !s && !r->last_kept) s = launch_recompute(nseg - 1);
  const bool last_was_kept = r->last_kept;
  for (int k = nseg - 1; k >= 0 && !s; --k) {
    const int t0 = k * K, len = std::min(K, n - t0), b = set_of(k);
    if (!(k == nseg - 1 && last_was_kept)) s = cst(cudaStreamWaitEvent(st, r->ev_rec[b], 0));
    if (!s && k > 0 && two) s = launch_recompute(k - 1);  // overlapped with this segment
    if (!(len == K && graphs && adjoint_segment_graph(c, r, b, cur)))
      s = adjoint_segment_eager(c, r, r->seg[b], len, cur);
    if (len & 1) cur = 1 - cur;
    if (!s) s = cst(cudaEventRecord(r->ev_adj[b], st));
    if (!s && k > 0 && !two) s = launch_recompute(k - 1);  // serial: after this segment
  }
  if (nseg > 1) r->last_kept = false;
  // the side streams' work is done before the stream continues
  if (!s) s = cst(cudaEventRecord(r->ev_rec[0], r->side));
  if (!s) s = cst(cudaStreamWaitEvent(st, r->ev_rec[0], 0));
  // leave the recorded final state current
  if (!s) s = load_state(c, r->fin);
  if (!s && dL_dT0) k_adj_T0<<<blocks_for(N), kT, 0, st>>>(c->P, r->gb[cur], dL_dT0);
  if (!s && dL_dTface && r->face_off[6] > 0)
    s = cst(cudaMemcpyAsync(dL_dTface, r->dTf, sizeof(double) * r->face_off[6], cudaMemcpyDeviceToDevice, st));
  if (!s) s = cst(cudaGetLastError());
  if (!s) s = flags(c);
  r->cur = cur;
  return s;
}

extern "C" int lbm_adjoint_state(lbm_ctx* c, float* f_bar, float* g_bar, int mem) {
  if (!c) return LBM_ERR_ARG;
  AdjRec* r = c->adj;
  if (!r) return LBM_ERR_STATE;
  const cudaMemcpyKind kd = mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  int s = LBM_OK;
  if (f_bar) s = cst(cudaMemcpyAsync(f_bar, r->fb[r->cur], 19ull * c->N * sizeof(float), kd, c->stream));
  if (!s && g_bar) s = cst(cudaMemcpyAsync(g_bar, r->gb[r->cur], 7ull * c->N * sizeof(float), kd, c->stream));
  if (!s) s = cst(cudaStreamSynchronize(c->stream));
  return s;
}
