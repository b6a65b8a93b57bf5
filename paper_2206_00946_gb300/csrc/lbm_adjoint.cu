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
#include <cstring>
#include <new>
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

// adjoint scratch fields, N floats each unless noted
struct AdjAux {
  float *Fb;     // 3N: d L / d F
  float *Rb;     // d L / d rho (partial)
  float *Ub;     // 3N: d L / d u from the D3Q7 collision at the cell itself
  float *Divb;   // d L / d (div u)
  float *Dpb;    // d L / d (dp/dT)
  float *gstar;  // 7N: post-collision D3Q7 populations of the recomputed step
};

// ---------------------------------------------------------------- forward --
__global__ void k_adj_A(Params P, const float* f, const float* g, Aux X, int* err) {
  int e = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x)
    phaseA<float>(P, c, f, g, X, nullptr, e, true);
  if (e) atomicOr(err, e);
}

__global__ void k_adj_B(Params P, Aux X) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) phaseB(P, c, X);
}

// g* of every cell (the D3Q7 collision of phaseC7_cell without the streaming)
__global__ void k_adj_gstar(Params P, const float* g, Aux X, float* gstar) {
  const Hint h = make_hint();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    Nb nb;
    make_nb(P, x, y, z, nb);
    float gl[7];
    for (int i = 0; i < 7; ++i) gl[i] = g[i * P.N + c];
    const float rho = X.rho[c], T = sum7(gl);
    const float du = divu_at(P, c, nb, X, h);
    float p, dpdT, gs[7];
    eos_pr(P, rho, T, p, dpdT);
    collide7(P, gl, rho, T, X.ux[c], X.uy[c], X.uz[c], du, dpdT, gs);
    for (int i = 0; i < 7; ++i) gstar[i * P.N + c] = gs[i];
  }
}

__global__ void k_adj_seed(Params P, const float* rhob, const float* Tb, float* fb, float* gb) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    const float r = rhob ? rhob[c] : 0.f, t = Tb ? Tb[c] : 0.f;
    for (int i = 0; i < 19; ++i) fb[i * P.N + c] = r;
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

__global__ void k_adj_faces(Params P, float* fb, float* gb, Aux X, float* Fb, DT6 dTf) {
  const long long N = P.N;
  const float w0 = 1.f - P.wbar, w1 = P.wbar * (1.f / 6.f);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)P.bd_total; k += gridDim.x * blockDim.x) {
    int x, y, z;
    boundary_candidate(P, k, x, y, z);
    const int m = node_faces(P, x, y, z);
    if (!m) continue;
    const int c = cell_of(P, x, y, z);
    int nnp = 0, nopen = 0, oface = -1, q[3] = {x, y, z};
    for (int fc = 0; fc < 6; ++fc) {
      if (!((m >> fc) & 1)) continue;
      ++nnp;
      if (P.face_kind[fc] == FACE_OPEN) {
        ++nopen;
        oface = fc;
      }
      q[fc >> 1] += (fc & 1) ? -1 : 1;
    }
    // extrapolation: g_k(x_b) = w_k T_b + g_k(x_f) - w_k sum_j g_j(x_f)
    float a[7], Tb = 0.f;
    for (int i = 0; i < 7; ++i) {
      a[i] = gb[i * N + c];
      gb[i * N + c] = 0.f;
      Tb += (i == 0 ? w0 : w1) * a[i];
    }
    const int cf = cell_of(P, q[0], q[1], q[2]);
    for (int i = 0; i < 7; ++i) atomicAdd(gb + i * N + cf, a[i] - Tb);
    for (int fc = 0; fc < 6; ++fc) {
      if (!((m >> fc) & 1)) continue;
      const int ax = fc >> 1;
      const int idx = ax == 0 ? y + P.ny * z : (ax == 1 ? x + P.nx * z : x + P.nx * y);
      dTf.p[fc][idx] += (double)Tb / nnp;  // one (face, node) entry per thread
    }
    if (nopen) {
      const unsigned unk = unknown19(P, x, y, z);
      float fl[19];
      for (int i = 0; i < 19; ++i) fl[i] = fb[i * N + c];
      if (nnp == 1) {
        float F3[3] = {0.f, 0.f, 0.f};
        zouhe_vjp(oface, P.face_rho[oface], fl, F3);
        Fb[c] += F3[0];
        Fb[N + c] += F3[1];
        Fb[2 * N + c] += F3[2];
      } else {
        for (int i = 1; i < 19; ++i)
          if ((unk >> i) & 1u) fl[i] = 0.f;  // f^eq(rho_b, 0): constant
      }
      for (int i = 0; i < 19; ++i) fb[i * N + c] = fl[i];
    }
  }
}

// ------------------------------------------------------- D3Q19 transpose ----
// d L / d f*(x) gathered from the slots the push wrote (bounce-back included),
// then the collision's vector-Jacobian product.
__global__ void k_adj_c19(Params P, const float* f, const float* fb1, float* fb0, Aux X, float* Fb) {
  const long long N = P.N;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    float fl[19], fsb[19], fbo[19], F3[3] = {X.Fx[c], X.Fy[c], X.Fz[c]}, Fo[3];
    for (int i = 0; i < 19; ++i) {
      fl[i] = f[i * N + c];
      const long long d = dest19(P, x, y, z, i);
      fsb[i] = d < 0 ? 0.f : fb1[d];
    }
    const int m = P.any_nonperiodic ? node_faces(P, x, y, z) : 0;
    const bool wall = m && on_wall(P, m);
    collide19_vjp(P, fl, !(wall && P.wall_ueq_zero), F3, fsb, fbo, Fo);
    for (int i = 0; i < 19; ++i) fb0[i * N + c] = fbo[i];
    Fb[c] += Fo[0];
    Fb[N + c] += Fo[1];
    Fb[2 * N + c] += Fo[2];
  }
}

// -------------------------------------------------------- D3Q7 transpose ----
// Relaxed streaming g'_i(y) = g_i(y) + (g*_i(y - c_i) - g_i(y)) / (rho(y) c_v)
// transposed at x both as a source (d L / d g*) and as a destination (the
// retained g_i(x) and rho(x) c_v), then the D3Q7 collision's product.
__global__ void k_adj_c7(Params P, const float* g, const float* gb1, float* gb0, Aux X, AdjAux A) {
  const long long N = P.N;
  const Hint h = make_hint();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    Nb nb;
    make_nb(P, x, y, z, nb);
    float gl[7], gsb[7], gout[7];
    for (int i = 0; i < 7; ++i) gl[i] = g[i * N + c];
    const float rho = X.rho[c], T = sum7(gl);
    const float beta = 1.f / (rho * P.cv);
    float rhob = 0.f;
    for (int i = 0; i < 7; ++i) {
      const float a = gb1[i * N + c];
      // as a source: population i goes to y = x + c_i
      const int yd = dest7_cell(P, x, y, z, i);
      gsb[i] = yd < 0 ? 0.f : gb1[i * N + yd] / (X.rho[yd] * P.cv);
      // as a destination: the source x - c_i
      const int s = dest7_cell(P, x, y, z, i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1));
      if (s < 0) {
        gout[i] = a;
      } else {
        gout[i] = (1.f - beta) * a;
        rhob -= a * (A.gstar[i * N + s] - gl[i]) * beta / rho;
      }
    }
    const float du = divu_at(P, c, nb, X, h);
    float p, dpdT;
    eos_pr(P, rho, T, p, dpdT);
    const float u3[3] = {X.ux[c], X.uy[c], X.uz[c]};
    float gbv[7], rb7, Tb, ub[3], divb, dpb;
    collide7_vjp(P, gl, rho, T, u3, du, dpdT, gsb, gbv, rb7, Tb, ub, divb, dpb);
    for (int i = 0; i < 7; ++i) gb0[i * N + c] = gout[i] + gbv[i] + Tb;
    A.Rb[c] = rhob + rb7;
    A.Ub[c] = ub[0];
    A.Ub[N + c] = ub[1];
    A.Ub[2 * N + c] = ub[2];
    A.Divb[c] = divb;
    A.Dpb[c] = dpb;
  }
}

// Per-axis preimages under the ghost rule of a stencil: the coordinates x_a
// whose move by c lands on ya.  mode 0 (psi): open faces copy the boundary
// node, walls mirror through the wall layer; mode 1 (velocity): open faces
// copy, moves across a wall contribute nothing.  Periodic faces wrap.
__device__ __forceinline__ int preimage_axis(const Params& P, int a, int ya, int c, int mode, int* xs) {
  if (c == 0) {
    xs[0] = ya;
    return 1;
  }
  const int n = dim_of(P, a);
  const bool per = P.face_kind[2 * a] == FACE_PERIODIC;
  int cnt = 0;
  const int s = ya - c;
  if (s >= 0 && s < n) xs[cnt++] = s;
  else if (per) xs[cnt++] = wrapi(s, n);
  if (!per) {
    const int b = c > 0 ? n - 1 : 0;  // the boundary coordinate a move by c leaves from
    const int kind = P.face_kind[2 * a + (c > 0 ? 1 : 0)];
    if (kind == FACE_OPEN && ya == b) xs[cnt++] = b;
    if (kind == FACE_WALL && mode == 0 && ya == b - c) xs[cnt++] = b;
  }
  return cnt;
}

// --------------------------------------- velocity, force and EOS transposes --
// d L / d u(y) = the D3Q7 collision's own term + the div u stencil transposed,
// then u = (j + F/2) / rho (zero at walls): d L / d j, d L / d F, d L / d rho.
__global__ void k_adj_u(Params P, Aux X, AdjAux A, float* Jb) {
  const long long N = P.N;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int q[3];
    cell_xyz(P, c, q[0], q[1], q[2]);
    float ub[3] = {A.Ub[c], A.Ub[N + c], A.Ub[2 * N + c]};
    for (int i = 1; i < 19; ++i) {
      const int ci[3] = {c19x(i), c19y(i), c19z(i)};
      int xs[3][2], cn[3];
      for (int a = 0; a < 3; ++a) cn[a] = preimage_axis(P, a, q[a], ci[a], 1, xs[a]);
      float s = 0.f;
      for (int i0 = 0; i0 < cn[0]; ++i0)
        for (int i1 = 0; i1 < cn[1]; ++i1)
          for (int i2 = 0; i2 < cn[2]; ++i2) s += A.Divb[cell_of(P, xs[0][i0], xs[1][i1], xs[2][i2])];
      const float k = 3.f * w19(i) * s;
      ub[0] += ci[0] * k;
      ub[1] += ci[1] * k;
      ub[2] += ci[2] * k;
    }
    const int m = P.any_nonperiodic ? node_faces(P, q[0], q[1], q[2]) : 0;
    float j3[3] = {0.f, 0.f, 0.f};
    if (!(m && on_wall(P, m))) {
      const float rho = X.rho[c], ir = 1.f / rho;
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

// d L / d psi(y) from F(x) = -G psi(x) sum_i varpi_i psi(x + c_i) c_i (own and
// transposed stencil terms), the EOS chain rule to rho and T, and the
// macroscopic fields rho = sum f, j = sum c f, T = sum g folded into the
// adjoint of the populations at time t.
__global__ void k_adj_psi(Params P, const float* f, const float* g, Aux X, AdjAux A, const float* Jb, float* fb0,
                          float* gb0) {
  const long long N = P.N;
  const Hint h = make_hint();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)N; c += gridDim.x * blockDim.x) {
    int q[3];
    cell_xyz(P, c, q[0], q[1], q[2]);
    Nb nb;
    make_nb(P, q[0], q[1], q[2], nb);
    const float psi = X.psi[c];
    float S[3] = {0.f, 0.f, 0.f};
    float psib = 0.f;
    for (int i = 1; i < 19; ++i) {
      const int ci[3] = {c19x(i), c19y(i), c19z(i)};
      const float v = varpi19(i) * ld_aux(X.psi + c + nb_off_psi(nb, ci[0], ci[1], ci[2]), h);
      S[0] += ci[0] * v;
      S[1] += ci[1] * v;
      S[2] += ci[2] * v;
      int xs[3][2], cn[3];
      for (int a = 0; a < 3; ++a) cn[a] = preimage_axis(P, a, q[a], ci[a], 0, xs[a]);
      for (int i0 = 0; i0 < cn[0]; ++i0)
        for (int i1 = 0; i1 < cn[1]; ++i1)
          for (int i2 = 0; i2 < cn[2]; ++i2) {
            const int x = cell_of(P, xs[0][i0], xs[1][i1], xs[2][i2]);
            psib += -P.G * X.psi[x] * varpi19(i) *
                    (ci[0] * A.Fb[x] + ci[1] * A.Fb[N + x] + ci[2] * A.Fb[2 * N + x]);
          }
    }
    psib += -P.G * (A.Fb[c] * S[0] + A.Fb[N + c] * S[1] + A.Fb[2 * N + c] * S[2]);
    float gl[7];
    for (int i = 0; i < 7; ++i) gl[i] = g[i * N + c];
    const float rho = X.rho[c], T = sum7(gl);
    float rhob = A.Rb[c], Tb = 0.f;
    psi_dpdT_vjp(P, rho, T, psi, psib, A.Dpb[c], rhob, Tb);
    const float jx = Jb[c], jy = Jb[N + c], jz = Jb[2 * N + c];
    for (int i = 0; i < 19; ++i) fb0[i * N + c] += rhob + c19x(i) * jx + c19y(i) * jy + c19z(i) * jz;
    for (int i = 0; i < 7; ++i) gb0[i * N + c] += Tb;
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
  long long N = 0;
  std::vector<float*> ckpt;  // f (19N) + g (7N) at steps 0, K, 2K, ...
  float* seg = nullptr;      // the K states of the segment being reversed
  float* fb[2] = {nullptr, nullptr};
  float* gb[2] = {nullptr, nullptr};
  float* scr = nullptr;      // AdjAux fields + Jb
  double* dTf = nullptr;     // per-face accumulators, faces concatenated
  long long face_off[7] = {0, 0, 0, 0, 0, 0, 0};
};

void adj_free(lbm_ctx* c) {
  if (!c || !c->adj) return;
  AdjRec* r = c->adj;
  for (float* p : r->ckpt) cudaFree(p);
  cudaFree(r->seg);
  for (int k = 0; k < 2; ++k) {
    cudaFree(r->fb[k]);
    cudaFree(r->gb[k]);
  }
  cudaFree(r->scr);
  cudaFree(r->dTf);
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

// One adjoint step through the step from state s (f = s, g = s + 19N):
// (fb1, gb1) = d L / d state(t+1) -> (fb0, gb0) = d L / d state(t).
int adjoint_one(lbm_ctx* c, AdjRec* r, const float* s, float* fb1, float* gb1, float* fb0, float* gb0) {
  const Params& P = c->P;
  const long long N = c->N;
  const float* f = s;
  const float* g = s + 19 * N;
  cudaStream_t st = c->stream;
  const int B = blocks_for(N);
  float* q = r->scr;
  AdjAux A;
  A.Fb = q;
  A.Rb = q + 3 * N;
  A.Ub = q + 4 * N;
  A.Divb = q + 7 * N;
  A.Dpb = q + 8 * N;
  A.gstar = q + 9 * N;
  float* Jb = q + 16 * N;
  // forward quantities of step t
  k_adj_A<<<B, kT, 0, st>>>(P, f, g, c->X, c->err_d);
  k_adj_B<<<B, kT, 0, st>>>(P, c->X);
  k_adj_gstar<<<B, kT, 0, st>>>(P, g, c->X, A.gstar);
  if (cudaMemsetAsync(A.Fb, 0, 3 * N * sizeof(float), st) != cudaSuccess) return LBM_ERR_CUDA;
  // transposes, last forward operation first
  if (P.bd_total > 0) {
    DT6 d;
    for (int k = 0; k < 6; ++k) d.p[k] = r->face_off[k + 1] > r->face_off[k] ? r->dTf + r->face_off[k] : nullptr;
    k_adj_faces<<<blocks_for(P.bd_total), kT, 0, st>>>(P, fb1, gb1, c->X, A.Fb, d);
  }
  k_adj_c19<<<B, kT, 0, st>>>(P, f, fb1, fb0, c->X, A.Fb);
  k_adj_c7<<<B, kT, 0, st>>>(P, g, gb1, gb0, c->X, A);
  k_adj_u<<<B, kT, 0, st>>>(P, c->X, A, Jb);
  k_adj_psi<<<B, kT, 0, st>>>(P, f, g, c->X, A, Jb, fb0, gb0);
  return cst(cudaGetLastError());
}

}  // namespace

extern "C" int lbm_record(lbm_ctx* c, int n, int K) {
  if (!c || n < 0 || K < 1) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  if (c->hp.storage != LBM_STORE_F32 || c->hp.vartheta) return LBM_ERR_ARG;
  for (int f = 0; f < 6; ++f)
    if (c->hp.face_kind[f] == LBM_FACE_WALL && c->hp.face_theta_deg[f] != 90.0) return LBM_ERR_ARG;
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
  if (!st) st = cst(cudaMalloc(&r->seg, 26ull * N * sizeof(float) * (size_t)std::min(K, std::max(n, 1))));
  for (int k = 0; k < 2 && !st; ++k) {
    st = cst(cudaMalloc(&r->fb[k], 19ull * N * sizeof(float)));
    if (!st) st = cst(cudaMalloc(&r->gb[k], 7ull * N * sizeof(float)));
  }
  if (!st) st = cst(cudaMalloc(&r->scr, 19ull * N * sizeof(float)));
  if (!st) st = cst(cudaMalloc(&r->dTf, sizeof(double) * std::max(1LL, r->face_off[6])));
  // forward run, a checkpoint every K steps
  int done = 0;
  if (!st) st = save_state(c, r->ckpt[0]);
  while (!st && done < n) {
    const int len = std::min(K, n - done);
    st = lbm_step(c, len);
    done += len;
    if (!st && done % K == 0 && done / K < nck) st = save_state(c, r->ckpt[done / K]);
  }
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
  for (int k = nseg - 1; k >= 0 && !s; --k) {
    const int t0 = k * K, len = std::min(K, n - t0);
    // recompute the segment's states from its checkpoint
    s = load_state(c, r->ckpt[k]);
    for (int t = 0; t < len && !s; ++t) {
      s = save_state(c, r->seg + 26 * N * t);
      if (!s && t + 1 < len) s = lbm_step(c, 1);
    }
    for (int t = len - 1; t >= 0 && !s; --t) {
      s = adjoint_one(c, r, r->seg + 26 * N * t, r->fb[cur], r->gb[cur], r->fb[1 - cur], r->gb[1 - cur]);
      cur = 1 - cur;
    }
  }
  // leave the recorded final state current
  if (!s) s = load_state(c, r->ckpt.back());
  if (!s && n % K != 0) s = lbm_step(c, n % K);
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
