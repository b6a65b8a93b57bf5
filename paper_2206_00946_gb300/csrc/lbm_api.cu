// C ABI of liblbm (declared in include/lbm.h): context management, launches
// of the step kernels on the caller's stream, FP64 reductions, host helpers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_fused.cuh"
#include "lbm_phases.cuh"
#include "lbm_stage.cuh"
#include "lbm_ctx.cuh"

using namespace lbm;

namespace {

constexpr int kThreads = 256;
#ifndef LBM_PHASEC_MINBLOCKS
#define LBM_PHASEC_MINBLOCKS 4
#endif

// ref: the per-cell references of buffer 0 (storage with per-cell references only):
// the initial rho0 and T0 themselves
template <typename T>
__global__ void k_init(Params P, const float* __restrict__ rho0, const float* __restrict__ T0, T* f, T* g,
                       float2* ref) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    float fe[19];
    const float r = rho0[c], Tc = T0[c];
    if (LocalRef<T>::on) ref[c] = make_float2(r, Tc);
    feq19(r, 0.f, 0.f, 0.f, fe);
#pragma unroll
    for (int i = 0; i < 19; ++i) PopStore<T>::st(f + i * P.N + c, fe[i], fbase_at<T>(P, i, r));
    PopStore<T>::st(g + c, (1.f - P.wbar) * Tc, gbase_at<T>(P, 0, Tc));
#pragma unroll
    for (int i = 1; i < 7; ++i) PopStore<T>::st(g + i * P.N + c, P.wbar * (1.f / 6.f) * Tc, gbase_at<T>(P, i, Tc));
  }
}

// per-cell references of a state given in FP32: component `comp` (0: rho = sum f,
// 1: T = sum g) of ref[c] from the q populations in src
__global__ void k_ref_sum(Params P, const float* __restrict__ src, int q, float2* ref, int comp) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < q; ++i) s += src[i * P.N + c];
    if (comp == 0)
      ref[c].x = s;
    else
      ref[c].y = s;
  }
}

// float populations (state exchanged with the caller) <-> storage, q directions
// (ref: the per-cell references of the buffer, storage with per-cell references only)
template <typename T>
__device__ __forceinline__ float state_base(const Params& P, const float2* ref, long long k, int is_g) {
  const int i = (int)(k / P.N);
  const float2 r = LocalRef<T>::on ? ref[k - (long long)i * P.N] : make_float2(0.f, 0.f);
  return is_g ? gbase_at<T>(P, i, r.y) : fbase_at<T>(P, i, r.x);
}

template <typename T>
__global__ void k_store(Params P, const float* __restrict__ src, T* dst, int q, int is_g, const float2* ref) {
  const long long n = (long long)q * P.N;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    PopStore<T>::st(dst + k, src[k], state_base<T>(P, ref, k, is_g));
}

template <typename T>
__global__ void k_load(Params P, const T* __restrict__ src, float* dst, int q, int is_g, const float2* ref) {
  const long long n = (long long)q * P.N;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    dst[k] = PopStore<T>::ld_plain(src + k, state_base<T>(P, ref, k, is_g));
}

// Phase kernels over the cell range [c0, c1) (whole planes) with grid-stride loops.
// write_j: store j for phase B (only lbm_macros runs phase B on its own).
// FUSE_D: also the face rules of the step that wrote the state (see phaseA)
template <typename T, bool FUSE_D = false>
__global__ void k_phaseA(Params P, const T* f, const T* g, AuxFor<T> X, float* Tout, int* err, int c0, int c1,
                         int write_j) {
  int e = 0;
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x)
    phaseA<T, FUSE_D>(P, c, f, g, X, Tout, e, write_j != 0);
  if (e) atomicOr(err, e);
}

int grid_for(long long n);

// phase A of the cell pairs of [c0, c1) (c0 and c1 even), one global 16-bit shift
template <typename T>
__global__ void k_phaseA2(Params P, const T* f, const T* g, AuxFor<T> X, int* err, int c0, int c1) {
  int e = 0;
  for (int c = c0 + 2 * (blockIdx.x * blockDim.x + threadIdx.x); c < c1; c += 2 * gridDim.x * blockDim.x)
    phaseA2<T>(P, c, f, g, X, e);
  if (e) atomicOr(err, e);
}

// phase A of [c0, c1) in a step: two cells per thread for the global 16-bit shifts when the
// planes have an even number of cells (every range then starts and ends on a pair)
template <typename T>
void launch_phaseA(const lbm_ctx* c, const AuxFor<T>& X, int blocks, cudaStream_t st, const T* f, const T* g, int c0,
                   int c1) {
  if constexpr (sizeof(T) == 2 && !LocalRef<T>::on) {
    if ((c->P.nx * c->P.ny) % 2 == 0) {
      const int grid = std::max(1, std::min(blocks, grid_for((long long)(c1 - c0) / 2)));
      k_phaseA2<T><<<grid, kThreads, 0, st>>>(c->P, f, g, X, c->err_d, c0, c1);
      return;
    }
  }
  k_phaseA<T><<<blocks, kThreads, 0, st>>>(c->P, f, g, X, nullptr, c->err_d, c0, c1, 0);
}

__global__ void k_phaseB(Params P, Aux X, int c0, int c1) {
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x) phaseB(P, c, X);
}

template <typename T>
__global__ void __launch_bounds__(256, LBM_PHASEC_MINBLOCKS) k_phaseC19(Params P, const T* __restrict__ fA, T* fB,
                                                                        AuxFor<T> X, int c0, int c1) {
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x)
    phaseC19(P, c, fA, fB, X);
}

// force, velocity and the D3Q19 collision + push in one pass (phases B and C19)
template <typename T>
__global__ void __launch_bounds__(256, LBM_PHASEC_MINBLOCKS) k_phaseBC19(Params P, const T* __restrict__ fA, T* fB,
                                                                         AuxFor<T> X, int c0, int c1) {
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x)
    phaseBC19(P, c, fA, fB, X);
}

// CTAs of a staged launch over ntiles tiles: `per` tiles each, but never fewer than the
// launch's share of four CTAs per SM among the slab launches that run at once (all of them
// for the phase schedule's single launch), and at most four per SM.
int staged_grid(const lbm_ctx* c, int ntiles, int per) {
  const int slots = 152 * 4;
  const int conc = c->slabs ? std::max(1, std::min(c->slabs->nslab, c->slabs->nstreams)) : 1;
  const int g = std::max((ntiles + per - 1) / per, slots / conc);
  return std::max(1, std::min(std::min(g, ntiles), slots));
}

// Force + D3Q19 over [c0, c1): with staged populations (k_phaseBC19_staged, stage19 tiles per
// CTA, at most four CTAs per SM) when the context allows it, else one cell per thread.
template <typename T>
void launch_bc19(const lbm_ctx* c, const AuxFor<T>& X, int blocks, cudaStream_t st, const T* fA, T* fB, int c0,
                 int c1) {
  if constexpr (std::is_same<T, float>::value) {
    if (c->stage19 > 0) {
      const int ntiles = (c1 - c0) / kStageT;
      const int grid = staged_grid(c, ntiles, c->stage19);
      const size_t smem = 2 * 19 * kStageT * sizeof(T) + 16;
      k_phaseBC19_staged<T><<<grid, kStageT, smem, st>>>(c->P, fA, fB, X, c0, c1, c->err_d);
      return;
    }
  }
  k_phaseBC19<T><<<blocks, kThreads, 0, st>>>(c->P, fA, fB, X, c0, c1);
}

// VT: vartheta of the context (a separate instantiation each, launched by launch_c7)
template <typename T, int VT>
__global__ void __launch_bounds__(256, 4) k_phaseC7(Params P, const T* __restrict__ gA, T* gB, AuxFor<T> X, int c0,
                                                    int c1) {
  for (int c = c0 + blockIdx.x * blockDim.x + threadIdx.x; c < c1; c += gridDim.x * blockDim.x)
    phaseC7<T, VT>(P, c, gA, gB, X);
}

template <typename T>
void launch_c7(const lbm_ctx* c, const AuxFor<T>& X, int blocks, cudaStream_t st, const T* gA, T* gB, int c0, int c1) {
  if constexpr (std::is_same<T, float>::value) {
    if (c->stage7 > 0) {
      const int ntiles = (c1 - c0) / kStageT;
      const int grid = staged_grid(c, ntiles, c->stage7);
      const size_t smem = 2 * 7 * kStageT * sizeof(T) + 16;
      if (c->P.vartheta)
        k_phaseC7_staged<T, 1><<<grid, kStageT, smem, st>>>(c->P, gA, gB, X, c0, c1, c->err_d);
      else
        k_phaseC7_staged<T, 0><<<grid, kStageT, smem, st>>>(c->P, gA, gB, X, c0, c1, c->err_d);
      return;
    }
  }
  if (c->P.vartheta)
    k_phaseC7<T, 1><<<blocks, kThreads, 0, st>>>(c->P, gA, gB, X, c0, c1);
  else
    k_phaseC7<T, 0><<<blocks, kThreads, 0, st>>>(c->P, gA, gB, X, c0, c1);
}

// one thread per boundary candidate (boundary_candidate enumerates them)
template <typename T>
__global__ void __launch_bounds__(256, 3) k_phaseD(Params P, T* fB, T* gB, AuxFor<T> X) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (int)P.bd_total; k += gridDim.x * blockDim.x) {
    int x, y, z;
    boundary_candidate(P, k, x, y, z);
    const int m = node_tfaces(P, x, y, z);
    if (m) phaseD(P, cell_of(P, x, y, z), x, y, z, m, fB, gB, X);
  }
}

// boundary nodes of planes z0 + blockIdx.y
template <typename T>
__global__ void __launch_bounds__(256, 3) k_phaseD_planes(Params P, T* fB, T* gB, AuxFor<T> X, int z0) {
  const int z = z0 + blockIdx.y;
  const int cnt = boundary_count(P, z);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    int x, y;
    boundary_xy(P, z, k, x, y);
    const int m = node_tfaces(P, x, y, z);
    if (m) phaseD(P, cell_of(P, x, y, z), x, y, z, m, fB, gB, X);
  }
}

// FP64 block reduction: mass, sum rho cv T, droplet volume, non-finite count.
template <typename S>
__global__ void k_reduce(Params P, const S* __restrict__ f, const S* __restrict__ g, double* partial,
                         const float2* ref) {
  double a[4] = {0, 0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    const float2 r = LocalRef<S>::on ? ref[c] : make_float2(0.f, 0.f);
    float fl[19], gl[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = PopStore<S>::ld_plain(f + i * P.N + c, fbase_at<S>(P, i, r.x));
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = PopStore<S>::ld_plain(g + i * P.N + c, gbase_at<S>(P, i, r.y));
    float rho, jx, jy, jz;
    sum19(fl, rho, jx, jy, jz);
    const float T = sum7(gl);
    bool fin = isfinite(rho) && isfinite(T);
#pragma unroll
    for (int i = 0; i < 19; ++i) fin = fin && isfinite(fl[i]);
#pragma unroll
    for (int i = 0; i < 7; ++i) fin = fin && isfinite(gl[i]);
    if (fin) {
      a[0] += (double)rho;
      a[1] += (double)rho * (double)P.cv * (double)T;
      double phi = ((double)rho - (double)P.rho_v) * (double)P.inv_drho;
      a[2] += phi < 0 ? 0.0 : (phi > 1 ? 1.0 : phi);
    } else {
      a[3] += 1.0;
    }
  }
  __shared__ double sh[4][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = a[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    partial[blockIdx.x * 4 + threadIdx.x] = v;
  }
}

// Sums the per-block partials in a fixed order (deterministic result).
__global__ void k_reduce_final(const double* partial, int nblocks, double* out) {
  if (threadIdx.x < 4) {
    double v = 0;
    for (int b = 0; b < nblocks; ++b) v += partial[b * 4 + threadIdx.x];
    out[threadIdx.x] = v;
  }
}

__global__ void k_maps(Params P, int* map19, int* map7, unsigned char* cls) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    if (cls) cls[c] = (unsigned char)node_faces(P, x, y, z);
    if (map19)
      for (int i = 0; i < 19; ++i) map19[i * P.N + c] = (int)dest19(P, x, y, z, i);
    if (map7)
      for (int i = 0; i < 7; ++i) {
        const int d = dest7_cell(P, x, y, z, i);
        map7[i * P.N + c] = d < 0 ? -1 : (int)(i * P.N + d);
      }
  }
}

__global__ void k_fill(float* p, long long n, float v) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    p[k] = v;
}

template <typename S>
__global__ void k_sumT(Params P, const S* __restrict__ g, float* T, const float2* ref) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)P.N; c += gridDim.x * blockDim.x) {
    const float t = LocalRef<S>::on ? ref[c].y : 0.f;
    float gl[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = PopStore<S>::ld_plain(g + i * P.N + c, gbase_at<S>(P, i, t));
    T[c] = sum7(gl);
  }
}

}  // namespace

namespace {

long long face_len(const lbm_params& p, int face) {
  const int a = face / 2;
  const int n[3] = {p.nx, p.ny, p.nz};
  long long L = 1;
  for (int b = 0; b < 3; ++b)
    if (b != a) L *= n[b];
  return L;
}

int check_params(const lbm_params* p) {
  if (!p) return LBM_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_ERR_ARG;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > (1LL << 31) - 1) return LBM_ERR_ARG;
  if (p->vartheta != 0 && p->vartheta != 1) return LBM_ERR_ARG;
  if (p->storage != LBM_STORE_F32 && p->storage != LBM_STORE_F16_SHIFTED && p->storage != LBM_STORE_BF16_SHIFTED &&
      p->storage != LBM_STORE_F16_LOCAL)
    return LBM_ERR_ARG;
  if (p->storage != LBM_STORE_F32 && p->schedule == LBM_SCHED_FUSED) return LBM_ERR_ARG;  // FP32 only
  if (p->schedule != LBM_SCHED_FUSED && p->schedule != LBM_SCHED_PHASES && p->schedule != LBM_SCHED_SLABS)
    return LBM_ERR_ARG;
  if (p->eos_kind != 0 && p->eos_kind != 1) return LBM_ERR_ARG;
  if (!(p->cv > 0) || !(p->wbar > 0 && p->wbar < 1) || !(p->lambda_l > 0) || !(p->lambda_v > 0)) return LBM_ERR_ARG;
  if (p->lambda_l != p->lambda_v && !(p->rho_l > p->rho_v)) return LBM_ERR_ARG;
  if (p->G == 0 || !std::isfinite(p->a) || !std::isfinite(p->b)) return LBM_ERR_ARG;
  if (p->eos_kind == 0 && !(p->a > 0 && p->b > 0 && p->R > 0)) return LBM_ERR_ARG;
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a) {
    const int k0 = p->face_kind[2 * a], k1 = p->face_kind[2 * a + 1];
    if (k0 < 0 || k0 > 2 || k1 < 0 || k1 > 2) return LBM_ERR_ARG;
    if ((k0 == LBM_FACE_PERIODIC) != (k1 == LBM_FACE_PERIODIC)) return LBM_ERR_ARG;
    if (k0 != LBM_FACE_PERIODIC && n[a] < 3) return LBM_ERR_ARG;
  }
  for (int f1 = 0; f1 < 6; ++f1)
    for (int f2 = 0; f2 < 6; ++f2)
      if (f1 / 2 != f2 / 2 && p->face_kind[f1] == LBM_FACE_WALL && p->face_kind[f2] == LBM_FACE_OPEN)
        return LBM_ERR_ARG;
  for (int f = 0; f < 6; ++f)
    if (p->face_kind[f] == LBM_FACE_OPEN && !(p->face_rho[f] > 0)) return LBM_ERR_ARG;
  for (int f = 0; f < 6; ++f) {
    if (p->face_T_fixed[f] != 0 && p->face_T_fixed[f] != 1) return LBM_ERR_ARG;
    if (p->face_T_fixed[f] && p->face_kind[f] == LBM_FACE_PERIODIC && n[f / 2] < 3) return LBM_ERR_ARG;
  }
  return LBM_OK;
}

Params make_device_params(const lbm_params& p) {
  Params P;
  std::memset(&P, 0, sizeof(P));
  P.nx = p.nx;
  P.ny = p.ny;
  P.nz = p.nz;
  P.N = (long long)p.nx * p.ny * p.nz;
  fdiv_init((unsigned)p.nx, P.dnx_mul, P.dnx_shr);
  fdiv_init((unsigned)p.ny, P.dny_mul, P.dny_shr);
  for (int f = 0; f < 6; ++f) P.tface[f] = p.face_kind[f] != LBM_FACE_PERIODIC || p.face_T_fixed[f] != 0;
  {
    const bool xnp = P.tface[0] || P.tface[1], ynp = P.tface[2] || P.tface[3];
    const bool znp = P.tface[4] || P.tface[5];
    P.bd_zplanes = znp ? 2 : 0;
    P.bd_perim = (xnp && ynp) ? 2 * p.nx + 2 * (p.ny - 2) : (xnp ? 2 * p.ny : (ynp ? 2 * p.nx : 0));
    fdiv_init((unsigned)(p.nx * p.ny), P.dpl_mul, P.dpl_shr);
    fdiv_init((unsigned)(P.bd_perim > 0 ? P.bd_perim : 1), P.dper_mul, P.dper_shr);
    P.bd_total = (long long)P.bd_zplanes * p.nx * p.ny + (long long)(p.nz - P.bd_zplanes) * P.bd_perim;
  }
  P.meq_printed = p.meq_printed;
  P.wall_ueq_zero = p.wall_ueq_zero;
  P.vartheta = p.vartheta;
  P.eos_kind = p.eos_kind;
  P.a = (float)p.a;
  P.b = (float)p.b;
  P.R = (float)p.R;
  P.kappa = (float)(0.37464 + 1.54226 * p.omega - 0.26992 * p.omega * p.omega);
  P.inv_Tc = p.eos_kind == 0 ? (float)(1.0 / lbm_Tc(&p)) : 1.f;
  P.G = (float)p.G;
  P.inv_G = (float)(1.0 / p.G);
  P.eos_c0 = (float)p.eos_c0;
  P.s_e = (float)p.s_e;
  P.s_v = (float)p.s_v;
  P.s_q = (float)p.s_q;
  P.s_pi = (float)p.s_pi;
  P.cv = (float)p.cv;
  P.inv_cv = (float)(1.0 / p.cv);
  P.wbar = (float)p.wbar;
  P.inv_cs2t = (float)(3.0 / p.wbar);
  P.lambda_l = (float)p.lambda_l;
  P.lambda_v = (float)p.lambda_v;
  P.rho_l = (float)p.rho_l;
  P.rho_v = (float)p.rho_v;
  P.inv_drho = (p.rho_l > p.rho_v) ? (float)(1.0 / (p.rho_l - p.rho_v)) : 0.f;
  P.lam_uniform = p.lambda_l == p.lambda_v;
  P.fast19 = p.s_q == 1.0 && p.s_pi == 1.0 && !p.meq_printed;
  // shifts of the 16-bit storage; defaults: rho_v, and the mean Dirichlet face temperature
  // (else 0.9 T_c for the Peng-Robinson fluid, else 1)
  double tref = p.store_T_ref;
  if (!(tref > 0)) {
    double s = 0;
    int n = 0;
    for (int f = 0; f < 6; ++f)
      if (P.tface[f]) {
        s += p.face_T[f];
        ++n;
      }
    tref = n ? s / n : (p.eos_kind == 0 ? 0.9 * lbm_Tc(&p) : 1.0);
  }
  P.rho_ref = (float)(p.store_rho_ref > 0 ? p.store_rho_ref : (p.rho_v > 0 ? p.rho_v : 0.0));
  P.T_ref = (float)tref;
  P.any_nonperiodic = 0;
  for (int f = 0; f < 6; ++f) {
    P.face_kind[f] = p.face_kind[f];
    P.face_rho[f] = (float)p.face_rho[f];
    const double th = p.face_theta_deg[f] * M_PI / 180.0;
    const double tn = std::tan(M_PI / 2.0 - th);
    P.tan_wet[f] = (p.face_theta_deg[f] == 90.0) ? 0.f : (float)tn;
    if (p.face_kind[f] != LBM_FACE_PERIODIC) P.any_nonperiodic = 1;
  }
  return P;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)(b < 1 ? 1 : b);
}

#define LBM_TRY(expr)                           \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return LBM_ERR_CUDA; \
  } while (0)

int copy_in(float* dst, const float* src, long long n, int mem, cudaStream_t s) {
  LBM_TRY(cudaMemcpyAsync(dst, src, sizeof(float) * n, mem == LBM_MEM_HOST ? cudaMemcpyHostToDevice
                                                                           : cudaMemcpyDeviceToDevice, s));
  return LBM_OK;
}

int copy_out(float* dst, const float* src, long long n, int mem, cudaStream_t s) {
  LBM_TRY(cudaMemcpyAsync(dst, src, sizeof(float) * n, mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                           : cudaMemcpyDeviceToDevice, s));
  return LBM_OK;
}

int read_flags(lbm_ctx* c) {
  LBM_TRY(cudaMemcpyAsync(c->err_h, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LBM_TRY(cudaStreamSynchronize(c->stream));
  const int e = *c->err_h;
  if (e & ERRF_TIMEOUT) return LBM_ERR_TIMEOUT;
  if (e & ERRF_NONFINITE) return LBM_ERR_NONFINITE;
  if (e & ERRF_PSI) return LBM_ERR_PSI_DOMAIN;
  return LBM_OK;
}

cudaEvent_t ev_get(lbm_ctx* c) {
  if (!c->pool->empty()) {
    cudaEvent_t e = c->pool->back();
    c->pool->pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Accumulates the recorded launch times (synchronises on the recorded events).
int prof_collect(lbm_ctx* c) {
  for (auto& e : *c->evs) {
    if (cudaEventSynchronize(e.b) != cudaSuccess) return LBM_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) != cudaSuccess) return LBM_ERR_CUDA;
    c->prof_ms[e.kind] += ms;
    c->prof_n[e.kind] += 1;
    c->pool->push_back(e.a);
    c->pool->push_back(e.b);
  }
  c->evs->clear();
  return LBM_OK;
}

// Start / end marks of one launch while profiling (no-ops otherwise).
cudaEvent_t prof_begin(lbm_ctx* c) {
  if (!c->profiling) return nullptr;
  if (c->evs->size() >= 8192) prof_collect(c);
  cudaEvent_t e = ev_get(c);
  cudaEventRecord(e, c->stream);
  return e;
}

void prof_end(lbm_ctx* c, int kind, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b = ev_get(c);
  cudaEventRecord(b, c->stream);
  c->evs->push_back({kind, a, b});
}

template <typename T>
T* fbuf(lbm_ctx* c, int k) {
  return static_cast<T*>(c->f[k]);
}
template <typename T>
T* gbuf(lbm_ctx* c, int k) {
  return static_cast<T*>(c->g[k]);
}

// calls FN<T>(args...) with T the population storage type of the context
#define LBM_WITH_STORAGE(c, FN, ...)                                                             \
  ((c)->hp.storage == LBM_STORE_F16_SHIFTED    ? FN<__half>(__VA_ARGS__)                          \
   : (c)->hp.storage == LBM_STORE_BF16_SHIFTED ? FN<__nv_bfloat16>(__VA_ARGS__)                   \
   : (c)->hp.storage == LBM_STORE_F16_LOCAL    ? FN<lhalf>(__VA_ARGS__)                           \
                                               : FN<float>(__VA_ARGS__))

// per-cell references of population buffer k (NULL without them)
float2* ref_of(const lbm_ctx* c, int k) { return c->ref ? c->ref + (long long)k * c->N : nullptr; }

// the scratch of a step that reads buffer a and writes buffer 1 - a
template <typename T>
AuxFor<T> aux_for(const lbm_ctx* c, int a) {
  AuxFor<T> X;
  static_cast<Aux&>(X) = c->X;
  if constexpr (LocalRef<T>::on) {
    X.ref_in = ref_of(c, a);
    X.ref_out = ref_of(c, 1 - a);
  }
  return X;
}

// Phases A and B on the current state (macros of time t); returns launch status.
// (with per-cell references phase A also writes those of the idle buffer: harmless)
template <typename T>
int run_macros_t(lbm_ctx* c, float* Tout) {
  k_phaseA<T><<<c->grid, kThreads, 0, c->stream>>>(c->P, fbuf<T>(c, c->cur), gbuf<T>(c, c->cur), aux_for<T>(c, c->cur),
                                                   Tout, c->err_d, 0, (int)c->N, 1);
  k_phaseB<<<c->grid, kThreads, 0, c->stream>>>(c->P, c->X, 0, (int)c->N);
  return cuda_status(cudaGetLastError());
}

int run_macros(lbm_ctx* c, float* Tout) { return LBM_WITH_STORAGE(c, run_macros_t, c, Tout); }

// One step, one launch per phase: A, force + D3Q19 collision/push (B and C19
// in one pass), D3Q7 collision/push, D on the face nodes of the new state.
template <typename T>
int step_phases_t(lbm_ctx* c) {
  const int a = c->cur, b = 1 - c->cur;
  const AuxFor<T> X = aux_for<T>(c, a);
  cudaEvent_t e = prof_begin(c);
  launch_phaseA<T>(c, X, c->grid, c->stream, fbuf<T>(c, a), gbuf<T>(c, a), 0, (int)c->N);
  prof_end(c, 0, e);
  e = prof_begin(c);
  launch_bc19<T>(c, X, c->grid, c->stream, fbuf<T>(c, a), fbuf<T>(c, b), 0, (int)c->N);
  prof_end(c, 2, e);
  // the D3Q7 phase needs the velocity of the neighbours: after the whole D3Q19 pass
  e = prof_begin(c);
  launch_c7<T>(c, X, c->grid, c->stream, gbuf<T>(c, a), gbuf<T>(c, b), 0, (int)c->N);
  prof_end(c, 5, e);
  if (c->P.bd_total > 0) {
    e = prof_begin(c);
    k_phaseD<T><<<grid_for(c->P.bd_total), kThreads, 0, c->stream>>>(c->P, fbuf<T>(c, b), gbuf<T>(c, b), X);
    prof_end(c, 3, e);
  }
  c->cur = b;
  return cuda_status(cudaGetLastError());
}

int step_phases(lbm_ctx* c) { return LBM_WITH_STORAGE(c, step_phases_t, c); }
}  // namespace

// one step of the phase schedule on the context's current buffers and scratch
int lbm_step_phases_internal(lbm_ctx* c) { return step_phases(c); }

namespace {


// ----------------------------------------------------------- slab pipeline --
int slab_of_wrap(const SlabPlan& S, bool zper, int q, bool& ok) {
  ok = true;
  if (q < 0 || q >= S.nslab) {
    if (!zper) {
      ok = false;
      return 0;
    }
    q = (q % S.nslab + S.nslab) % S.nslab;
  }
  return q;
}

// stage codes this stage waits for within one step
void slab_deps_within(const SlabPlan& S, bool zper, int ph, int s, std::vector<int>& d) {
  d.clear();
  auto add = [&](int p, int q) {
    bool ok;
    const int w = slab_of_wrap(S, zper, q, ok);
    if (ok) d.push_back(p * S.nslab + w);
  };
  if (ph == SPH_C19)
    for (int k = -1; k <= 1; ++k) add(SPH_A, s + k);
  if (ph == SPH_C7)
    for (int k = -1; k <= 1; ++k) add(SPH_C19, s + k);
  if (ph == SPH_D)
    for (int k = -1; k <= 1; ++k) {
      add(SPH_C19, s + k);
      add(SPH_C7, s + k);
    }
}

// stages of the previous step that phase A of slab s waits for: the pushes and
// boundary rules that write slab s, and the reads of the scratch of slab s
// that phase A overwrites.  with_d: the previous step ran its phase D stages (otherwise
// this phase A applies the face rules itself; see phaseA)
void slab_deps_prev(const SlabPlan& S, bool zper, int s, std::vector<int>& d, bool with_d = true) {
  d.clear();
  for (int k = -1; k <= 1; ++k) {
    bool ok;
    const int w = slab_of_wrap(S, zper, s + k, ok);
    if (!ok) continue;
    d.push_back(SPH_C19 * S.nslab + w);
    d.push_back(SPH_C7 * S.nslab + w);
  }
  if (with_d && S.has_d[s]) d.push_back(SPH_D * S.nslab + s);
}

int env_int(const char* name, int dflt) {
  const char* e = std::getenv(name);
  return e ? std::atoi(e) : dflt;
}

void slab_plan_destroy(SlabPlan* S) {
  if (!S) return;
  for (int k = 0; k < 2; ++k) {
    if (S->graph[k]) cudaGraphExecDestroy(S->graph[k]);
    if (S->graph1[k]) cudaGraphExecDestroy(S->graph1[k]);
  }
  for (auto e : S->ev)
    if (e) cudaEventDestroy(e);
  if (S->fork) cudaEventDestroy(S->fork);
  for (int i = 0; i < S->nstreams; ++i) {
    if (S->join[i]) cudaEventDestroy(S->join[i]);
    if (S->st[i]) {
      cudaStreamSynchronize(S->st[i]);
      cudaStreamDestroy(S->st[i]);
    }
  }
  delete S;
}

// The host part of a slab plan: slabs of about sp planes (at least 3), which of them
// hold face nodes, and the stage order (a topological order of the within-step
// dependencies along the diagonal wavefront slab + lag(phase)).  Returns false if no
// order exists (not reachable: the dependency graph is acyclic).
bool slab_plan_layout(const Params& P, int sp, SlabPlan* S) {
  const int nz = P.nz;
  sp = std::max(3, std::min(sp, nz));
  S->nslab = std::max(1, nz / sp);
  S->zb.clear();
  for (int s = 0; s <= S->nslab; ++s) S->zb.push_back((int)((long long)nz * s / S->nslab));
  S->has_d.assign(S->nslab, 0);
  for (int s = 0; s < S->nslab; ++s)
    for (int z = S->zb[s]; z < S->zb[s + 1]; ++z)
      if (plane_has_boundary(P, z)) S->has_d[s] = 1;
  const bool zper = P.face_kind[4] == FACE_PERIODIC;
  const int lag[SPH_N] = {0, 1, 2, 3};
  const int n = S->nslab;
  std::vector<char> placed(SPH_N * n, 0), exists(SPH_N * n, 1);
  for (int s = 0; s < n; ++s) exists[SPH_D * n + s] = S->has_d[s];
  int total = 0;
  for (int k = 0; k < SPH_N * n; ++k) total += exists[k];
  std::vector<int> d;
  S->order.clear();
  while ((int)S->order.size() < total) {
    int best = -1, bestkey = 1 << 30;
    for (int ph = SPH_N - 1; ph >= 0; --ph)
      for (int s = 0; s < n; ++s) {
        const int id = ph * n + s;
        if (!exists[id] || placed[id]) continue;
        slab_deps_within(*S, zper, ph, s, d);
        bool ready = true;
        for (int q : d) ready = ready && placed[q];
        if (!ready) continue;
        const int key = s + lag[ph];
        if (key < bestkey) {
          bestkey = key;
          best = id;
        }
      }
    if (best < 0) return false;
    placed[best] = 1;
    S->order.push_back(best);
  }
  return true;
}

int slab_plan_create(lbm_ctx* c) {
  SlabPlan* S = new (std::nothrow) SlabPlan();
  if (!S) return LBM_ERR_ARG;
  const int plane = c->P.nx * c->P.ny;
  int sp = env_int("LBM_SLAB_PLANES", 0);
  if (sp <= 0) sp = std::max(3, (262144 + plane - 1) / plane);  // about 256 Ki cells per slab kernel
  if (!slab_plan_layout(c->P, sp, S)) {
    slab_plan_destroy(S);
    return LBM_ERR_ARG;
  }
  const int n = S->nslab;
  S->nstreams = std::max(1, std::min(kMaxSlabStreams, env_int("LBM_SLAB_STREAMS", 8)));
  bool ok = cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < S->nstreams && ok; ++i) {
    ok = cudaStreamCreateWithFlags(&S->st[i], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&S->join[i], cudaEventDisableTiming) == cudaSuccess;
  }
  S->ev.assign(SPH_N * n, nullptr);
  for (int k = 0; k < SPH_N * n && ok; ++k)
    if (k / n != SPH_D || S->has_d[k % n])  // the stages that exist
      ok = cudaEventCreateWithFlags(&S->ev[k], cudaEventDisableTiming) == cudaSuccess;
  S->graph_steps = std::max(0, env_int("LBM_GRAPH_STEPS", 8));
  if (S->graph_steps & 1) S->graph_steps += 1;  // even: the buffers return to their parity
  c->slabs = S;
  return ok ? LBM_OK : LBM_ERR_CUDA;
}

// Enqueues one time step (buffers cur -> 1-cur) on the slab streams.  `first`:
// the previous step's per-slab events are not waited for (the caller forked
// all slab streams from the main stream after that step).  `fuse`: the previous step left
// its face rules to this step's phase A (it enqueued no phase D).  `emit_d`: this step
// enqueues its phase D stages (the last step of every sequence does).
template <typename T>
int slab_enqueue_step_t(lbm_ctx* c, bool first, bool fuse, bool emit_d) {
  SlabPlan& S = *c->slabs;
  const int a = c->cur, b = 1 - c->cur;
  const AuxFor<T> X = aux_for<T>(c, a);
  const bool zper = c->P.face_kind[4] == FACE_PERIODIC;
  const int n = S.nslab, plane = c->P.nx * c->P.ny;
  std::vector<int> d;
  for (int code : S.order) {
    const int ph = code / n, s = code % n;
    if (ph == SPH_D && !emit_d) continue;
    cudaStream_t st = S.st[s % S.nstreams];
    if (ph == SPH_A) {
      if (!first) slab_deps_prev(S, zper, s, d, !fuse);
      else d.clear();
    } else {
      slab_deps_within(S, zper, ph, s, d);
    }
    for (int q : d) cudaStreamWaitEvent(st, S.ev[q], 0);
    const int z0 = S.zb[s], z1 = S.zb[s + 1];
    const int c0 = z0 * plane, c1 = z1 * plane;
    const int blocks = std::min(grid_for((long long)(c1 - c0)), 152 * 8);
    switch (ph) {
      case SPH_A:
        if constexpr (!LocalRef<T>::on) {
          if (fuse && S.has_d[s]) {
            k_phaseA<T, true><<<blocks, kThreads, 0, st>>>(c->P, fbuf<T>(c, a), gbuf<T>(c, a), X, nullptr, c->err_d,
                                                           c0, c1, 0);
            break;
          }
        }
        launch_phaseA<T>(c, X, blocks, st, fbuf<T>(c, a), gbuf<T>(c, a), c0, c1);
        break;
      case SPH_C19:
        launch_bc19<T>(c, X, blocks, st, fbuf<T>(c, a), fbuf<T>(c, b), c0, c1);
        break;
      case SPH_C7:
        launch_c7<T>(c, X, blocks, st, gbuf<T>(c, a), gbuf<T>(c, b), c0, c1);
        break;
      default: {
        int maxcnt = 0;
        for (int z = z0; z < z1; ++z) {
          const bool zb = (c->P.tface[4] || c->P.tface[5]) && (z == 0 || z == c->P.nz - 1);
          maxcnt = std::max(maxcnt, zb ? plane : c->P.bd_perim);
        }
        dim3 gd((unsigned)std::max(1, (maxcnt + kThreads - 1) / kThreads), (unsigned)(z1 - z0));
        k_phaseD_planes<T><<<gd, kThreads, 0, st>>>(c->P, fbuf<T>(c, b), gbuf<T>(c, b), X, z0);
      }
    }
    cudaEventRecord(S.ev[code], st);
  }
  c->cur = b;
  return cuda_status(cudaGetLastError());
}

int slab_enqueue_step(lbm_ctx* c, bool first, bool fuse, bool emit_d) {
  return LBM_WITH_STORAGE(c, slab_enqueue_step_t, c, first, fuse, emit_d);
}

// Steps k = 0 .. steps-1 of one sequence of slab steps: phase D of every step but the last
// goes into the next step's phase A, so that the state is complete when the sequence ends.
// Only where the face nodes are whole z planes (the x and y faces periodic, without held
// temperature layers): there every lane of a phase-A warp on a face plane applies the rules.
// With x or y face nodes one lane in a warp would apply them while the others wait, and the
// separate pass measured faster.  Not with per-cell references.
bool slab_fuse_d(const lbm_ctx* c) {
  const Params& P = c->P;
  return c->hp.storage != LBM_STORE_F16_LOCAL && !(P.tface[0] || P.tface[1] || P.tface[2] || P.tface[3]);
}
int slab_enqueue_seq_step(lbm_ctx* c, int k, int steps) {
  const bool fd = slab_fuse_d(c);
  return slab_enqueue_step(c, k == 0, fd && k > 0, !fd || k == steps - 1);
}

// every slab stream waits for `main`
void slab_fork(lbm_ctx* c, cudaStream_t main) {
  SlabPlan& S = *c->slabs;
  cudaEventRecord(S.fork, main);
  for (int i = 0; i < S.nstreams; ++i)
    if (S.st[i] != main) cudaStreamWaitEvent(S.st[i], S.fork, 0);
}

// `main` waits for every slab stream
void slab_join(lbm_ctx* c, cudaStream_t main) {
  SlabPlan& S = *c->slabs;
  for (int i = 0; i < S.nstreams; ++i) {
    if (S.st[i] == main) continue;
    cudaEventRecord(S.join[i], S.st[i]);
    cudaStreamWaitEvent(main, S.join[i], 0);
  }
}

// Captures `steps` steps starting from the current parity into *dst.  The capture
// runs on the first slab stream (the caller's stream may be the legacy default
// stream, which cannot be captured); the graph is then launched on the caller's
// stream.
int slab_capture(lbm_ctx* c, int steps, cudaGraphExec_t* dst) {
  SlabPlan& S = *c->slabs;
  const int parity = c->cur;
  cudaStream_t cs = S.st[0];
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
  slab_fork(c, cs);
  int st = LBM_OK;
  for (int k = 0; k < steps && st == LBM_OK; ++k) st = slab_enqueue_seq_step(c, k, steps);
  slab_join(c, cs);
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  c->cur = parity;  // capture recorded the steps without running them
  if (st != LBM_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(dst, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return LBM_ERR_CUDA;
  // move the graph to the device now rather than at its first launch
  return cudaGraphUpload(*dst, cs) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Captures (and uploads) the graphs of both buffer parities up front (lbm_init), so that no
// lbm_step pays a capture or an upload: graph_steps steps for long runs and one step for the
// remainder.
int slab_capture_both(lbm_ctx* c) {
  SlabPlan& S = *c->slabs;
  if (S.graph_steps <= 0) return LBM_OK;
  const int cur = c->cur;
  int st = LBM_OK;
  for (int k = 0; k < 2 && st == LBM_OK; ++k) {
    c->cur = k;
    if (!S.graph[k]) st = slab_capture(c, S.graph_steps, &S.graph[k]);
    if (st == LBM_OK && !S.graph1[k]) st = slab_capture(c, 1, &S.graph1[k]);
  }
  c->cur = cur;
  return st;
}

int step_slabs(lbm_ctx* c, int n) {
  SlabPlan& S = *c->slabs;
  cudaEvent_t e = prof_begin(c);
  int st = LBM_OK;
  int done = 0;
  if (S.graph_steps > 0) {
    while (n - done >= S.graph_steps && st == LBM_OK) {
      if (!S.graph[c->cur]) st = slab_capture(c, S.graph_steps, &S.graph[c->cur]);
      if (st != LBM_OK) break;
      if (cudaGraphLaunch(S.graph[c->cur], c->stream) != cudaSuccess) st = LBM_ERR_CUDA;
      done += S.graph_steps;  // parity unchanged: graph_steps is even
    }
    for (; done < n && st == LBM_OK && S.graph1[c->cur]; ++done) {
      if (cudaGraphLaunch(S.graph1[c->cur], c->stream) != cudaSuccess) st = LBM_ERR_CUDA;
      c->cur = 1 - c->cur;
    }
  }
  if (st == LBM_OK && done < n) {
    slab_fork(c, c->stream);
    const int rest = n - done;
    for (int k = 0; done < n && st == LBM_OK; ++done, ++k) st = slab_enqueue_seq_step(c, k, rest);
    slab_join(c, c->stream);
  }
  prof_end(c, 4, e);
  return st;
}
}  // namespace

namespace {

// Moves f/g (float, caller memory) into or out of 16-bit shifted storage through a
// temporary device buffer (not on the time-stepping path).
template <typename T>
int convert_state_t(lbm_ctx* c, float* f, float* g, int mem, bool in) {
  const long long N = c->N;
  float* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(float) * 19 * N) != cudaSuccess) return LBM_ERR_CUDA;
  int st = LBM_OK;
  const int blocks = grid_for(19 * N);
  float* user[2] = {f, g};
  const int q[2] = {19, 7};
  void* buf[2] = {c->f[c->cur], c->g[c->cur]};
  float2* ref = ref_of(c, c->cur);
  for (int k = 0; k < 2 && st == LBM_OK; ++k) {
    if (!user[k]) continue;
    if (in) {
      st = copy_in(tmp, user[k], q[k] * N, mem, c->stream);
      // per-cell references of the state set: its own rho and T
      if (!st && ref) k_ref_sum<<<c->grid, kThreads, 0, c->stream>>>(c->P, tmp, q[k], ref, k);
      if (!st) k_store<T><<<blocks, kThreads, 0, c->stream>>>(c->P, tmp, static_cast<T*>(buf[k]), q[k], k, ref);
    } else {
      k_load<T><<<blocks, kThreads, 0, c->stream>>>(c->P, static_cast<const T*>(buf[k]), tmp, q[k], k, ref);
      st = copy_out(user[k], tmp, q[k] * N, mem, c->stream);
    }
    if (!st) st = cuda_status(cudaStreamSynchronize(c->stream));
  }
  cudaFree(tmp);
  return st;
}

int convert_state(lbm_ctx* c, float* f, float* g, int mem, bool in) {
  return LBM_WITH_STORAGE(c, convert_state_t, c, f, g, mem, in);
}

}  // namespace

namespace {

// vartheta = 1: the T history of a state taken to be at rest before now,
// T(t-1) = T(t-2) = T = sum g of the current populations.
template <typename T>
int hist_reset_t(lbm_ctx* c) {
  k_sumT<T><<<c->grid, kThreads, 0, c->stream>>>(c->P, gbuf<T>(c, c->cur), c->X.T1, ref_of(c, c->cur));
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  return cuda_status(cudaMemcpyAsync(c->X.T2, c->X.T1, sizeof(float) * c->N, cudaMemcpyDeviceToDevice, c->stream));
}

int hist_reset(lbm_ctx* c) { return c->hist ? LBM_WITH_STORAGE(c, hist_reset_t, c) : LBM_OK; }

// T = sum g of the current state into T (lbm_macros)
template <typename S>
int launch_sumT(lbm_ctx* c, float* T) {
  k_sumT<S><<<c->grid, kThreads, 0, c->stream>>>(c->P, gbuf<S>(c, c->cur), T, ref_of(c, c->cur));
  return LBM_OK;
}

// per-block FP64 partial sums of the current state (lbm_reduce)
template <typename S>
int launch_reduce(lbm_ctx* c) {
  k_reduce<S><<<c->red_blocks, kThreads, 0, c->stream>>>(c->P, fbuf<S>(c, c->cur), gbuf<S>(c, c->cur), c->partial,
                                                         ref_of(c, c->cur));
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_status_string(int s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_NONFINITE: return "non-finite population";
    case LBM_ERR_PSI_DOMAIN: return "psi undefined: 2(p_EOS - rho/3)/G < 0";
    case LBM_ERR_TIMEOUT: return "bounded device wait gave up";
    case LBM_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

double lbm_Tc(const lbm_params* p) { return 0.0778 * p->a / (0.45724 * p->b * p->R); }

// Maxwell equal-area construction for the PR EOS (Sec. 4.2): bisection on
// p_sat between the spinodal pressures, the area by composite Simpson rule.
int lbm_maxwell(const lbm_params* p, double T, double* rho_v, double* rho_l, double* p_sat) {
  if (!p || p->eos_kind != 0) return LBM_ERR_ARG;
  const double Tc = lbm_Tc(p);
  if (!(T > 0 && T < Tc)) return LBM_ERR_ARG;
  const double k = 0.37464 + 1.54226 * p->omega - 0.26992 * p->omega * p->omega;
  const double s = 1.0 + k * (1.0 - std::sqrt(T / Tc));
  const double axi = p->a * s * s, b = p->b, R = p->R;
  auto pr = [&](double r) { return r * R * T / (1.0 - b * r) - axi * r * r / (1.0 + 2.0 * b * r - b * b * r * r); };
  // spinodals by a scan of p on (0, 1/b)
  const int n = 100000;
  const double h = (1.0 / b) / n;
  double rmax = -1, rmin = -1;
  for (int i = 1; i < n - 1; ++i) {
    const double r = i * h;
    const double d0 = pr(r + h) - pr(r), d1 = pr(r + 2 * h) - pr(r + h);
    if (rmax < 0 && d0 > 0 && d1 <= 0) rmax = r + h;
    if (rmax > 0 && d0 < 0 && d1 >= 0) {
      rmin = r + h;
      break;
    }
  }
  if (rmax < 0 || rmin < 0) return LBM_ERR_ARG;
  auto root = [&](double ps, double lo, double hi) {
    const bool inc = pr(hi) > pr(lo);
    for (int it = 0; it < 120; ++it) {
      const double mid = 0.5 * (lo + hi);
      if ((pr(mid) < ps) == inc)
        lo = mid;
      else
        hi = mid;
    }
    return 0.5 * (lo + hi);
  };
  double lo = std::fmax(pr(rmin), 1e-14), hi = pr(rmax), rv = 0, rl = 0, ps = 0;
  for (int it = 0; it < 100; ++it) {
    ps = 0.5 * (lo + hi);
    rv = root(ps, 1e-12, rmax);
    rl = root(ps, rmin, (1.0 / b) * (1 - 1e-9));
    // area of (p - ps)/rho^2 from rv to rl, Simpson with 4000 panels
    const int m = 4000;
    const double hh = (rl - rv) / m;
    double acc = 0;
    for (int j = 0; j <= m; ++j) {
      const double r = rv + j * hh;
      const double w = (j == 0 || j == m) ? 1 : ((j & 1) ? 4 : 2);
      acc += w * (pr(r) - ps) / (r * r);
    }
    const double area = acc * hh / 3.0;
    if (area > 0)
      lo = ps;
    else
      hi = ps;
  }
  if (rho_v) *rho_v = rv;
  if (rho_l) *rho_l = rl;
  if (p_sat) *p_sat = ps;
  return LBM_OK;
}

int lbm_init(lbm_ctx** out, const lbm_params* p, const float* rho0, const float* T0, int mem, void* stream) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  int st = check_params(p);
  if (st) return st;
  if ((rho0 == nullptr) != (T0 == nullptr)) return LBM_ERR_ARG;
  lbm_ctx* c = new (std::nothrow) lbm_ctx;
  if (!c) return LBM_ERR_ARG;
  std::memset(c, 0, sizeof(*c));
  c->evs = new (std::nothrow) std::vector<lbm_ctx::Ev>();
  c->pool = new (std::nothrow) std::vector<cudaEvent_t>();
  if (!c->evs || !c->pool) {
    delete c->evs;
    delete c->pool;
    delete c;
    return LBM_ERR_ARG;
  }
  c->hp = *p;
  c->P = make_device_params(*p);
  c->stream = (cudaStream_t)stream;
  c->N = c->P.N;
  c->grid = grid_for(c->N);
  // Force + D3Q19 and D3Q7 with staged populations: FP32, every slab and the lattice divide
  // into whole tiles, and the lattice has at least four tiles per resident CTA (four per SM),
  // so that the copy of the next tile has one to overlap.  Smaller lattices, and the 16-bit
  // forms (tile rows of 512 bytes), measured slower staged.  LBM_STAGE19 and LBM_STAGE7 set
  // the tiles per CTA (0: off).
  {
    const bool stage = p->storage == LBM_STORE_F32 && (p->nx * p->ny) % kStageT == 0 &&
                       c->N >= 4ll * 152 * 4 * kStageT;
    c->stage19 = stage ? std::max(0, env_int("LBM_STAGE19", 4)) : 0;
    c->stage7 = stage ? std::max(0, env_int("LBM_STAGE7", 4)) : 0;
  }
  c->esize = p->storage == LBM_STORE_F32 ? sizeof(float) : 2;
  cudaGetDevice(&c->device);
  const long long N = c->N;
  bool ok = true;
  for (int k = 0; k < 2; ++k) {
    ok = ok && cudaMalloc(&c->f[k], c->esize * 19 * N) == cudaSuccess;
    ok = ok && cudaMalloc(&c->g[k], c->esize * 7 * N) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&c->aux, sizeof(float) * 11 * N) == cudaSuccess;
  if (p->vartheta) ok = ok && cudaMalloc(&c->hist, sizeof(float) * 2 * N) == cudaSuccess;
  if (p->storage == LBM_STORE_F16_LOCAL) ok = ok && cudaMalloc(&c->ref, sizeof(float2) * 2 * N) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMalloc(&c->err_d, 2 * sizeof(int)) == cudaSuccess;  // error flags, stall request
  ok = ok && cudaMallocHost(&c->err_h, sizeof(int)) == cudaSuccess;
  c->red_blocks = grid_for(N) < 1024 ? grid_for(N) : 1024;
  ok = ok && cudaMalloc(&c->partial, sizeof(double) * 4 * c->red_blocks) == cudaSuccess;
  ok = ok && cudaMalloc(&c->red_out, sizeof(double) * 4) == cudaSuccess;
  ok = ok && cudaMallocHost(&c->red_h, sizeof(double) * 4) == cudaSuccess;
  for (int f = 0; f < 6 && ok; ++f) {
    if (!c->P.tface[f]) continue;
    c->tface_n[f] = face_len(*p, f);
    ok = cudaMalloc(&c->tface[f], sizeof(float) * c->tface_n[f]) == cudaSuccess;
    if (ok) {
      k_fill<<<grid_for(c->tface_n[f]), kThreads, 0, c->stream>>>(c->tface[f], c->tface_n[f], (float)p->face_T[f]);
      c->P.Tface[f] = c->tface[f];
    }
  }
  if (!ok) {
    lbm_destroy(c);
    return LBM_ERR_CUDA;
  }
  float* a = c->aux;
  c->X = Aux{a, a + N, a + 2 * N, a + 3 * N, a + 4 * N, a + 5 * N, a + 6 * N, a + 7 * N, a + 8 * N, a + 9 * N, a + 10 * N};
  if (c->hist) {
    c->X.T1 = c->hist;
    c->X.T2 = c->hist + N;
  }
  if (cudaMemsetAsync(c->err_d, 0, 2 * sizeof(int), c->stream) != cudaSuccess) {
    lbm_destroy(c);
    return LBM_ERR_CUDA;
  }
  if (p->schedule == LBM_SCHED_SLABS) {
    st = slab_plan_create(c);
    if (st == LBM_OK) st = slab_capture_both(c);
    if (st != LBM_OK) {
      lbm_destroy(c);
      return st;
    }
  }
  st = fused_plan(c->P, &c->plan);
  if (st == LBM_OK && p->schedule == LBM_SCHED_FUSED) st = fused_alloc(&c->plan, c->P, c->stream);
  if (st != LBM_OK) st = st == -1 ? LBM_ERR_ARG : LBM_ERR_CUDA;
  if (st != LBM_OK) {
    lbm_destroy(c);
    return st;
  }
  if (rho0) {
    float *r = nullptr, *t = nullptr;
    if (mem == LBM_MEM_HOST) {
      r = c->aux;  // stage through the scratch area
      t = c->aux + N;
      if (copy_in(r, rho0, N, mem, c->stream) || copy_in(t, T0, N, mem, c->stream)) {
        lbm_destroy(c);
        return LBM_ERR_CUDA;
      }
    } else {
      r = (float*)rho0;
      t = (float*)T0;
    }
    if (p->storage == LBM_STORE_F16_SHIFTED)
      k_init<__half><<<c->grid, kThreads, 0, c->stream>>>(c->P, r, t, fbuf<__half>(c, 0), gbuf<__half>(c, 0), nullptr);
    else if (p->storage == LBM_STORE_BF16_SHIFTED)
      k_init<__nv_bfloat16><<<c->grid, kThreads, 0, c->stream>>>(c->P, r, t, fbuf<__nv_bfloat16>(c, 0),
                                                                 gbuf<__nv_bfloat16>(c, 0), nullptr);
    else if (p->storage == LBM_STORE_F16_LOCAL)
      k_init<lhalf><<<c->grid, kThreads, 0, c->stream>>>(c->P, r, t, fbuf<lhalf>(c, 0), gbuf<lhalf>(c, 0),
                                                         ref_of(c, 0));
    else
      k_init<float><<<c->grid, kThreads, 0, c->stream>>>(c->P, r, t, fbuf<float>(c, 0), gbuf<float>(c, 0), nullptr);
    if (cudaGetLastError() != cudaSuccess || hist_reset(c) != LBM_OK) {
      lbm_destroy(c);
      return LBM_ERR_CUDA;
    }
    c->has_state = true;
  }
  *out = c;
  return LBM_OK;
}

int lbm_set_state(lbm_ctx* c, const float* f, const float* g, int mem) {
  if (!c || !f || !g) return LBM_ERR_ARG;
  int st = LBM_OK;
  if (c->hp.storage == LBM_STORE_F32) {
    st = copy_in(fbuf<float>(c, c->cur), f, 19 * c->N, mem, c->stream);
    if (!st) st = copy_in(gbuf<float>(c, c->cur), g, 7 * c->N, mem, c->stream);
  } else {
    st = convert_state(c, const_cast<float*>(f), const_cast<float*>(g), mem, true);
  }
  if (!st) st = hist_reset(c);
  if (!st && mem == LBM_MEM_HOST) st = cuda_status(cudaStreamSynchronize(c->stream));
  if (!st && fused_reset(&c->plan, c->P, c->stream)) st = LBM_ERR_CUDA;
  if (!st) st = cuda_status(cudaMemsetAsync(c->err_d, 0, 2 * sizeof(int), c->stream));  // flags and stall request
  if (!st) c->has_state = true;
  return st;
}

int lbm_get_state(lbm_ctx* c, float* f, float* g, int mem) {
  if (!c) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  int st = LBM_OK;
  if (c->hp.storage == LBM_STORE_F32) {
    if (f) st = copy_out(f, fbuf<float>(c, c->cur), 19 * c->N, mem, c->stream);
    if (!st && g) st = copy_out(g, gbuf<float>(c, c->cur), 7 * c->N, mem, c->stream);
  } else {
    st = convert_state(c, f, g, mem, false);
  }
  if (st) return st;
  return read_flags(c);
}

namespace {

// Checkpoint image: this header, then f (19 N) and g (7 N) in the storage format,
// then, for vartheta = 1, the T history (2 N floats), then, for FP16 storage with
// per-cell references, those of the stored populations (2 N floats: rho, T per cell).
struct CkptHeader {
  char magic[8];
  int32_t version, nx, ny, nz, storage, esize;
  float rho_ref, T_ref;
  int32_t vartheta;
  int32_t pad[64 - 11];
};
static_assert(sizeof(CkptHeader) == 256, "checkpoint header is 256 bytes");
constexpr char kCkptMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};

CkptHeader ckpt_header(const lbm_ctx* c) {
  CkptHeader h{};
  for (int i = 0; i < 8; ++i) h.magic[i] = kCkptMagic[i];
  h.version = 1;
  h.nx = c->hp.nx;
  h.ny = c->hp.ny;
  h.nz = c->hp.nz;
  h.storage = c->hp.storage;
  h.esize = (int32_t)c->esize;
  h.rho_ref = c->P.rho_ref;
  h.T_ref = c->P.T_ref;
  h.vartheta = c->P.vartheta;
  return h;
}

}  // namespace

long long lbm_checkpoint_bytes(const lbm_ctx* c) {
  if (!c) return 0;
  return (long long)sizeof(CkptHeader) + 26LL * c->N * (long long)c->esize +
         (c->hist ? 2LL * c->N * (long long)sizeof(float) : 0LL) + (c->ref ? c->N * (long long)sizeof(float2) : 0LL);
}

int lbm_checkpoint(lbm_ctx* c, void* dst, int mem) {
  if (!c || !dst) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  const CkptHeader h = ckpt_header(c);
  const cudaMemcpyKind kd = mem == LBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  char* d = static_cast<char*>(dst);
  const size_t fb = 19ull * c->N * c->esize, gb = 7ull * c->N * c->esize;
  LBM_TRY(cudaMemcpyAsync(d + sizeof(h), c->f[c->cur], fb, kd, c->stream));
  LBM_TRY(cudaMemcpyAsync(d + sizeof(h) + fb, c->g[c->cur], gb, kd, c->stream));
  const size_t hb = c->hist ? 2ull * c->N * sizeof(float) : 0;
  if (c->hist) LBM_TRY(cudaMemcpyAsync(d + sizeof(h) + fb + gb, c->hist, hb, kd, c->stream));
  if (c->ref)
    LBM_TRY(cudaMemcpyAsync(d + sizeof(h) + fb + gb + hb, ref_of(c, c->cur), c->N * sizeof(float2), kd, c->stream));
  if (mem == LBM_MEM_HOST) {
    std::memcpy(d, &h, sizeof(h));
  } else {
    LBM_TRY(cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  }
  return read_flags(c);  // synchronises: the header source is on this stack frame
}

int lbm_restore(lbm_ctx* c, const void* src, int mem) {
  if (!c || !src) return LBM_ERR_ARG;
  CkptHeader h{};
  const char* s = static_cast<const char*>(src);
  if (mem == LBM_MEM_HOST) {
    std::memcpy(&h, s, sizeof(h));
  } else {
    LBM_TRY(cudaMemcpyAsync(&h, s, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    LBM_TRY(cudaStreamSynchronize(c->stream));
  }
  const CkptHeader e = ckpt_header(c);
  if (std::memcmp(h.magic, e.magic, 8) != 0 || h.version != e.version || h.nx != e.nx || h.ny != e.ny ||
      h.nz != e.nz || h.storage != e.storage || h.esize != e.esize || h.rho_ref != e.rho_ref || h.T_ref != e.T_ref ||
      h.vartheta != e.vartheta)
    return LBM_ERR_ARG;
  const cudaMemcpyKind kd = mem == LBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t fb = 19ull * c->N * c->esize, gb = 7ull * c->N * c->esize;
  LBM_TRY(cudaMemcpyAsync(c->f[c->cur], s + sizeof(h), fb, kd, c->stream));
  LBM_TRY(cudaMemcpyAsync(c->g[c->cur], s + sizeof(h) + fb, gb, kd, c->stream));
  const size_t hb = c->hist ? 2ull * c->N * sizeof(float) : 0;
  if (c->hist) LBM_TRY(cudaMemcpyAsync(c->hist, s + sizeof(h) + fb + gb, hb, kd, c->stream));
  if (c->ref)
    LBM_TRY(cudaMemcpyAsync(ref_of(c, c->cur), s + sizeof(h) + fb + gb + hb, c->N * sizeof(float2), kd, c->stream));
  if (mem == LBM_MEM_HOST) LBM_TRY(cudaStreamSynchronize(c->stream));
  if (fused_reset(&c->plan, c->P, c->stream)) return LBM_ERR_CUDA;
  LBM_TRY(cudaMemsetAsync(c->err_d, 0, 2 * sizeof(int), c->stream));  // flags and stall request
  c->has_state = true;
  return LBM_OK;
}

int lbm_set_face_T(lbm_ctx* c, int face, const float* T_face, int mem) {
  if (!c || face < 0 || face > 5 || !T_face) return LBM_ERR_ARG;
  if (!c->tface[face]) return LBM_ERR_ARG;
  int st = copy_in(c->tface[face], T_face, c->tface_n[face], mem, c->stream);
  if (!st && mem == LBM_MEM_HOST) st = cuda_status(cudaStreamSynchronize(c->stream));
  return st;
}

int lbm_inject_stall(lbm_ctx* c) {
  if (!c) return LBM_ERR_ARG;
  if (c->hp.schedule != LBM_SCHED_FUSED) {
    // staged kernels: the next one that runs expects 16 bytes more than its first tile's
    // copies bring, so that its bounded mbarrier waits give up
    if (!(c->stage19 > 0 || c->stage7 > 0)) return LBM_ERR_ARG;
    const int one = 1;
    LBM_TRY(cudaMemcpyAsync(c->err_d + 1, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return cuda_status(cudaStreamSynchronize(c->stream));
  }
  if (!c->plan.done_d) return LBM_ERR_ARG;
  if (c->plan.epoch == 0) return LBM_ERR_STATE;  // the counters are at their start anyway
  // the next launch waits for (epoch + 1) * tiles completions per plane; from zero it
  // reaches one step's worth only
  return cuda_status(cudaMemsetAsync(c->plan.done_d, 0, sizeof(unsigned) * 4 * c->P.nz, c->stream));
}

int lbm_step(lbm_ctx* c, int n) {
  if (!c || n < 0) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  if (c->hp.schedule == LBM_SCHED_SLABS) return n > 0 ? step_slabs(c, n) : LBM_OK;
  for (int s = 0; s < n; ++s) {
    int st;
    if (c->hp.schedule == LBM_SCHED_FUSED) {
      cudaEvent_t e = prof_begin(c);
      st = fused_step(&c->plan, c->P, fbuf<float>(c, c->cur), gbuf<float>(c, c->cur), fbuf<float>(c, 1 - c->cur),
                      gbuf<float>(c, 1 - c->cur), c->X, c->err_d, c->stream);
      prof_end(c, 4, e);
      c->cur = 1 - c->cur;
    } else {
      st = step_phases(c);
    }
    if (st) return st;
  }
  return LBM_OK;
}

int lbm_profile(lbm_ctx* c, int enable) {
  if (!c) return LBM_ERR_ARG;
  int st = prof_collect(c);
  for (int k = 0; k < LBM_PROF_KINDS; ++k) {
    c->prof_ms[k] = 0;
    c->prof_n[k] = 0;
  }
  c->profiling = enable != 0;
  return st;
}

int lbm_profile_read(lbm_ctx* c, long long* launches, double* ms, int nkinds) {
  if (!c || nkinds < 0) return LBM_ERR_ARG;
  const int st = prof_collect(c);
  for (int k = 0; k < nkinds && k < LBM_PROF_KINDS; ++k) {
    if (launches) launches[k] = c->prof_n[k];
    if (ms) ms[k] = c->prof_ms[k];
  }
  return st;
}

namespace {
int slab_d_stages(const lbm_ctx* c) {
  int nd = 0;
  for (char h : c->slabs->has_d) nd += h != 0;
  return nd;
}
}  // namespace

int lbm_launches_per_step(const lbm_ctx* c) {
  if (!c) return 0;
  // slab schedule: in a long run the face rules of a step go into the next step's phase A
  if (c->hp.schedule == LBM_SCHED_SLABS)
    return (int)c->slabs->order.size() - (slab_fuse_d(c) ? slab_d_stages(c) : 0);
  if (c->hp.schedule == LBM_SCHED_FUSED) return fused_launches(&c->plan);
  return c->P.bd_total > 0 ? 4 : 3;
}

long long lbm_step_launches(const lbm_ctx* c, int n) {
  if (!c || n < 0) return -1;
  if (c->hp.schedule != LBM_SCHED_SLABS || !slab_fuse_d(c)) return (long long)n * lbm_launches_per_step(c);
  // every sequence (a replayed graph, a one-step graph or an eager run) ends with phase D
  const SlabPlan& S = *c->slabs;
  long long seq = 0;
  if (n > 0) {
    if (S.graph_steps > 0 && S.graph1[0] && S.graph1[1])
      seq = n / S.graph_steps + n % S.graph_steps;
    else
      seq = S.graph_steps > 0 ? n / S.graph_steps + (n % S.graph_steps ? 1 : 0) : 1;
  }
  return (long long)n * lbm_launches_per_step(c) + seq * slab_d_stages(c);
}

int lbm_macros(lbm_ctx* c, float* rho, float* ux, float* uy, float* uz, float* T, int mem) {
  if (!c) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  // T is summed into the ux slot of the scratch first when requested, then copied
  float* Tscratch = c->aux + 5 * c->N;  // Fx slot, rewritten by phase B below
  if (T) {
    LBM_WITH_STORAGE(c, launch_sumT, c, Tscratch);
    int st = copy_out(T, Tscratch, c->N, mem, c->stream);
    if (st) return st;
  }
  int st = run_macros(c, nullptr);
  if (st) return st;
  if (rho) st = copy_out(rho, c->X.rho, c->N, mem, c->stream);
  if (!st && ux) st = copy_out(ux, c->X.ux, c->N, mem, c->stream);
  if (!st && uy) st = copy_out(uy, c->X.uy, c->N, mem, c->stream);
  if (!st && uz) st = copy_out(uz, c->X.uz, c->N, mem, c->stream);
  if (st) return st;
  return read_flags(c);
}

int lbm_reduce(lbm_ctx* c, double out[4]) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->has_state) return LBM_ERR_STATE;
  LBM_WITH_STORAGE(c, launch_reduce, c);
  k_reduce_final<<<1, 32, 0, c->stream>>>(c->partial, c->red_blocks, c->red_out);
  LBM_TRY(cudaGetLastError());
  LBM_TRY(cudaMemcpyAsync(c->red_h, c->red_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
  const int st = read_flags(c);
  for (int k = 0; k < 4; ++k) out[k] = c->red_h[k];
  return st;
}

int lbm_sync(lbm_ctx* c) {
  if (!c) return LBM_ERR_ARG;
  return read_flags(c);
}

int lbm_stream_map(lbm_ctx* c, int32_t* map19, int32_t* map7, uint8_t* node_class) {
  if (!c) return LBM_ERR_ARG;
  if (19 * c->N > (1LL << 31) - 1) return LBM_ERR_ARG;
  const long long N = c->N;
  int *m19 = nullptr, *m7 = nullptr;
  unsigned char* cl = nullptr;
  int st = LBM_OK;
  if (map19 && cudaMalloc(&m19, sizeof(int) * 19 * N) != cudaSuccess) st = LBM_ERR_CUDA;
  if (!st && map7 && cudaMalloc(&m7, sizeof(int) * 7 * N) != cudaSuccess) st = LBM_ERR_CUDA;
  if (!st && node_class && cudaMalloc(&cl, N) != cudaSuccess) st = LBM_ERR_CUDA;
  if (!st) {
    k_maps<<<c->grid, kThreads, 0, c->stream>>>(c->P, m19, m7, cl);
    st = cuda_status(cudaGetLastError());
  }
  if (!st && m19) st = cuda_status(cudaMemcpyAsync(map19, m19, sizeof(int) * 19 * N, cudaMemcpyDeviceToHost, c->stream));
  if (!st && m7) st = cuda_status(cudaMemcpyAsync(map7, m7, sizeof(int) * 7 * N, cudaMemcpyDeviceToHost, c->stream));
  if (!st && cl) st = cuda_status(cudaMemcpyAsync(node_class, cl, N, cudaMemcpyDeviceToHost, c->stream));
  if (!st) st = cuda_status(cudaStreamSynchronize(c->stream));
  cudaFree(m19);
  cudaFree(m7);
  cudaFree(cl);
  return st;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  adj_free(c);
  for (int k = 0; k < 2; ++k) {
    cudaFree(c->f[k]);
    cudaFree(c->g[k]);
  }
  cudaFree(c->aux);
  cudaFree(c->hist);
  cudaFree(c->ref);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  cudaFree(c->err_d);
  cudaFreeHost(c->err_h);
  cudaFree(c->partial);
  cudaFree(c->red_out);
  cudaFreeHost(c->red_h);
  for (int f = 0; f < 6; ++f) cudaFree(c->tface[f]);
  fused_free(&c->plan);
  slab_plan_destroy(c->slabs);
  if (c->evs) {
    for (auto& e : *c->evs) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    delete c->evs;
  }
  if (c->pool) {
    for (auto e : *c->pool) cudaEventDestroy(e);
    delete c->pool;
  }
  delete c;
}

}  // extern "C"
