// The phases of one time step, written per cell so that every schedule (one
// launch per phase, per-slab launches, the persistent pipelined kernel, the
// batched kernels, the adjoint's recomputation) runs the same code.
//   A  macro: rho, j = sum c f, T = sum g, p_EOS, psi          (Eqs. 3, 7, 37)
//   B  force: F = -G psi sum varpi psi(x+c) c, u = (j + F/2)/rho (Eqs. 5, 6, 36)
//   C  collide + stream: D3Q19 MRT-EDM collision pushed to x+c (bounce-back at
//      walls), D3Q7 collision with the source pushed with the relaxed streaming
//      (Eqs. 8, 13-15, 27-29, 34)
//   D  boundary: constant-pressure open faces (Sec. 3.3) and non-equilibrium
//      extrapolation of g at Dirichlet nodes (Sec. 3.1), on the new state
// The time-stepping schedules run B inside the D3Q19 part of C (phaseBC19); B
// alone serves lbm_macros and the persistent kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lbm_lattice.cuh"

namespace lbm {

struct Aux {
  float *rho, *jx, *jy, *jz, *psi;  // phase A
  float *Fx, *Fy, *Fz, *ux, *uy, *uz;  // phase B
  float *gstar, *divu;  // optional (NULL): the D3Q7 phase also stores g* (7N) and div u
  float *T1, *T2;       // vartheta = 1: T at the two previous steps, kept by the D3Q7 phase
};

// The scratch of the FP16 storage with per-cell references: (rho_ref, T_ref) of every
// cell for the populations read this step (ref_in) and for those written (ref_out).
// Only that storage form's kernels take it, so the others keep the plain Aux.
struct AuxRef : Aux {
  const float2* ref_in;
  float2* ref_out;
};

// L2 residency: population loads stream through once per kernel (evict-first),
// while the 44 B/cell of scratch written by phases A and B and read by the
// next phases (92 MB at 128^3) is kept (evict-last), so that it is served from
// L2 instead of making a round trip to HBM between kernels.
// FREE: the loads below are plain asm statements, which the compiler may reorder and
// interleave; otherwise they are volatile and keep the order of the source, which the
// kernels were written for (the per-cell-reference D3Q7 kernel is faster with FREE, the
// others without).
template <bool FREE>
struct HintT {
  unsigned long long stream, keep;
};
using Hint = HintT<false>;

template <bool FREE = false>
LBM_DEV HintT<FREE> make_hint() {
  HintT<FREE> h;
#if defined(__CUDA_ARCH__)
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(h.stream));
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(h.keep));
#else
  h.stream = h.keep = 0;  // host harness: no cache policies
#endif
  return h;
}

// Population stores keep the default policy: a push-streamed warp store is shifted
// by one cell for x-moving directions and so covers two sectors partially; evicting
// early would write each sector twice and force an ECC read-modify-write in HBM.
template <bool F>
LBM_DEV void st_pop(float* a, float v, const HintT<F>&) { *a = v; }

#if defined(LBM_NO_L2HINT)
template <bool F>
LBM_DEV float ld_pop(const float* a, const HintT<F>&) {
#if defined(__CUDA_ARCH__)
  return __ldg(a);
#else
  return *a;
#endif
}
template <bool F>
LBM_DEV float ld_aux(const float* a, const HintT<F>&) { return *a; }
template <bool F>
LBM_DEV void st_aux(float* a, float v, const HintT<F>&) { *a = v; }
#else
// populations of the previous time step (read-only during the step)
template <bool F>
LBM_DEV float ld_pop(const float* a, const HintT<F>& h) {
#if defined(__CUDA_ARCH__)
  float v;
  if constexpr (F)
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(h.stream));
  else
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(h.stream));
  return v;
#else
  return *a;
#endif
}

// scratch written and read within the step
template <bool F>
LBM_DEV float ld_aux(const float* a, const HintT<F>& h) {
#if defined(__CUDA_ARCH__)
  float v;
  if constexpr (F)
    asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(h.keep));
  else
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(h.keep));
  return v;
#else
  return *a;
#endif
}
template <bool F>
LBM_DEV void st_aux(float* a, float v, const HintT<F>& h) {
#if defined(__CUDA_ARCH__)
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(h.keep));
#else
  *a = v;
#endif
}
#endif

// Population storage.  FP32 stores f_i itself; the shifted 16-bit forms store
// f_i - w_i rho_ref and g_i - w_i T_ref in IEEE half or bfloat16, and every
// arithmetic operation stays in FP32: decode = base + (float)stored.  With one
// global shift (__half, __nv_bfloat16) rho_ref and T_ref are parameters; with
// per-cell references (lhalf) they are the density and temperature that the
// destination cell had before the step that wrote the population: the pushes
// know them (phase A has stored them), and a later load reads the cell's own.
struct lhalf {
  __half v;
};
static_assert(sizeof(lhalf) == 2, "lhalf is stored as one IEEE half");

template <typename ST>
struct LocalRef {
  static constexpr bool on = false;
};
template <>
struct LocalRef<lhalf> {
  static constexpr bool on = true;
};

template <typename ST>
using AuxFor = typename std::conditional<LocalRef<ST>::on, AuxRef, Aux>::type;

template <typename ST>
struct PopStore;

template <>
struct PopStore<float> {
  template <bool F>
  LBM_DEV static float ld(const float* a, float, const HintT<F>& h) {
    return ld_pop(a, h);
  }
  LBM_DEV static float ld_plain(const float* a, float) { return *a; }
  LBM_DEV static void st(float* a, float v, float) { *a = v; }
  LBM_DEV static float round(float v, float) { return v; }
};

template <bool F>
LBM_DEV unsigned short ld_u16_stream(const void* a, const HintT<F>& h) {
#if defined(__CUDA_ARCH__)
  unsigned short v;
  if constexpr (F)
    asm("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(h.stream));
  else
    asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(h.stream));
  return v;
#else
  return *static_cast<const unsigned short*>(a);
#endif
}

// two neighbouring stored 16-bit populations as one 32-bit word (the lower cell in the low
// half); a must be 4-byte aligned
LBM_DEV unsigned ld_u32_stream(const void* a, const Hint& h) {
#if defined(__CUDA_ARCH__)
  unsigned v;
  asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(h.stream));
  return v;
#else
  (void)h;
  return *static_cast<const unsigned*>(a);
#endif
}

template <>
struct PopStore<__half> {
  template <bool F>
  LBM_DEV static float ld(const __half* a, float base, const HintT<F>& h) {
    return base + __half2float(__ushort_as_half(ld_u16_stream(a, h)));
  }
  // the value of stored bits b
  LBM_DEV static float dec(unsigned short b, float base) { return base + __half2float(__ushort_as_half(b)); }
  LBM_DEV static float ld_plain(const __half* a, float base) { return base + __half2float(*a); }
  LBM_DEV static void st(__half* a, float v, float base) { *a = __float2half_rn(v - base); }
  // the value a later load of st(v) returns
  LBM_DEV static float round(float v, float base) {
    return base + __half2float(__float2half_rn(v - base));
  }
};

template <>
struct PopStore<lhalf> {
  template <bool F>
  LBM_DEV static float ld(const lhalf* a, float base, const HintT<F>& h) {
    return base + __half2float(__ushort_as_half(ld_u16_stream(a, h)));
  }
  LBM_DEV static float ld_plain(const lhalf* a, float base) { return base + __half2float(a->v); }
  LBM_DEV static void st(lhalf* a, float v, float base) { a->v = __float2half_rn(v - base); }
  LBM_DEV static float round(float v, float base) {
    return base + __half2float(__float2half_rn(v - base));
  }
};

template <>
struct PopStore<__nv_bfloat16> {
  template <bool F>
  LBM_DEV static float ld(const __nv_bfloat16* a, float base, const HintT<F>& h) {
    return base + __bfloat162float(__ushort_as_bfloat16(ld_u16_stream(a, h)));
  }
  LBM_DEV static float dec(unsigned short b, float base) {
    return base + __bfloat162float(__ushort_as_bfloat16(b));
  }
  LBM_DEV static float ld_plain(const __nv_bfloat16* a, float base) {
    return base + __bfloat162float(*a);
  }
  LBM_DEV static void st(__nv_bfloat16* a, float v, float base) {
    *a = __float2bfloat16_rn(v - base);
  }
  LBM_DEV static float round(float v, float base) {
    return base + __bfloat162float(__float2bfloat16_rn(v - base));
  }
};

// shift bases of direction i (one global shift)
LBM_DEV float fbase(const Params& P, int i) { return w19(i) * P.rho_ref; }
LBM_DEV float gbase(const Params& P, int i) {
  return (i == 0 ? 1.f - P.wbar : P.wbar * (1.f / 6.f)) * P.T_ref;
}
// shift bases for storage type ST at a cell whose references are r (density) and
// t (temperature); the global shift ignores them
template <typename ST>
LBM_DEV float fbase_at(const Params& P, int i, float r) {
  return LocalRef<ST>::on ? w19(i) * r : fbase(P, i);
}
template <typename ST>
LBM_DEV float gbase_at(const Params& P, int i, float t) {
  return LocalRef<ST>::on ? (i == 0 ? 1.f - P.wbar : P.wbar * (1.f / 6.f)) * t : gbase(P, i);
}
// the references of the populations read (in) or written (out) at cell c, (0, 0)
// when the storage has none
template <typename ST>
LBM_DEV float2 ref_in_at(const AuxFor<ST>& X, long long c) {
  if constexpr (LocalRef<ST>::on)
    return X.ref_in[c];
  else
    return make_float2(0.f, 0.f);
}
template <typename ST>
LBM_DEV float2 ref_out_at(const AuxFor<ST>& X, long long c) {
  if constexpr (LocalRef<ST>::on)
    return X.ref_out[c];
  else
    return make_float2(0.f, 0.f);
}

LBM_DEV void sum19(const float* f, float& rho, float& jx, float& jy, float& jz) {
  rho = ((f[0] + (f[1] + f[2])) + ((f[3] + f[4]) + (f[5] + f[6]))) +
        (((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14]))) + ((f[15] + f[16]) + (f[17] + f[18]));
  jx = ((f[1] - f[2]) + (f[7] - f[8])) + ((f[9] - f[10]) + (f[11] - f[12])) + (f[13] - f[14]);
  jy = ((f[3] - f[4]) + (f[7] - f[8])) + ((f[10] - f[9]) + (f[15] - f[16])) + (f[17] - f[18]);
  jz = ((f[5] - f[6]) + (f[11] - f[12])) + ((f[14] - f[13]) + (f[15] - f[16])) + (f[18] - f[17]);
}

LBM_DEV float sum7(const float* g) {
  return (g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]));
}

LBM_DEV void cell_xyz(const Params& P, int c, int& x, int& y, int& z) {
  const int row = (int)fdiv((unsigned)c, P.dnx_mul, P.dnx_shr);
  x = c - row * P.nx;
  z = (int)fdiv((unsigned)row, P.dny_mul, P.dny_shr);
  y = row - z * P.ny;
}

// Boundary nodes of plane z are enumerated as candidates k = 0..count-1: the
// whole plane when z lies on a z face that holds a Dirichlet temperature, otherwise
// its perimeter rows/columns on such x or y faces (non-periodic faces, and periodic
// faces whose node layer is held).
LBM_DEV bool axis_bounded(const Params& P, int a) { return P.tface[2 * a] || P.tface[2 * a + 1]; }

LBM_DEV int boundary_count(const Params& P, int z) {
  const bool xnp = axis_bounded(P, 0), ynp = axis_bounded(P, 1);
  if (axis_bounded(P, 2) && (z == 0 || z == P.nz - 1)) return P.nx * P.ny;
  if (xnp && ynp) return 2 * P.nx + 2 * (P.ny - 2);
  if (xnp) return 2 * P.ny;
  if (ynp) return 2 * P.nx;
  return 0;
}

LBM_DEV void boundary_xy(const Params& P, int z, int k, int& x, int& y) {
  const bool xnp = axis_bounded(P, 0), ynp = axis_bounded(P, 1);
  if (axis_bounded(P, 2) && (z == 0 || z == P.nz - 1)) {
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

// All boundary nodes of the lattice as one flat index range: the whole planes
// z = 0 and nz-1 when a z face holds a Dirichlet temperature, then the perimeter
// candidates of the other planes.
LBM_DEV void boundary_candidate(const Params& P, int idx, int& x, int& y, int& z) {
  const int plane = P.nx * P.ny;
  int k;
  if (idx < P.bd_zplanes * plane) {
    const int zz = (int)fdiv((unsigned)idx, P.dpl_mul, P.dpl_shr);
    z = zz == 0 ? 0 : P.nz - 1;
    k = idx - zz * plane;
  } else {
    const int j = idx - P.bd_zplanes * plane;
    const int zi = (int)fdiv((unsigned)j, P.dper_mul, P.dper_shr);
    k = j - zi * P.bd_perim;
    z = (P.bd_zplanes ? 1 : 0) + zi;
  }
  boundary_xy(P, z, k, x, y);
}

// ------------------------------------------------------------------- A -----
LBM_DEV float face_T_at(const Params& P, int face, int x, int y, int z) {
  const int a = face >> 1;
  const float* t = P.Tface[face];
  if (a == 0) return t[y + P.ny * z];
  if (a == 1) return t[x + P.nx * z];
  return t[x + P.nx * y];
}

// Unknown D3Q19 directions of a node: those arriving from beyond a non-periodic face.
LBM_DEV unsigned unknown19(const Params& P, int x, int y, int z) {
  unsigned unk = 0;
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int sx = x - c19x(i), sy = y - c19y(i), sz = z - c19z(i);
    const bool u = ((sx < 0 || sx >= P.nx) && P.face_kind[0] != FACE_PERIODIC) ||
                   ((sy < 0 || sy >= P.ny) && P.face_kind[2] != FACE_PERIODIC) ||
                   ((sz < 0 || sz >= P.nz) && P.face_kind[4] != FACE_PERIODIC);
    unk |= (u ? 1u : 0u) << i;
  }
  return unk;
}

// The rules of phase D (constant-pressure open faces, Sec. 3.3; the
// non-equilibrium extrapolation of g, Sec. 3.1) at a face node (m: node_tfaces)
// whose streamed populations are in fl: the rewritten populations are stored (and replaced in
// fl / gl by the values a later load returns).  Every load is issued before the
// first store, so that the node's memory round trips overlap.
template <typename ST>
LBM_DEV void boundary_rules(const Params& P, int c, int x, int y, int z, int m, float* fl,
                                                  float* gl, ST* f, ST* g, const AuxFor<ST>& X) {
  const long long N = P.N;
  int nnp = 0, nvel = 0, nopen = 0, oface = -1;  // faces holding T; of them, non-periodic; open
  float rb = 0.f, Tb = 0.f;
  int q[3] = {x, y, z};
#pragma unroll
  for (int fc = 0; fc < 6; ++fc) {
    if (!((m >> fc) & 1)) continue;
    ++nnp;
    if (P.face_kind[fc] != FACE_PERIODIC) ++nvel;
    if (P.face_kind[fc] == FACE_OPEN) {
      ++nopen;
      oface = fc;
      rb += P.face_rho[fc];
    }
    Tb += face_T_at(P, fc, x, y, z);
    q[fc >> 1] += (fc & 1) ? -1 : 1;
  }
  const int cf = cell_of(P, q[0], q[1], q[2]);
  // references of the new state (written this step) at the inward neighbour and here
  const float2 rf = ref_out_at<ST>(X, cf), rc = ref_out_at<ST>(X, c);
  float gf[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) gf[i] = PopStore<ST>::ld_plain(g + i * N + cf, gbase_at<ST>(P, i, rf.y));
  const float Fx = X.Fx[c], Fy = X.Fy[c], Fz = X.Fz[c];
  if (nopen) {
    // one open face: Zou-He (writes only the unknowns); edges and corners of open
    // faces: every unknown = f^eq(rho_b, 0) = w_i rho_b, rho_b the faces' mean
    const unsigned unk = unknown19(P, x, y, z);
    if (nvel == 1) zouhe(oface, P.face_rho[oface], Fx, Fy, Fz, fl);
    const float rbm = rb / (float)nopen;
#pragma unroll
    for (int i = 1; i < 19; ++i)
      if ((unk >> i) & 1u) {
        const float v = nvel == 1 ? fl[i] : w19(i) * rbm;
        PopStore<ST>::st(f + i * N + c, v, fbase_at<ST>(P, i, rc.x));
        fl[i] = PopStore<ST>::round(v, fbase_at<ST>(P, i, rc.x));
      }
  }
  Tb /= (float)nnp;
  const float Tf = sum7(gf);
  const float w0 = 1.f - P.wbar, w1 = P.wbar * (1.f / 6.f);
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const float w = i == 0 ? w0 : w1;
    const float v = w * Tb + gf[i] - w * Tf;
    PopStore<ST>::st(g + i * N + c, v, gbase_at<ST>(P, i, rc.y));
    gl[i] = PopStore<ST>::round(v, gbase_at<ST>(P, i, rc.y));
  }
}

// The sums, the EOS and psi of one cell whose stored populations are in fl, gl, and the
// stores of phase A (shared by the per-cell and the two-cell forms).
template <typename ST>
LBM_DEV void phaseA_finish(const Params& P, int c, const float* fl, const float* gl, const AuxFor<ST>& X,
                           float* __restrict__ Tout, int& err, bool write_j) {
  const Hint h = make_hint();
  float rho, jx, jy, jz;
  sum19(fl, rho, jx, jy, jz);
  const float T = sum7(gl);
  // the references of the populations this step writes: this state's rho and T
  if constexpr (LocalRef<ST>::on) X.ref_out[c] = make_float2(rho, T);
  if (!isfinite(rho) || !isfinite(T) || !isfinite(jx + jy + jz)) err |= ERRF_NONFINITE;
  float p, dpdT, psi;
  eos_pr(P, rho, T, p, dpdT);
  if (!psi_of(P, rho, p, psi)) err |= ERRF_PSI;
  st_aux(X.rho + c, rho, h);
  if (write_j) {
    st_aux(X.jx + c, jx, h);
    st_aux(X.jy + c, jy, h);
    st_aux(X.jz + c, jz, h);
  }
  st_aux(X.psi + c, psi, h);
  if (Tout) Tout[c] = T;
}

// write_j: store j for phase B (the fused force + D3Q19 pass recomputes it).
// FUSE_D: the state's face rules were not applied by the step that wrote it (the slab
// schedule leaves phase D of every step but the last of a call to the next step's phase A):
// at a face node the rules of phase D (open-face rule, NEE) are applied here to the loaded
// populations, written back to f and g, and the sums of phaseA_finish use the corrected values.  The
// rules read only the node's own populations, its force F and g at its inward neighbour,
// which lies inside along every face normal and is never a face node, so no other thread of
// this pass reads what they write.  Not for per-cell references, whose rules need the
// references of the state being written.
template <typename ST, bool FUSE_D = false>
LBM_DEV void phaseA(const Params& P, int c, const ST* f, const ST* g, const AuxFor<ST>& X,
                    float* __restrict__ Tout, int& err, bool write_j = true) {
  static_assert(!(FUSE_D && LocalRef<ST>::on), "fused face rules need a global storage shift");
  const Hint h = make_hint();
  const float2 rin = ref_in_at<ST>(X, c);
  float fl[19], gl[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) fl[i] = PopStore<ST>::ld(f + i * P.N + c, fbase_at<ST>(P, i, rin.x), h);
#pragma unroll
  for (int i = 0; i < 7; ++i) gl[i] = PopStore<ST>::ld(g + i * P.N + c, gbase_at<ST>(P, i, rin.y), h);
  if constexpr (FUSE_D) {
    int x, y, z;
    cell_xyz(P, c, x, y, z);
    const int m = node_tfaces(P, x, y, z);
    if (m) boundary_rules<ST>(P, c, x, y, z, m, fl, gl, const_cast<ST*>(f), const_cast<ST*>(g), X);
  }
  phaseA_finish<ST>(P, c, fl, gl, X, Tout, err, write_j);
}

// Phase A of the two cells c and c + 1 (c even; N even) with one global storage shift: each
// population pair is one 32-bit load, half the load instructions of two per-cell passes.
template <typename ST>
LBM_DEV void phaseA2(const Params& P, int c, const ST* f, const ST* g, const AuxFor<ST>& X, int& err) {
  static_assert(sizeof(ST) == 2 && !LocalRef<ST>::on, "the two-cell form is for one global 16-bit shift");
  const Hint h = make_hint();
  unsigned wf[19], wg[7];
#pragma unroll
  for (int i = 0; i < 19; ++i) wf[i] = ld_u32_stream(f + i * P.N + c, h);
#pragma unroll
  for (int i = 0; i < 7; ++i) wg[i] = ld_u32_stream(g + i * P.N + c, h);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float fl[19], gl[7];
#pragma unroll
    for (int i = 0; i < 19; ++i)
      fl[i] = PopStore<ST>::dec((unsigned short)(k ? wf[i] >> 16 : wf[i] & 0xffffu), fbase_at<ST>(P, i, 0.f));
#pragma unroll
    for (int i = 0; i < 7; ++i)
      gl[i] = PopStore<ST>::dec((unsigned short)(k ? wg[i] >> 16 : wg[i] & 0xffffu), gbase_at<ST>(P, i, 0.f));
    phaseA_finish<ST>(P, c + k, fl, gl, X, nullptr, err, false);
  }
}

// ------------------------------------------------------------------- B -----
// Wetting term of Eq. 36 is needed only next to a wall face with theta != 90.
LBM_DEV bool needs_wetting(const Params& P, const Nb& nb) {
  bool w = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < 2; ++k) w |= nb.kind[a][k] == FACE_WALL && P.tan_wet[2 * a + k] != 0.f;
  return w;
}

// F = -G psi(x) sum_i varpi_i psi(x + c_i) c_i (Eq. 6), ghost psi beyond the faces
// (INNER: no move of the cell crosses a wall or an open face)
template <bool INNER = false>
LBM_DEV void force_at(const Params& P, int c, int x, int y, int z, const Nb& nb, const Aux& X,
                                         const Hint& h, float& Fx, float& Fy, float& Fz) {
  const float* psi = X.psi;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  if (INNER || !needs_wetting(P, nb)) {
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const float v = varpi19(i) * ld_aux(psi + c + nbo_psi<INNER>(nb, c19x(i), c19y(i), c19z(i)), h);
      if (c19x(i)) sx += c19x(i) * v;  // zero components skipped (0 * v is not folded away)
      if (c19y(i)) sy += c19y(i) * v;
      if (c19z(i)) sz += c19z(i) * v;
    }
  } else {
    for (int i = 1; i < 19; ++i) {
      const float v = varpi19(i) * psi_ext(P, psi, x + c19x(i), y + c19y(i), z + c19z(i));
      if (c19x(i)) sx += c19x(i) * v;  // zero components skipped (0 * v is not folded away)
      if (c19y(i)) sy += c19y(i) * v;
      if (c19z(i)) sz += c19z(i) * v;
    }
  }
  const float k = -P.G * ld_aux(psi + c, h);
  Fx = k * sx;
  Fy = k * sy;
  Fz = k * sz;
}

LBM_DEV void phaseB(const Params& P, int c, const Aux& X) {
  int x, y, z;
  cell_xyz(P, c, x, y, z);
  Nb nb;
  make_nb(P, x, y, z, nb);
  const Hint h = make_hint();
  float Fx, Fy, Fz;
  force_at(P, c, x, y, z, nb, X, h, Fx, Fy, Fz);
  st_aux(X.Fx + c, Fx, h);
  st_aux(X.Fy + c, Fy, h);
  st_aux(X.Fz + c, Fz, h);
  const int m = P.any_nonperiodic ? node_faces(P, x, y, z) : 0;
  float ux = 0.f, uy = 0.f, uz = 0.f;
  if (!(m && on_wall(P, m))) {
    const float ir = rcp(ld_aux(X.rho + c, h));
    ux = (ld_aux(X.jx + c, h) + 0.5f * Fx) * ir;
    uy = (ld_aux(X.jy + c, h) + 0.5f * Fy) * ir;
    uz = (ld_aux(X.jz + c, h) + 0.5f * Fz) * ir;
  }
  st_aux(X.ux + c, ux, h);
  st_aux(X.uy + c, uy, h);
  st_aux(X.uz + c, uz, h);
}

// ------------------------------------------------------------------- C -----
// Phase C, D3Q19 part, for one cell whose pre-collision populations are in fl:
// collision with the exact-difference forcing, push streaming, bounce-back.
template <typename ST>
LBM_DEV void phaseC19_cell(const Params& P, int c, const float* fl, ST* fB, const AuxFor<ST>& X) {
  int x, y, z;
  cell_xyz(P, c, x, y, z);
  Nb nb;
  make_nb(P, x, y, z, nb);
  const long long N = P.N;
  const Hint h = make_hint();
  const float Fx = ld_aux(X.Fx + c, h), Fy = ld_aux(X.Fy + c, h), Fz = ld_aux(X.Fz + c, h);
  float rho, jx, jy, jz;
  sum19(fl, rho, jx, jy, jz);
  const int m = P.any_nonperiodic ? node_faces(P, x, y, z) : 0;
  const bool wall = m && on_wall(P, m);
  const float ir = rcp(rho);
  float ux = jx * ir, uy = jy * ir, uz = jz * ir;
  if (wall && P.wall_ueq_zero) ux = uy = uz = 0.f;
  float fs[19];
  if (P.fast19)
    collide19_fast(P, fl, rho, ux, uy, uz, Fx, Fy, Fz, fs);
  else
    collide19(P, fl, rho, ux, uy, uz, Fx, Fy, Fz, fs);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int k = nb_kind(nb, c19x(i), c19y(i), c19z(i));
    if (k == 0) {
      const int d = c + nb_off(nb, c19x(i), c19y(i), c19z(i));
      // per-cell references: the destination's rho of this step (phase A stored it)
      const float r = LocalRef<ST>::on ? ld_aux(X.rho + d, h) : 0.f;
      PopStore<ST>::st(fB + i * N + d, fs[i], fbase_at<ST>(P, i, r));
    } else if (k & FACE_WALL) {
      const float r = LocalRef<ST>::on ? ld_aux(X.rho + c, h) : 0.f;
      PopStore<ST>::st(fB + opp19(i) * N + c, fs[i], fbase_at<ST>(P, opp19(i), r));  // modified bounce-back
    }
    // else: leaves through an open face
  }
}

// Phases B and C19 of one cell in one pass: the force from the psi stencil, the
// real velocity (both stored for the D3Q7 phase and the next step's open faces),
// then the D3Q19 collision and push of phaseC19_cell.  INNER: no move of the cell
// crosses a wall or an open face (periodic faces only wrap the offsets).
// STAGED: the cell's stored populations are read from sf[i * kStaged] (a tile staged in
// shared memory) instead of fA.
constexpr int kStaged = 256;
template <typename ST, bool INNER, bool STAGED>
LBM_DEV void phaseBC19_body(const Params& P, int c, int x, int y, int z, const ST* __restrict__ fA, ST* fB,
                            const AuxFor<ST>& X, const ST* sf) {
  Nb nb;
  if (INNER)
    make_nb_inner(P, x, nb);
  else
    make_nb(P, x, y, z, nb);
  const long long N = P.N;
  const Hint h = make_hint();
  // the populations first (they come from HBM), so that their latency overlaps the
  // psi stencil of the force (mostly served by L1 and L2)
  const float rin = ref_in_at<ST>(X, c).x;
  float fl[19];
  if constexpr (STAGED) {
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = PopStore<ST>::ld_plain(sf + i * kStaged, fbase_at<ST>(P, i, rin));
  } else {
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = PopStore<ST>::ld(fA + i * N + c, fbase_at<ST>(P, i, rin), h);
  }
  float Fx, Fy, Fz;
  force_at<INNER>(P, c, x, y, z, nb, X, h, Fx, Fy, Fz);
  // F is read again only by the open-face rule at face nodes (never in an interior warp)
  // and by the adjoint, whose recomputed steps pass the g* slot
  if (!INNER || X.gstar) {
    st_aux(X.Fx + c, Fx, h);
    st_aux(X.Fy + c, Fy, h);
    st_aux(X.Fz + c, Fz, h);
  }
  float rho, jx, jy, jz;
  sum19(fl, rho, jx, jy, jz);
  const int m = (!INNER && P.any_nonperiodic) ? node_faces(P, x, y, z) : 0;
  const bool wall = m && on_wall(P, m);
  const float ir = rcp(rho);
  float vx = 0.f, vy = 0.f, vz = 0.f;
  if (!wall) {
    vx = (jx + 0.5f * Fx) * ir;
    vy = (jy + 0.5f * Fy) * ir;
    vz = (jz + 0.5f * Fz) * ir;
  }
  st_aux(X.ux + c, vx, h);
  st_aux(X.uy + c, vy, h);
  st_aux(X.uz + c, vz, h);
  float ux = jx * ir, uy = jy * ir, uz = jz * ir;
  if (wall && P.wall_ueq_zero) ux = uy = uz = 0.f;
  float fs[19];
  if (P.fast19)
    collide19_fast(P, fl, rho, ux, uy, uz, Fx, Fy, Fz, fs);
  else
    collide19(P, fl, rho, ux, uy, uz, Fx, Fy, Fz, fs);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int k = nbk<INNER>(nb, c19x(i), c19y(i), c19z(i));
    if (k == 0) {
      const int d = c + nb_off(nb, c19x(i), c19y(i), c19z(i));
      // per-cell references: the destination's rho of this step (phase A stored it)
      const float r = LocalRef<ST>::on ? ld_aux(X.rho + d, h) : 0.f;
      PopStore<ST>::st(fB + i * N + d, fs[i], fbase_at<ST>(P, i, r));
    } else if (k & FACE_WALL) {
      const float r = LocalRef<ST>::on ? ld_aux(X.rho + c, h) : 0.f;
      PopStore<ST>::st(fB + opp19(i) * N + c, fs[i], fbase_at<ST>(P, opp19(i), r));  // modified bounce-back
    }
  }
}

// The force + D3Q19 pass of one cell: warps none of whose cells crosses a wall or an open
// face take the interior form (the same arithmetic without the face rules).
template <typename ST, bool STAGED = false>
LBM_DEV void phaseBC19(const Params& P, int c, int x, int y, int z, const ST* __restrict__ fA, ST* fB,
                       const AuxFor<ST>& X, const ST* sf = nullptr) {
  if (warp_all(inner_cell(P, x, y, z)))
    phaseBC19_body<ST, true, STAGED>(P, c, x, y, z, fA, fB, X, sf);
  else
    phaseBC19_body<ST, false, STAGED>(P, c, x, y, z, fA, fB, X, sf);
}
template <typename ST>
LBM_DEV void phaseBC19(const Params& P, int c, const ST* __restrict__ fA, ST* fB, const AuxFor<ST>& X) {
  int x, y, z;
  cell_xyz(P, c, x, y, z);
  phaseBC19<ST, false>(P, c, x, y, z, fA, fB, X);
}

// div u = 3 sum_i w_i c_i . u(x + c_i): the isotropic D3Q19 difference of the
// real velocity (zero beyond a wall, the boundary node's value beyond an open face).
template <bool INNER = false, bool F = false>
LBM_DEV float divu_at(const Params& P, int c, const Nb& nb, const Aux& X, const HintT<F>& h) {
  float du = 0.f;
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int k = nbk<INNER>(nb, c19x(i), c19y(i), c19z(i));
    if (k & FACE_WALL) continue;  // zero velocity beyond a wall
    const int n = c + nb_off(nb, c19x(i), c19y(i), c19z(i));
    float s = 0.f;
    if (c19x(i)) s += c19x(i) * ld_aux(X.ux + n, h);
    if (c19y(i)) s += c19y(i) * ld_aux(X.uy + n, h);
    if (c19z(i)) s += c19z(i) * ld_aux(X.uz + n, h);
    du += w19(i) * s;
  }
  return du * 3.f;
}

// Phase C, D3Q7 part: div u by the isotropic D3Q19 difference, grad T from the
// local moments, collision with the source, relaxed push streaming.  rho and the
// real velocity of the cell come from phases A and B.
// VT: vartheta known at compile time (0 or 1), or -1 to read it from P.  INNER: no move
// of the cell crosses a wall or an open face.
template <typename ST, int VT, bool INNER>
LBM_DEV void phaseC7_body(const Params& P, int c, int x, int y, int z, const float* gl, const ST* __restrict__ gA,
                          ST* gB, const AuxFor<ST>& X) {
  const bool vt = VT < 0 ? P.vartheta != 0 : VT != 0;
  Nb nb;
  if (INNER)
    make_nb_inner(P, x, nb);
  else
    make_nb(P, x, y, z, nb);
  const long long N = P.N;
  const auto h = make_hint<LocalRef<ST>::on>();
  // the destinations' g_i and rho of the relaxed streaming, loaded first so that
  // their latency overlaps the stencil and the collision (a move beyond a
  // non-periodic face reads the cell itself and stores nothing)
  // (per-cell references: g_i(y) decodes with y's reference of the state read and is
  // encoded with y's reference of this step, (rho, T)(y) as phase A stored them)
  float gold[7], ry[7], ty[7];
  int yc[7];
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    const bool ok = nbk<INNER>(nb, c7x(i), c7y(i), c7z(i)) == 0;
    yc[i] = c + (ok ? nb_off(nb, c7x(i), c7y(i), c7z(i)) : 0);
    gold[i] = PopStore<ST>::ld(gA + i * N + yc[i], gbase_at<ST>(P, i, ref_in_at<ST>(X, yc[i]).y), h);
    if constexpr (LocalRef<ST>::on) {
      const float2 ro = X.ref_out[yc[i]];
      ry[i] = ok ? ro.x : 0.f;
      ty[i] = ro.y;
    } else {
      ry[i] = ok ? ld_aux(X.rho + yc[i], h) : 0.f;
      ty[i] = 0.f;
    }
  }
  const float2 rc = ref_out_at<ST>(X, c);
  const float rho = LocalRef<ST>::on ? rc.x : ld_aux(X.rho + c, h);
  const float T = sum7(gl);
  // vartheta = 1: d^2T/dt^2 as the backward difference T - 2 T(t-1) + T(t-2); the cell's
  // history moves on by one step after the populations are stored
  float d2T = 0.f, T1 = 0.f;
  if (vt) {
    T1 = X.T1[c];
    d2T = T - 2.f * T1 + X.T2[c];
  }
  const float du = divu_at<INNER>(P, c, nb, X, h);
  float p, dpdT;
  eos_pr(P, rho, T, p, dpdT);
  float gs[7];
  collide7<float, VT>(P, gl, rho, T, ld_aux(X.ux + c, h), ld_aux(X.uy + c, h), ld_aux(X.uz + c, h), du, dpdT, d2T,
                      gs);
  if (X.gstar) {  // kept for the adjoint's recomputed steps
    X.divu[c] = du;
#pragma unroll
    for (int i = 0; i < 7; ++i) X.gstar[i * N + c] = gs[i];
  }
  // relaxed streaming: g_i(y) += (g*_i(y - c_i) - g_i(y)) / (rho(y) c_v)
  PopStore<ST>::st(gB + c, gl[0] + (gs[0] - gl[0]) * rcp(rho * P.cv), gbase_at<ST>(P, 0, rc.y));
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    if (nbk<INNER>(nb, c7x(i), c7y(i), c7z(i))) continue;
    PopStore<ST>::st(gB + i * N + yc[i], gold[i] + (gs[i] - gold[i]) * rcp(ry[i] * P.cv), gbase_at<ST>(P, i, ty[i]));
  }
  if (vt) {
    X.T2[c] = T1;
    X.T1[c] = T;
  }
}

// The D3Q7 pass of one cell: warps none of whose cells crosses a wall or an open face
// take the interior form.
template <typename ST, int VT = -1>
LBM_DEV void phaseC7_cell(const Params& P, int c, const float* gl, const ST* __restrict__ gA, ST* gB,
                                             const AuxFor<ST>& X) {
  int x, y, z;
  cell_xyz(P, c, x, y, z);
  if (warp_all(inner_cell(P, x, y, z)))
    phaseC7_body<ST, VT, true>(P, c, x, y, z, gl, gA, gB, X);
  else
    phaseC7_body<ST, VT, false>(P, c, x, y, z, gl, gA, gB, X);
}

template <typename ST>
LBM_DEV void phaseC_cell(const Params& P, int c, const float* fl, const float* gl,
                                            const ST* __restrict__ gA, ST* fB, ST* gB, const AuxFor<ST>& X) {
  phaseC19_cell<ST>(P, c, fl, fB, X);
  phaseC7_cell<ST>(P, c, gl, gA, gB, X);
}

template <typename ST>
LBM_DEV void phaseC19(const Params& P, int c, const ST* __restrict__ fA, ST* fB, const AuxFor<ST>& X) {
  const long long N = P.N;
  const Hint h = make_hint();
  const float rin = ref_in_at<ST>(X, c).x;
  float fl[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) fl[i] = PopStore<ST>::ld(fA + i * N + c, fbase_at<ST>(P, i, rin), h);
  phaseC19_cell<ST>(P, c, fl, fB, X);
}

template <typename ST, int VT = -1>
LBM_DEV void phaseC7(const Params& P, int c, const ST* __restrict__ gA, ST* gB, const AuxFor<ST>& X) {
  const long long N = P.N;
  const auto h = make_hint<LocalRef<ST>::on>();
  const float tin = ref_in_at<ST>(X, c).y;
  float gl[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) gl[i] = PopStore<ST>::ld(gA + i * N + c, gbase_at<ST>(P, i, tin), h);
  phaseC7_cell<ST, VT>(P, c, gl, gA, gB, X);
}

// phaseC7 with the cell's 7 stored populations read from sg[i * kStaged] (a staged tile)
template <typename ST, int VT>
LBM_DEV void phaseC7_staged(const Params& P, int c, int x, int y, int z, const ST* sg, const ST* __restrict__ gA,
                            ST* gB, const AuxFor<ST>& X) {
  const float tin = ref_in_at<ST>(X, c).y;
  float gl[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) gl[i] = PopStore<ST>::ld_plain(sg + i * kStaged, gbase_at<ST>(P, i, tin));
  if (warp_all(inner_cell(P, x, y, z)))
    phaseC7_body<ST, VT, true>(P, c, x, y, z, gl, gA, gB, X);
  else
    phaseC7_body<ST, VT, false>(P, c, x, y, z, gl, gA, gB, X);
}

template <typename ST>
LBM_DEV void phaseC(const Params& P, int c, const ST* __restrict__ fA, const ST* __restrict__ gA,
                                       ST* fB, ST* gB, const AuxFor<ST>& X) {
  phaseC19<ST>(P, c, fA, fB, X);
  phaseC7<ST>(P, c, gA, gB, X);
}

// ------------------------------------------------------------------- D -----
template <typename ST>
LBM_DEV void phaseD(const Params& P, int c, int x, int y, int z, int m, ST* fB, ST* gB,
                                       const AuxFor<ST>& X) {
  const long long N = P.N;
  float fl[19], gl[7];
  // only the open-face rule reads f, and only its known populations
  const unsigned skip = on_open(P, m) ? unknown19(P, x, y, z) : 0x7ffffu;
  const float rout = ref_out_at<ST>(X, c).x;  // the state written this step
#pragma unroll
  for (int i = 0; i < 19; ++i)
    fl[i] = ((skip >> i) & 1u) ? 0.f : PopStore<ST>::ld_plain(fB + i * N + c, fbase_at<ST>(P, i, rout));
  boundary_rules<ST>(P, c, x, y, z, m, fl, gl, fB, gB, X);
}

}  // namespace lbm
