// Host harness for the per-cell phase code of the library (csrc/lbm_phases.cuh):
// the same phase functions, compiled for the host with LBM_HOST_PHASES, run
// over a small lattice in the order of the one-launch-per-phase schedule
// (A for every cell, then force + D3Q19 collide/push, then D3Q7
// collide/push, then the boundary rules on the face nodes), with the
// double-buffered populations in any storage form.  CPU tests compare it with
// the FP64 oracle before any GPU run.  It also exposes the host part of the slab
// pipeline and of the persistent kernel (their stage orders and dependency lists)
// for the CPU checks of their ordering.  Test infrastructure only.
#define LBM_HOST_PHASES
#include "lbm_api.cu"

// the harness never records an adjoint (lbm_adjoint.cu is not linked in)
void adj_free(lbm_ctx*) {}

namespace {

// tface[f] (may be NULL, as may any entry): a per-node Dirichlet temperature of face f, as
// lbm_set_face_T takes it; NULL entries use face_T[f].  mode bit 1: the face rules of every
// step but the last are applied by the next step's phase A (phaseA<ST, true>), as the slab
// schedule does; bit 2: phase A two cells at a time (phaseA2; global 16-bit shifts, even N).
template <typename ST>
int host_run(const lbm_params* hp, const float* f0, const float* g0, int nsteps, float* f_out, float* g_out,
             const float* const* tface_in, int mode = 0) {
  if (check_params(hp) != LBM_OK) return LBM_ERR_ARG;
  Params P = make_device_params(*hp);
  const long long N = P.N;
  std::vector<std::vector<float>> tface(6);
  for (int f = 0; f < 6; ++f)
    if (P.tface[f]) {
      tface[f].assign((size_t)face_len(*hp, f), (float)hp->face_T[f]);
      if (tface_in && tface_in[f])
        for (size_t k = 0; k < tface[f].size(); ++k) tface[f][k] = tface_in[f][k];
      P.Tface[f] = tface[f].data();
    }
  std::vector<ST> fb[2], gb[2];
  for (int k = 0; k < 2; ++k) {
    fb[k].resize((size_t)(19 * N));
    gb[k].resize((size_t)(7 * N));
  }
  std::vector<float> aux((size_t)(11 * N), 0.f);
  std::vector<float2> ref(LocalRef<ST>::on ? (size_t)(2 * N) : 0);
  std::vector<float> hist(hp->vartheta ? (size_t)(2 * N) : 0);  // T(t-1), T(t-2) for vartheta = 1
  float* a = aux.data();
  Aux X = Aux{a, a + N, a + 2 * N, a + 3 * N, a + 4 * N, a + 5 * N, a + 6 * N, a + 7 * N, a + 8 * N, a + 9 * N,
                    a + 10 * N};
  if (hp->vartheta) {
    X.T1 = hist.data();
    X.T2 = hist.data() + N;
  }
  auto refs = [&](int k) -> float2* { return LocalRef<ST>::on ? ref.data() + (size_t)k * N : nullptr; };
  // the state into buffer 0: per-cell references of the state itself (as lbm_set_state)
  for (long long c = 0; c < N; ++c) {
    float r = 0.f, t = 0.f;
    for (int i = 0; i < 19; ++i) r += f0[i * N + c];
    for (int i = 0; i < 7; ++i) t += g0[i * N + c];
    if (LocalRef<ST>::on) refs(0)[c] = make_float2(r, t);
    const float2 rc = LocalRef<ST>::on ? refs(0)[c] : make_float2(0.f, 0.f);
    for (int i = 0; i < 19; ++i) PopStore<ST>::st(&fb[0][i * N + c], f0[i * N + c], fbase_at<ST>(P, i, rc.x));
    for (int i = 0; i < 7; ++i) PopStore<ST>::st(&gb[0][i * N + c], g0[i * N + c], gbase_at<ST>(P, i, rc.y));
  }
  // vartheta = 1: the state is taken to be at rest before, T(t-1) = T(t-2) = sum g as stored
  if (hp->vartheta)
    for (long long c = 0; c < N; ++c) {
      const float t = LocalRef<ST>::on ? refs(0)[c].y : 0.f;
      float gl[7];
      for (int i = 0; i < 7; ++i) gl[i] = PopStore<ST>::ld_plain(&gb[0][i * N + c], gbase_at<ST>(P, i, t));
      X.T1[c] = X.T2[c] = sum7(gl);
    }
  int err = 0, cur = 0;
  for (int s = 0; s < nsteps; ++s) {
    const int A = cur, B = 1 - cur;
    AuxFor<ST> Xs;
    static_cast<Aux&>(Xs) = X;
    if constexpr (LocalRef<ST>::on) {
      Xs.ref_in = refs(A);
      Xs.ref_out = refs(B);
    }
    bool done_a = false;
    if constexpr (!LocalRef<ST>::on) {
      if ((mode & 1) && s > 0) {
        for (long long c = 0; c < N; ++c)
          phaseA<ST, true>(P, (int)c, fb[A].data(), gb[A].data(), Xs, nullptr, err, false);
        done_a = true;
      } else if constexpr (sizeof(ST) == 2) {
        if ((mode & 2) && N % 2 == 0) {
          for (long long c = 0; c < N; c += 2) phaseA2<ST>(P, (int)c, fb[A].data(), gb[A].data(), Xs, err);
          done_a = true;
        }
      }
    }
    if (!done_a)
      for (long long c = 0; c < N; ++c) phaseA<ST>(P, (int)c, fb[A].data(), gb[A].data(), Xs, nullptr, err, false);
    for (long long c = 0; c < N; ++c) phaseBC19<ST>(P, (int)c, fb[A].data(), fb[B].data(), Xs);
    for (long long c = 0; c < N; ++c) {
      if (hp->vartheta)
        phaseC7<ST, 1>(P, (int)c, gb[A].data(), gb[B].data(), Xs);
      else
        phaseC7<ST, 0>(P, (int)c, gb[A].data(), gb[B].data(), Xs);
    }
    const bool fused_next = (mode & 1) && !LocalRef<ST>::on && s < nsteps - 1;
    for (long long k = 0; k < (fused_next ? 0 : P.bd_total); ++k) {
      int x, y, z;
      boundary_candidate(P, (int)k, x, y, z);
      const int m = node_tfaces(P, x, y, z);
      if (m) phaseD<ST>(P, cell_of(P, x, y, z), x, y, z, m, fb[B].data(), gb[B].data(), Xs);
    }
    cur = B;
  }
  for (long long c = 0; c < N; ++c) {
    const float2 rc = LocalRef<ST>::on ? refs(cur)[c] : make_float2(0.f, 0.f);
    for (int i = 0; i < 19; ++i) f_out[i * N + c] = PopStore<ST>::ld_plain(&fb[cur][i * N + c], fbase_at<ST>(P, i, rc.x));
    for (int i = 0; i < 7; ++i) g_out[i * N + c] = PopStore<ST>::ld_plain(&gb[cur][i * N + c], gbase_at<ST>(P, i, rc.y));
  }
  return err;
}

}  // namespace

extern "C" {
// nsteps steps of the lattice hp from the FP32 state (f0, g0) in hp->storage, with the
// per-node face temperatures tface (NULL: the constant face_T);
// returns the phase error flags (ERRF_*) or a negative lbm_status
int h_run(const lbm_params* hp, const float* f0, const float* g0, int nsteps, float* f_out, float* g_out,
          const float* const* tface) {
  switch (hp->storage) {
    case LBM_STORE_F32: return host_run<float>(hp, f0, g0, nsteps, f_out, g_out, tface);
    case LBM_STORE_F16_SHIFTED: return host_run<__half>(hp, f0, g0, nsteps, f_out, g_out, tface);
    case LBM_STORE_BF16_SHIFTED: return host_run<__nv_bfloat16>(hp, f0, g0, nsteps, f_out, g_out, tface);
    case LBM_STORE_F16_LOCAL: return host_run<lhalf>(hp, f0, g0, nsteps, f_out, g_out, tface);
    default: return LBM_ERR_ARG;
  }
}

// h_run with the schedule variants of host_run's mode (1: face rules in the next step's
// phase A; 2: phase A two cells at a time)
int h_run_mode(const lbm_params* hp, const float* f0, const float* g0, int nsteps, float* f_out, float* g_out,
               const float* const* tface, int mode) {
  switch (hp->storage) {
    case LBM_STORE_F32: return host_run<float>(hp, f0, g0, nsteps, f_out, g_out, tface, mode);
    case LBM_STORE_F16_SHIFTED: return host_run<__half>(hp, f0, g0, nsteps, f_out, g_out, tface, mode);
    case LBM_STORE_BF16_SHIFTED: return host_run<__nv_bfloat16>(hp, f0, g0, nsteps, f_out, g_out, tface, mode);
    case LBM_STORE_F16_LOCAL: return host_run<lhalf>(hp, f0, g0, nsteps, f_out, g_out, tface, mode);
    default: return LBM_ERR_ARG;
  }
}
}

extern "C" {
// The slab plan of lattice hp with slabs of about sp planes (the host part of the
// pipelined schedule): *nslab slabs with plane bounds zb[0..nslab], the stage order
// (stage code = phase * nslab + slab; phases A, BC19, C7, D = 0..3), for every stage
// code the stages of the same step it waits for (deps_within, 8 per code, -1 padded),
// and for every slab the stages of the previous step its phase A waits for
// (deps_prev, 8 per slab, -1 padded), and the same when the previous step left its face
// rules to this phase A (deps_prev_fused).  max_slab bounds the arrays: zb holds
// max_slab + 1, order and deps_within 4 * max_slab (x 8), deps_prev and deps_prev_fused
// max_slab x 8.  has_d (max_slab) receives the slabs that hold face nodes.  Returns 0 or -1.
int h_slab_plan(const lbm_params* hp, int sp, int max_slab, int* nslab, int* zb, int* order, int* norder,
                int* deps_within, int* deps_prev, int* deps_prev_fused, int* has_d) {
  if (check_params(hp) != LBM_OK) return -1;
  const Params P = make_device_params(*hp);
  SlabPlan S;
  if (!slab_plan_layout(P, sp, &S) || S.nslab > max_slab) return -1;
  const bool zper = P.face_kind[4] == FACE_PERIODIC;
  *nslab = S.nslab;
  for (int s = 0; s <= S.nslab; ++s) zb[s] = S.zb[s];
  *norder = (int)S.order.size();
  for (size_t k = 0; k < S.order.size(); ++k) order[k] = S.order[k];
  std::vector<int> d;
  for (int code = 0; code < SPH_N * S.nslab; ++code) {
    slab_deps_within(S, zper, code / S.nslab, code % S.nslab, d);
    if (d.size() > 8) return -1;
    for (int k = 0; k < 8; ++k) deps_within[code * 8 + k] = k < (int)d.size() ? d[k] : -1;
  }
  for (int s = 0; s < S.nslab; ++s) {
    slab_deps_prev(S, zper, s, d);
    if (d.size() > 8) return -1;
    for (int k = 0; k < 8; ++k) deps_prev[s * 8 + k] = k < (int)d.size() ? d[k] : -1;
    slab_deps_prev(S, zper, s, d, false);
    if (d.size() > 8) return -1;
    for (int k = 0; k < 8; ++k) deps_prev_fused[s * 8 + k] = k < (int)d.size() ? d[k] : -1;
    has_d[s] = S.has_d[s];
  }
  return 0;
}
}

extern "C" {
// The persistent schedule's stage order for lattice hp with the given gap (stage code =
// phase << 24 | plane, phases A, B, C, D = 0..3) into order (capacity cap); *n receives
// the count.  deps (8 per stage code, -1 padded, indexed phase * nz + plane) lists the
// stage codes each stage waits for.  Returns 0 or -1.
int h_fused_plan(const lbm_params* hp, int gap, int cap, int* order, int* n, int* deps) {
  if (check_params(hp) != LBM_OK) return -1;
  const Params P = make_device_params(*hp);
  const std::vector<int> o = fused_order(P, gap);
  if ((int)o.size() > cap) return -1;
  *n = (int)o.size();
  for (size_t k = 0; k < o.size(); ++k) order[k] = o[k];
  for (int ph = 0; ph < 4; ++ph)
    for (int z = 0; z < P.nz; ++z) {
      int* d = deps + (ph * P.nz + z) * 8;
      int m = 0;
      const int r = dep_radius(ph);
      for (int k = -r; r > 0 && k <= r; ++k) {
        bool valid;
        const int q = dep_plane(P, z, k, valid);
        if (valid && m < 8) d[m++] = ((ph - 1) << 24) | q;
      }
      for (; m < 8; ++m) d[m] = -1;
    }
  return 0;
}
}
