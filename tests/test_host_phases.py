"""CPU run of the library's per-cell phase code against the FP64 oracle.

tests/harness/step_harness.cu compiles csrc/lbm_phases.cuh for the host (LBM_HOST_PHASES)
and runs whole steps over small lattices in the order of the one-launch-per-phase
schedule: phase A for every cell, then force + D3Q19 collide/push, then D3Q7
collide/push, then the boundary rules on the face nodes, with double-buffered
populations in each storage form.  Index, boundary and storage mistakes in the
kernels' code therefore show up without a GPU.  The arithmetic differs from the
GPU's only in the reciprocals (a correctly rounded division here, the fast
intrinsic there) and in the contraction of multiply-adds, so the FP32 tolerance
of the GPU parity tests applies.

The same harness exposes the host part of the two pipelined schedules (the slab
plan and the persistent kernel's stage order), whose ordering of conflicting
stages is checked at the end of this file.
"""
import ctypes as ct

import numpy as np
import pytest

import harness_build
from cases import (CASES, HALF_ULP, STORAGES_16, W7, _face_nodes, _local_refs, _storage_bound_ok, case_params,
                   droplet_state, f32, pop_err)
from oracle import Oracle
from paper_2206_00946_gb300 import lbm, workloads as W


@pytest.fixture(scope="module")
def H():
    if not harness_build.nvcc():
        pytest.skip("nvcc not available")
    L = ct.CDLL(harness_build.build_harness("step_harness", ("-gencode", "arch=compute_103a,code=sm_103a")))
    L.h_run.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    L.h_run_mode.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                             ct.c_int]
    return L


def host_run(H, p, f, g, n, tface=None, mode=0):
    """n steps of the phase code on the host (one-launch-per-phase order); n = 0 returns the state as
    stored.  tface: {face: per-node temperatures} as lbm_set_face_T takes them.  mode 1: the face
    rules of every step but the last applied by the next step's phase A (the slab schedule's
    fused sequences); mode 2: phase A two cells at a time (the global 16-bit shifts)."""
    P = lbm.make_params(dict(p, schedule=lbm.SCHED_PHASES))
    f, g = f32(f), f32(g)
    fo, go = np.empty_like(f), np.empty_like(g)
    keep = {k: f32(v).reshape(-1) for k, v in (tface or {}).items()}
    tf = (ct.c_void_p * 6)(*[keep[k].ctypes.data if k in keep else None for k in range(6)])
    err = H.h_run_mode(ct.byref(P), f.ctypes.data, g.ctypes.data, n, fo.ctypes.data, go.ctypes.data, tf, mode)
    assert err == 0, err
    return fo, go


@pytest.mark.parametrize("storage", [lbm.STORE_F32, lbm.STORE_F16_SHIFTED, lbm.STORE_BF16_SHIFTED])
@pytest.mark.parametrize("name", ["open_all", "wall_bottom_open_top", "walls_xy_theta", "ragged_open_x",
                                  "periodic_held_T"])
def test_fused_face_rules_and_two_cell_phase_a_are_the_same_step(H, name, storage, thermo):
    """Three steps with the face rules of the first two applied by the next step's phase A, and
    with phase A two cells at a time, give the same bits as three complete steps."""
    p = dict(case_params(name, thermo), storage=storage)
    # a smooth vapour state (random states with open faces leave the psi domain within steps)
    x, y, z = W.grid(p["nx"], p["ny"], p["nz"])
    r2 = (x - 0.45 * p["nx"]) ** 2 + (y - 0.55 * p["ny"]) ** 2 + (z - 0.5 * p["nz"]) ** 2
    rho0 = W.perturb(thermo["rho_v"] * (1.0 + 0.03 * np.exp(-r2 / 4.0)), 1e-3, seed=21)
    T0 = thermo["Ts"] * (1 + 0.01 * np.sin(0.7 * x + 0.5 * y + 0.3 * z))
    f, g = Oracle(p).init_state(rho0, T0)
    f0, g0 = host_run(H, p, f, g, 3)
    f1, g1 = host_run(H, p, f, g, 3, mode=1)
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    f2, g2 = host_run(H, p, f, g, 3, mode=2)
    assert np.array_equal(f0, f2) and np.array_equal(g0, g2)


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_populations_match_oracle(H, name, thermo):
    p = case_params(name, thermo)
    f, g = droplet_state(p, thermo, seed=11)
    st_o, fo, go = Oracle(p).step(f.astype(np.float64), g.astype(np.float64))
    assert st_o == 0
    fh, gh = host_run(H, p, f, g, 1)
    assert pop_err(fh, fo, thermo) < 1e-5
    assert pop_err(gh, go, thermo) < 1e-5


def test_per_node_face_temperature_field(H, thermo):
    """A per-node temperature on the bottom wall (as lbm_set_face_T gives it) against the
    oracle given the same field."""
    p = case_params("wall_bottom_open_top", thermo)
    f, g = droplet_state(p, thermo, seed=13)
    tz = thermo["Ts"] * (1.05 + 0.01 * W.uniform(3, p["nx"] * p["ny"]).reshape(p["ny"], p["nx"]))
    o = Oracle(p)
    o.set_face_T([None, None, None, None, f32(tz).astype(np.float64), None])
    _, fo, go = o.step(f.astype(np.float64), g.astype(np.float64))
    fh, gh = host_run(H, p, f, g, 1, tface={4: tz})
    assert pop_err(gh, go, thermo) < 1e-5 and pop_err(fh, fo, thermo) < 1e-5


# the general moment-space collision (rates other than s_q = s_pi = 1, or the printed m^eq rows)
@pytest.mark.parametrize("rates", [dict(s_q=1.1, s_pi=0.9), dict(meq_printed=1), dict(s_q=0.7, s_pi=1.3, s_e=0.9)])
@pytest.mark.parametrize("name", ["open_all", "walls_z", "periodic"])
def test_one_step_general_collision_matches_oracle(H, name, rates, thermo):
    p = dict(case_params(name, thermo), **rates)
    f, g = droplet_state(p, thermo, seed=13)
    st_o, fo, go = Oracle(p).step(f.astype(np.float64), g.astype(np.float64))
    assert st_o == 0
    fh, gh = host_run(H, p, f, g, 1)
    assert pop_err(fh, fo, thermo) < 1e-5
    assert pop_err(gh, go, thermo) < 1e-5


@pytest.mark.parametrize("storage", STORAGES_16)
@pytest.mark.parametrize("name", ["periodic", "open_all", "wall_bottom_open_top", "walls_xy_theta", "ragged_open_x"])
def test_16bit_storage_one_step_within_half_ulp(H, name, storage, thermo):
    """As the GPU test of the same name: one step from the stored state is within half an ulp
    of the stored deviations of the oracle's step (per-cell shifts for STORE_F16_LOCAL)."""
    p = case_params(name, thermo)
    rho_ref, T_ref = 0.8 * thermo["rho_v"], thermo["Ts"]
    p.update(storage=storage, store_rho_ref=rho_ref, store_T_ref=T_ref)
    f, g = droplet_state(p, thermo, seed=11)
    fq, gq = host_run(H, p, f, g, 0)
    fh, gh = host_run(H, p, f, g, 1)
    st_o, fo, go = Oracle(p).step(fq.astype(np.float64), gq.astype(np.float64))
    assert st_o == 0
    face = _face_nodes(p)
    fref, gref = (_local_refs(fq, gq) if storage == lbm.STORE_F16_LOCAL else (W.W19 * rho_ref, W7 * T_ref))
    ex_f, rel_f = _storage_bound_ok(fh, fo, fref, HALF_ULP[storage], thermo, face)
    ex_g, rel_g = _storage_bound_ok(gh, go, gref, HALF_ULP[storage], thermo, face)
    assert ex_f <= 0 and ex_g <= 0, (rel_f, rel_g)


@pytest.mark.parametrize("storage", [lbm.STORE_F32, lbm.STORE_F16_LOCAL])
@pytest.mark.parametrize("name", ["walls_z", "open_all", "wall_bottom_open_top", "periodic"])
def test_vartheta_one_steps_match_oracle(H, name, storage, thermo):
    """The D3Q7 phase with the correction of Eq. 16 (vartheta = 1): three steps of a vapour
    density bump with a 1 % temperature wave, the state taken to be at rest before, against
    the oracle given the same history.  FP32 within the one-step tolerance; FP16 with
    per-cell references within its storage rounding over three steps, with the bounds of
    the GPU test of the 16-bit forms (next to the open faces the stored deviations of f
    reach about 10 % of f, so 2^-11 of that per step: measured 1.3e-4 on f)."""
    p = dict(case_params(name, thermo), vartheta=1, storage=storage)
    x, y, z = W.grid(p["nx"], p["ny"], p["nz"])
    r2 = (x - 0.45 * p["nx"]) ** 2 + (y - 0.55 * p["ny"]) ** 2 + (z - 0.5 * p["nz"]) ** 2
    rho0 = W.perturb(thermo["rho_v"] * (1.0 + 0.03 * np.exp(-r2 / 4.0)), 1e-3, seed=12)
    T0 = thermo["Ts"] * (1 + 0.01 * np.sin(0.7 * x + 0.5 * y + 0.3 * z))
    o = Oracle(p)
    f, g = o.init_state(rho0, T0)
    f, g = f32(f), f32(g)
    fq, gq = host_run(H, p, f, g, 0)
    st_o, fo, go, _ = o.run_hist(fq.astype(np.float64), gq.astype(np.float64), o.history(gq.astype(np.float64)), 3)
    assert st_o == 0
    _, f0, g0 = Oracle(dict(p, vartheta=0)).run(fq.astype(np.float64), gq.astype(np.float64), 3)
    assert pop_err(g0, go, thermo) > 1e-4  # the correction matters at this tolerance
    fh, gh = host_run(H, p, f, g, 3)
    tf, tg = (1e-5, 1e-5) if storage == lbm.STORE_F32 else (5e-4, 1e-4)
    ef, eg = pop_err(fh, fo, thermo), pop_err(gh, go, thermo)
    assert ef < tf and eg < tg, (ef, eg)


def test_per_cell_references_cut_the_fp16_error(H, thermo):
    """300 steps of the evaporating 20^3 droplet (open faces) from the FP32 initial state,
    against the oracle.  Measured on the host: FP32 1.5e-5 (max relative rho); FP16 with one
    global shift 3.4e-3 / 7.5e-4 (rho / T), relative L2 1.2e-3 on rho; FP16 with per-cell
    references 2.4e-4 / 4.0e-5, L2 6.3e-5: the per-cell references make the stored
    deviations the change of a cell over one step plus its non-equilibrium part."""
    p, rho0, T0 = W.droplet(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], n=20, R=5.0, W=3.0, seed=2206)
    o = Oracle(p)
    f0, g0 = o.init_state(rho0, T0)
    f0, g0 = f32(f0), f32(g0)
    st, fo, go = o.run(f0.astype(np.float64), g0.astype(np.float64), 300)
    assert st == 0
    rho_o, T_o = fo.sum(0), go.sum(0)

    def errors(storage):
        fh, gh = host_run(H, dict(p, storage=storage), f0, g0, 300)
        rho, T = fh.sum(0).astype(np.float64), gh.sum(0).astype(np.float64)
        return (float(np.max(np.abs(rho - rho_o) / rho_o)), float(np.max(np.abs(T - T_o) / T_o)),
                float(np.linalg.norm(rho - rho_o) / np.linalg.norm(rho_o)))

    e32 = errors(lbm.STORE_F32)
    eg = errors(lbm.STORE_F16_SHIFTED)
    el = errors(lbm.STORE_F16_LOCAL)
    print(f"300 droplet steps, max rho / max T / L2 rho: FP32 {e32}, FP16 global {eg}, FP16 per-cell {el}")
    assert e32[0] < 1e-4
    assert el[0] < 1e-3 and el[1] < 2e-4 and el[2] < 2.5e-4
    assert eg[0] > 1e-3 and el[2] < eg[2] / 5


@pytest.mark.slow
def test_per_cell_references_meet_1e3_on_the_slab(H, thermo):
    """1000 steps of the 16x16x64 flat slab between bounce-back walls (bottom T_s + 0.02 T_c),
    from the state as stored, against the oracle.  Measured on the host: FP16 with per-cell
    references 1.6e-3 / 4.8e-5 (max relative rho / T) and 2.7e-4 / 1.4e-5 (relative L2); one
    global shift 2.1e-2 / 2.4e-3 and 3.8e-3 / 9.6e-4.  Per-cell references bring both fields
    within 1e-3 in the relative L2 norm; the global shift does not."""
    p, rho0, T0 = W.slab(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], nx=16, ny=16, nz=64)
    rho0 = W.perturb(rho0, 1e-3, seed=5)
    o = Oracle(p)
    f0, g0 = o.init_state(rho0, T0)
    f0, g0 = f32(f0), f32(g0)

    def l2(storage):
        q = dict(p, storage=storage)
        fq, gq = host_run(H, q, f0, g0, 0)
        st, fo, go = o.run(fq.astype(np.float64), gq.astype(np.float64), 1000)
        assert st == 0
        fh, gh = host_run(H, q, f0, g0, 1000)
        rho, T = fh.sum(0).astype(np.float64), gh.sum(0).astype(np.float64)
        return (float(np.linalg.norm(rho - fo.sum(0)) / np.linalg.norm(fo.sum(0))),
                float(np.linalg.norm(T - go.sum(0)) / np.linalg.norm(go.sum(0))))

    el, eg = l2(lbm.STORE_F16_LOCAL), l2(lbm.STORE_F16_SHIFTED)
    print(f"1000 slab steps, relative L2 rho / T: FP16 per-cell {el}, FP16 global {eg}")
    assert el[0] < 1e-3 and el[1] < 1e-4
    assert eg[0] > 1e-3


# ------------------------------------------------------- slab pipeline order --
# The slab schedule runs every phase per z-slab on several streams; a stage waits
# for other stages only through the dependency lists of the plan (and through the
# order of its own stream).  This replays two consecutive steps of the plan the
# library builds and checks, against the planes each phase kernel reads and writes,
# that every pair of conflicting stages is ordered.

A_, BC19_, C7_, D_ = 0, 1, 2, 3
N_STREAMS = 8  # the default number of slab streams; slab s runs on stream s % 8


def slab_plan(H, p, sp, max_slab=64):
    P = lbm.make_params(dict(p, schedule=lbm.SCHED_SLABS))
    nslab, norder = ct.c_int(), ct.c_int()
    zb = np.zeros(max_slab + 1, np.int32)
    order = np.zeros(4 * max_slab, np.int32)
    dw = np.zeros(4 * max_slab * 8, np.int32)
    dp = np.zeros(max_slab * 8, np.int32)
    dpf = np.zeros(max_slab * 8, np.int32)
    hd = np.zeros(max_slab, np.int32)
    H.h_slab_plan.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                              ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    assert H.h_slab_plan(ct.byref(P), sp, max_slab, ct.byref(nslab), zb.ctypes.data, order.ctypes.data,
                         ct.byref(norder), dw.ctypes.data, dp.ctypes.data, dpf.ctypes.data, hd.ctypes.data) == 0
    n = nslab.value
    within = {c: [q for q in dw[c * 8:(c + 1) * 8] if q >= 0] for c in range(4 * n)}
    prev = {s: [q for q in dp[s * 8:(s + 1) * 8] if q >= 0] for s in range(n)}
    prev_fused = {s: [q for q in dpf[s * 8:(s + 1) * 8] if q >= 0] for s in range(n)}
    slab_plan.fused = (prev_fused, [bool(h) for h in hd[:n]])
    return n, list(zb[:n + 1]), list(order[:norder.value]), within, prev


def stage_access(ph, s, t, zb, nz, zper, fused=False):
    """(resource, mode, planes) of stage (phase ph, slab s) in step t: what its kernel reads ('r')
    and writes ('w').  'p' marks the writes of the streaming pushes: every (direction,
    destination) has exactly one source cell, so two pushes never write the same element.
    Buffers by absolute index: step t reads populations a = t % 2 and writes b."""
    a, b = t % 2, 1 - t % 2
    own = set(range(zb[s], zb[s + 1]))
    halo = set(own)
    for z in (zb[s] - 1, zb[s + 1]):
        if 0 <= z < nz:
            halo.add(z)
        elif zper:
            halo.add(z % nz)
    if ph == A_:
        acc = [(f"f{a}", "r", own), (f"g{a}", "r", own), (f"ref{a}", "r", own),
               ("rho", "w", own), ("psi", "w", own), (f"ref{b}", "w", own)]
        if fused:  # the previous step's face rules on this slab's face nodes (F of that step)
            acc += [("F", "r", own), (f"f{a}", "w", own), (f"g{a}", "w", own)]
        return acc
    if ph == BC19_:  # force from the psi stencil; collide; push (with the destinations' rho)
        return [("psi", "r", halo), ("rho", "r", halo), (f"f{a}", "r", own), (f"ref{a}", "r", own),
                ("F", "w", own), ("u", "w", own), (f"f{b}", "p", halo)]
    if ph == C7_:  # div u stencil; destinations' old g, rho and references; relaxed push
        return [("u", "r", halo), ("rho", "r", halo), (f"ref{a}", "r", halo), (f"ref{b}", "r", halo),
                (f"g{a}", "r", halo), ("T12", "r", own), ("T12", "w", own), (f"g{b}", "p", halo)]
    return [(f"f{b}", "r", own), (f"g{b}", "r", own), ("F", "r", own), (f"ref{b}", "r", own),
            (f"f{b}", "w", own), (f"g{b}", "w", own)]


def unordered_conflicts(n, zb, order, within, prev, nz, zper, modes=((False, True, True), (False, True, False)),
                        prev_fused=None, has_d=None):
    """modes[t] = (fused, emit_d, first) of step t: its phase A applies the previous step's
    face rules (waiting on prev_fused instead of prev), it runs its phase D stages, it starts
    a new sequence (the library joins every slab stream before it)."""
    seq = [(t, code) for t in range(len(modes)) for code in order if code // n != D_ or modes[t][1]]
    pos = {st: i for i, st in enumerate(seq)}
    preds = {st: set() for st in seq}
    for t, code in seq:
        fused, _, first = modes[t]
        for q in within[code]:
            if (t, q) in pos:
                preds[(t, code)].add((t, q))
        if t > 0 and first:  # a new sequence: after everything before it
            preds[(t, code)] |= {st for st in seq if st[0] < t}
        elif t > 0 and code // n == A_:
            for q in (prev_fused if fused else prev)[code % n]:
                assert (t - 1, q) in pos, (t, code, q)
                preds[(t, code)].add((t - 1, q))
    last_on_stream = {}
    for st in seq:  # the order of each stream
        k = (st[1] % n) % N_STREAMS
        if k in last_on_stream:
            preds[st].add(last_on_stream[k])
        last_on_stream[k] = st
    before = {}
    for st in seq:  # every stage that is ordered before st
        acc = set()
        for q in preds[st]:
            assert pos[q] < pos[st]
            acc.add(q)
            acc |= before[q]
        before[st] = acc
    acc = {st: stage_access(st[1] // n, st[1] % n, st[0], zb, nz, zper,
                            modes[st[0]][0] and st[1] // n == A_ and has_d is not None and has_d[st[1] % n])
           for st in seq}
    bad = []
    for i, x in enumerate(seq):
        for y in seq[i + 1:]:
            if x in before[y]:
                continue
            for rx, mx, px in acc[x]:
                for ry, my, py in acc[y]:
                    if rx == ry and {mx, my} != {"r"} and {mx, my} != {"p"} and px & py:
                        bad.append((x, y, rx))
    return bad


@pytest.mark.parametrize("faces_z", [0, 1, 2])
@pytest.mark.parametrize("nz,sp", [(9, 3), (12, 3), (13, 4), (40, 5), (6, 3), (3, 3), (64, 3)])
def test_slab_pipeline_orders_every_conflict(H, faces_z, nz, sp, thermo):
    """Periodic, wall and open z faces; one to twenty-one slabs (with periodic z, one or two
    slabs make a slab its own neighbour)."""
    kinds = {0: [0, 0, 0, 0, 0, 0], 1: [0, 0, 0, 0, 1, 1], 2: [2, 2, 0, 0, 2, 2]}[faces_z]
    p = W.base_params(5, 4, nz, rho_l=thermo["rho_l"], rho_v=thermo["rho_v"], face_kind=kinds,
                      face_T=[thermo["Ts"]] * 6, face_rho=[thermo["rho_v"]] * 6)
    n, zb, order, within, prev = slab_plan(H, p, sp)
    assert len(set(order)) == len(order) and all(0 <= c < 4 * n for c in order)
    assert {c for c in order if c // n != D_} == {c for c in range(3 * n)}  # every A, BC19, C7 stage once
    bad = unordered_conflicts(n, zb, order, within, prev, nz, faces_z == 0)
    assert not bad, bad[:5]
    # sequences whose face rules go into the next step's phase A: three steps (plain, fused,
    # fused with phase D), then a second sequence of two
    prev_fused, has_d = slab_plan.fused
    modes = ((False, False, True), (True, False, False), (True, True, False), (False, False, True), (True, True, False))
    bad = unordered_conflicts(n, zb, order, within, prev, nz, faces_z == 0, modes, prev_fused, has_d)
    assert not bad, bad[:5]


# ------------------------------------------------- persistent schedule order --
def fused_access(ph, z, nz, zper, faces_z):
    """(resource, mode, planes) of the persistent schedule's stage (phase ph, plane z); phase C
    is the D3Q19 and the D3Q7 collide/push of the plane.  'p': streaming pushes (disjoint).
    Phase D rewrites face nodes ('@bnd') and reads g at their inward neighbours x_b - sum n,
    which lie strictly inside along every face normal of x_b and so are never face nodes
    ('@inw'); the two parts do not overlap."""
    def planes(k):
        out = set()
        for d in range(-k, k + 1):
            q = z + d
            if 0 <= q < nz:
                out.add(q)
            elif zper:
                out.add(q % nz)
        return out
    own, n1 = {z}, planes(1)
    if ph == 0:
        return [("f", "r", own), ("g", "r", own), ("rho", "w", own), ("psi", "w", own), ("j", "w", own)]
    if ph == 1:
        return [("psi", "r", n1), ("rho", "r", own), ("j", "r", own), ("F", "w", own), ("u", "w", own)]
    if ph == 2:
        return [("f", "r", own), ("F", "r", own), ("fB", "p", n1), ("g", "r", n1), ("rho", "r", n1),
                ("u", "r", n1), ("gB", "p", n1)]
    inward = n1 if faces_z else own  # a z-face node's inward neighbour is on the next plane
    return [("fB@bnd", "r", own), ("gB@inw", "r", inward), ("F", "r", own), ("fB@bnd", "w", own),
            ("gB@bnd", "w", own)]


def _same(rx, ry):
    """Resources overlap: the same buffer, and the same part unless one is the whole buffer."""
    bx, _, px = rx.partition("@")
    by, _, py = ry.partition("@")
    return bx == by and (px == py or not px or not py)


@pytest.mark.parametrize("gap", [0, 3, 9])
@pytest.mark.parametrize("faces", [(0, 0), (0, 1), (2, 2), (1, 0)])
@pytest.mark.parametrize("nz", [3, 4, 7, 16])
def test_fused_plan_is_dispensable_and_orders_every_conflict(H, faces, nz, gap, thermo):
    """Every stage of the persistent kernel's order waits only for stages dispensed before it
    (so the earliest unfinished item can always run: no deadlock), and the dependency radii
    order every pair of conflicting stages of one step.  faces: (x/y kind, z kind)."""
    fxy, fz = faces
    kinds = [fxy, fxy, fxy, fxy, fz, fz]
    p = W.base_params(5, 4, nz, rho_l=thermo["rho_l"], rho_v=thermo["rho_v"], face_kind=kinds,
                      face_T=[thermo["Ts"]] * 6, face_rho=[thermo["rho_v"]] * 6)
    if fxy == 1 and fz == 2:
        pytest.skip("a wall face may not share an edge with an open face")
    P = lbm.make_params(dict(p, schedule=lbm.SCHED_FUSED))
    cap = 4 * nz
    order = np.zeros(cap, np.int32)
    deps = np.zeros(cap * 8, np.int32)
    n = ct.c_int()
    H.h_fused_plan.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    assert H.h_fused_plan(ct.byref(P), gap, cap, order.ctypes.data, ct.byref(n), deps.ctypes.data) == 0
    seq = [int(c) for c in order[:n.value]]
    assert len(set(seq)) == len(seq)
    pos = {c: i for i, c in enumerate(seq)}
    for ph in range(3):  # phases A, B, C of every plane; D where the plane holds face nodes
        assert all((ph << 24 | z) in pos for z in range(nz))
    wait = {c: [int(q) for q in deps[((c >> 24) * nz + (c & 0xffffff)) * 8:][:8] if q >= 0] for c in seq}
    for c in seq:
        for q in wait[c]:
            assert q in pos and pos[q] < pos[c], (c, q)
    before = {}
    for c in seq:
        acc = set()
        for q in wait[c]:
            acc |= {q} | before[q]
        before[c] = acc
    zper = fz == 0
    access = {c: fused_access(c >> 24, c & 0xffffff, nz, zper, fz != 0) for c in seq}
    bad = []
    for i, x in enumerate(seq):
        for y in seq[i + 1:]:
            if x in before[y] or y in before[x]:
                continue
            for rx, mx, px in access[x]:
                for ry, my, py in access[y]:
                    if _same(rx, ry) and {mx, my} != {"r"} and {mx, my} != {"p"} and px & py:
                        bad.append((hex(x), hex(y), rx))
    assert not bad, bad[:5]
