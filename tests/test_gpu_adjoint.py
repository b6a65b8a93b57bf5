"""Discrete adjoint of the CUDA library against FP64 references.

The loss is the smooth liquid mass of the final density plus a weighted sum of
the final temperature.  Its gradients with respect to the initial temperature
field T0 and the per-node face temperatures, computed by lbm_record +
lbm_adjoint_step (FP32 step, FP64 accumulation) through the autograd wrapper,
are compared with
  * torch.autograd through the independent FP64 plain-torch step (every
    element), and
  * central differences of the FP64 C oracle at seeded probe points, among them
    the adjoint workload's own check in reduced form: a 12^3 open droplet (the
    64^3 workload's faces, radius 3), 100 steps with a checkpoint every 10, 32
    seeded probes of T0 and of the bottom-face temperature field, h = 1e-6 in
    FP64, gradients within 1e-4 of their largest magnitude.
Several checkpoint segments and a ragged last segment are exercised (K does
not divide the step count).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from cases import F16_LOCAL
from oracle import Oracle
from oracle.torch_step import TorchStep
from paper_2206_00946_gb300 import lbm
from paper_2206_00946_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()


def _case(kind, thermo):
    Tc, rv, rl = thermo["Tc"], thermo["rho_v"], thermo["rho_l"]
    if kind == "open":
        p, rho0, T0 = W.droplet(Tc, rv, rl, n=8, R=2.5, W=2.0, seed=4, amp=1e-3)
        p.update(lambda_l=0.4, lambda_v=0.2)
        face = 4
    elif kind == "open12":
        p, rho0, T0 = W.droplet(Tc, rv, rl, n=12, R=3.0, W=2.0, seed=5, amp=1e-3)
        p.update(lambda_l=0.4, lambda_v=0.2)
        face = 1
    else:  # heated bottom wall, open top, periodic in x and y
        p, rho0, T0 = W.sessile(Tc, rv, rl, nx=8, ny=7, nz=9, R=3.0, W=2.0)
        face = 4
    rho0 = rho0.reshape(-1).astype(np.float32).astype(np.float64)
    T0 = T0.reshape(-1).astype(np.float32).astype(np.float64)
    ts = TorchStep(p)
    nf = int(np.prod(ts.face_shape(face)))
    rng = np.random.default_rng(11)
    Tb = (p["face_T"][face] * (1 + 0.01 * rng.standard_normal(nf))).astype(np.float32).astype(np.float64)
    wT = rng.standard_normal(p["nx"] * p["ny"] * p["nz"])  # weights of the final-T term
    return p, rho0, T0, face, Tb, wT


def _loss(rho, T, p, wT):
    mid = 0.5 * (p["rho_l"] + p["rho_v"])
    lm = (rho * 0.5 * (1 + torch.tanh((rho - mid) / (0.1 * (p["rho_l"] - p["rho_v"]))))).sum()
    return lm + 100.0 * (T * wT).sum()


def _gpu_grads(p, rho0, T0, face, Tb, wT, n, K):
    from paper_2206_00946_gb300 import adjoint
    dev = "cuda"
    T0_t = torch.tensor(T0, device=dev, requires_grad=True)
    faces = [None] * 6
    faces[face] = torch.tensor(Tb, device=dev, requires_grad=True)
    rho, T = adjoint.run(p, torch.tensor(rho0, device=dev), T0_t, n, K=K, faces=faces)
    L = _loss(rho.double(), T.double(), p, torch.tensor(wT, device=dev))
    L.backward()
    return float(L.detach()), T0_t.grad.cpu().numpy(), faces[face].grad.cpu().numpy()


def _ref_grads(p, rho0, T0, face, Tb, wT, n):
    ts = TorchStep(p)
    T0_t = torch.tensor(T0, requires_grad=True)
    Tb_t = torch.tensor(Tb, requires_grad=True)
    f, g = ts.init_state(torch.tensor(rho0), T0_t)
    for _ in range(n):
        f, g = ts.step(f, g, {face: Tb_t})
    L = _loss(f.sum(0), g.sum(0), p, torch.tensor(wT))
    L.backward()
    return float(L), T0_t.grad.numpy(), Tb_t.grad.numpy()


@pytest.mark.parametrize("kind,n,K", [("open", 12, 5), ("wall_open", 12, 5), ("open12", 20, 7)])
def test_adjoint_matches_fp64_autograd(kind, n, K, thermo):
    p, rho0, T0, face, Tb, wT = _case(kind, thermo)
    Lg, dT0_g, dTb_g = _gpu_grads(p, rho0, T0, face, Tb, wT, n, K)
    Lr, dT0_r, dTb_r = _ref_grads(p, rho0, T0, face, Tb, wT, n)
    assert abs(Lg - Lr) < 1e-5 * abs(Lr)
    e0 = np.max(np.abs(dT0_g - dT0_r)) / np.max(np.abs(dT0_r))
    eb = np.max(np.abs(dTb_g - dTb_r)) / np.max(np.abs(dTb_r))
    print(f"{kind}: |dL/dT0 err| / max = {e0:.2e}, |dL/dTface err| / max = {eb:.2e}")
    assert e0 < 1e-4 and eb < 1e-4, (e0, eb)


def test_adjoint_matches_oracle_differences(thermo):
    """Central differences of the FP64 C oracle at seeded probes (h = 1e-4 relative)."""
    p, rho0, T0, face, Tb, wT = _case("open", thermo)
    n, K = 12, 5
    _, dT0_g, dTb_g = _gpu_grads(p, rho0, T0, face, Tb, wT, n, K)
    tf = [None] * 6

    def L_oracle(T0v, Tbv):
        o = Oracle(p)
        tf2 = list(tf)
        tf2[face] = Tbv
        o.set_face_T(tf2)
        f, g = o.init_state(rho0, T0v)
        st, f, g = o.run(f, g, n)
        assert st == 0
        return float(_loss(torch.tensor(f.sum(0)), torch.tensor(g.sum(0)), p, torch.tensor(wT)))

    rng = np.random.default_rng(2206)
    scale0, scaleb = np.max(np.abs(dT0_g)), np.max(np.abs(dTb_g))
    for c in rng.choice(T0.size, 6, replace=False):
        h = 1e-4 * T0[c]
        a, b = T0.copy(), T0.copy()
        a[c] += h
        b[c] -= h
        fd = (L_oracle(a, Tb) - L_oracle(b, Tb)) / (2 * h)
        assert abs(dT0_g[c] - fd) <= 2e-3 * scale0, (c, dT0_g[c], fd)
    for k in rng.choice(Tb.size, 4, replace=False):
        h = 1e-4 * Tb[k]
        a, b = Tb.copy(), Tb.copy()
        a[k] += h
        b[k] -= h
        fd = (L_oracle(T0, a) - L_oracle(T0, b)) / (2 * h)
        assert abs(dTb_g[k] - fd) <= 2e-3 * scaleb, (k, dTb_g[k], fd)


def test_adjoint_matches_fp64_central_differences_at_32_probes(thermo):
    """The adjoint workload's accuracy check, reduced to a size the FP64 oracle runs 64
    times in seconds: 12^3 open droplet of radius 3, 100 steps, checkpoints every 10;
    16 probes of T0 and 16 of the bottom-face (z = 0) temperature field, central
    differences with h = 1e-6 of the FP64 C oracle; every gradient within 1e-4 of the
    largest gradient magnitude of its field."""
    Tc, rv, rl = thermo["Tc"], thermo["rho_v"], thermo["rho_l"]
    p, rho0, T0 = W.droplet(Tc, rv, rl, n=12, R=3.0, W=2.0, seed=9, amp=1e-3)
    rho0 = rho0.reshape(-1).astype(np.float32).astype(np.float64)
    T0 = T0.reshape(-1).astype(np.float32).astype(np.float64)
    face, n, K = 4, 100, 10
    rng = np.random.default_rng(2206)
    Tb = (p["face_T"][face] * (1 + 0.01 * rng.standard_normal(12 * 12))).astype(np.float32).astype(np.float64)
    wT = rng.standard_normal(T0.size)
    _, dT0_g, dTb_g = _gpu_grads(p, rho0, T0, face, Tb, wT, n, K)

    def L_oracle(args):
        T0v, Tbv = args
        o = Oracle(p)
        tf = [None] * 6
        tf[face] = Tbv
        o.set_face_T(tf)
        f, g = o.init_state(rho0, T0v)
        st, f, g = o.run(f, g, n)
        assert st == 0
        return float(_loss(torch.tensor(f.sum(0)), torch.tensor(g.sum(0)), p, torch.tensor(wT)))

    h = 1e-6
    jobs, probes = [], []
    for c in rng.choice(T0.size, 16, replace=False):
        a, b = T0.copy(), T0.copy()
        a[c] += h
        b[c] -= h
        jobs += [(a, Tb), (b, Tb)]
        probes.append(("T0", c))
    for k in rng.choice(Tb.size, 16, replace=False):
        a, b = Tb.copy(), Tb.copy()
        a[k] += h
        b[k] -= h
        jobs += [(T0, a), (T0, b)]
        probes.append(("Tb", k))
    with ThreadPoolExecutor(8) as ex:  # the oracle releases the GIL
        Ls = list(ex.map(L_oracle, jobs))
    worst = 0.0
    for j, (field, idx) in enumerate(probes):
        fd = (Ls[2 * j] - Ls[2 * j + 1]) / (2 * h)
        got, scale = (dT0_g[idx], np.max(np.abs(dT0_g))) if field == "T0" else (dTb_g[idx], np.max(np.abs(dTb_g)))
        worst = max(worst, abs(got - fd) / scale)
        assert abs(got - fd) <= 1e-4 * scale, (field, idx, got, fd)
    print(f"adjoint vs central differences (h = 1e-6, 32 probes): max |err| / scale = {worst:.2e}")


@pytest.mark.parametrize("schedule", [lbm.SCHED_PHASES, lbm.SCHED_SLABS, lbm.SCHED_FUSED])
def test_record_leaves_the_same_state_as_stepping(schedule, thermo):
    """lbm_record steps like lbm_step (its last segment runs the phase kernels, so
    the persistent schedule agrees to rounding only: it contracts other FMAs)."""
    p, rho0, T0, face, Tb, wT = _case("open", thermo)
    p = dict(p, schedule=schedule)
    a = lbm.Lattice(dict(p), rho0.astype(np.float32), T0.astype(np.float32))
    b = lbm.Lattice(dict(p), rho0.astype(np.float32), T0.astype(np.float32))
    a.lbm_step(13)
    b.lbm_record(13, 4)
    sa, fa, ga = a.state()
    sb, fb, gb = b.state()
    assert sa == sb == lbm.OK
    if schedule == lbm.SCHED_FUSED:
        assert np.max(np.abs(fa - fb)) <= 1e-6 * np.max(np.abs(fa))
        assert np.max(np.abs(ga - gb)) <= 1e-6 * np.max(np.abs(ga))
        fa, ga = fb, gb
    else:
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    # the adjoint leaves the recorded final state current
    seed = np.ones(b.N, dtype=np.float32)
    dev = torch.tensor(seed, device="cuda")
    b.lbm_adjoint_step(13, dev, None, None, None)
    sc, fc, gc = b.state()
    assert np.array_equal(fa, fc) and np.array_equal(ga, gc)
    with pytest.raises(lbm.LBMError):
        b.lbm_adjoint_step(12, dev, None, None, None)  # not the recorded count
    a.close()
    b.close()


@pytest.mark.parametrize("storage", [lbm.STORE_F16_SHIFTED, F16_LOCAL])
def test_record_rejects_16bit_storage(storage, thermo):
    p, rho0, T0, face, Tb, wT = _case("open", thermo)
    lat = lbm.Lattice(dict(p, storage=storage, schedule=lbm.SCHED_PHASES),
                      rho0.astype(np.float32), T0.astype(np.float32))
    with pytest.raises(lbm.LBMError) as e:
        lat.lbm_record(4, 2)
    assert e.value.status == lbm.ERR_ARG
    lat.close()


def test_segment_graphs_match_step_launches(thermo, monkeypatch):
    """Full K-step segments (adjoint and recomputation) replayed from CUDA graphs
    (odd K: both parities of the adjoint buffers, both segment buffers) against
    launching every step on its own, and with programmatic dependent launches
    against without.  The NEE transpose adds with atomics, so all agree to
    rounding."""
    p, rho0, T0, face, Tb, wT = _case("open12", thermo)
    graph = _gpu_grads(p, rho0, T0, face, Tb, wT, 20, 7)
    monkeypatch.setenv("LBM_ADJ_EAGER", "1")
    eager = _gpu_grads(p, rho0, T0, face, Tb, wT, 20, 7)
    monkeypatch.setenv("LBM_ADJ_NOPDL", "1")
    plain = _gpu_grads(p, rho0, T0, face, Tb, wT, 20, 7)
    monkeypatch.delenv("LBM_ADJ_EAGER")
    graph_plain = _gpu_grads(p, rho0, T0, face, Tb, wT, 20, 7)
    for other in (eager, plain, graph_plain):
        assert graph[0] == other[0]
        for a, b in zip(graph[1:], other[1:]):
            assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
