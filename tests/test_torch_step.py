"""The plain-torch FP64 step (oracle/torch_step.py) against the C oracle.

Two independent writings of the same step must agree to rounding (1e-12
relative to the population scale) on random states, for every kind of face,
with per-node face temperatures; the torch step is the reference for the
discrete adjoint, so its autograd gradient is also checked against central
differences of the C oracle.
"""
import numpy as np
import pytest

from oracle import Oracle, tables
from oracle.torch_step import TorchStep, mhat_rows, m7_rows, C19
from paper_2206_00946_gb300 import workloads as W

torch = pytest.importorskip("torch")

CFG = {
    "periodic": ((6, 5, 4), [0] * 6),
    "open_all": ((5, 6, 5), [2] * 6),
    "walls_z": ((4, 5, 6), [0, 0, 0, 0, 1, 1]),
    "wall_bottom_open_top": ((5, 4, 6), [0, 0, 0, 0, 1, 2]),
    "open_x": ((6, 5, 4), [2, 2, 0, 0, 0, 0]),
    "walls_xy": ((5, 4, 3), [1, 1, 1, 1, 0, 0]),
}


def _params(name, thermo, **kw):
    shape, kinds = CFG[name]
    Ts = thermo["Ts"]
    return W.base_params(*shape, rho_l=thermo["rho_l"], rho_v=thermo["rho_v"], lambda_l=0.4, lambda_v=0.2,
                         face_kind=kinds, face_T=[Ts * (1 + 0.01 * k) for k in range(6)],
                         face_rho=[thermo["rho_v"] * (1 + 0.02 * k) for k in range(6)], **kw)


def _state(p, thermo, seed):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x, y, z = W.grid(nx, ny, nz)
    r = np.sqrt((x - 0.45 * nx) ** 2 + (y - 0.55 * ny) ** 2 + (z - 0.5 * nz) ** 2)
    rho = W.tanh_profile(r - 0.3 * min(nx, ny, nz) - 0.5, thermo["rho_v"], thermo["rho_l"], 2.0)
    Tm = thermo["Ts"] * (1 + 0.01 * np.sin(0.3 * x + 0.2 * y + 0.1 * z))
    return W.random_populations(nx, ny, nz, rho.reshape(-1), Tm.reshape(-1), W.W19, W.w7(p["wbar"]), 0.02, seed)


def test_matrices_match_the_oracle_tables():
    t = tables()
    assert np.array_equal(C19, t["c19"])
    assert np.array_equal(mhat_rows(C19), t["Mhat"])
    assert np.array_equal(m7_rows(C19[:7]), t["M7"])


@pytest.mark.parametrize("name", list(CFG))
@pytest.mark.parametrize("meq_printed", [0, 1])
def test_torch_step_matches_c_oracle(name, meq_printed, thermo):
    p = _params(name, thermo, meq_printed=meq_printed)
    f, g = _state(p, thermo, seed=5)
    o = Oracle(p)
    ts = TorchStep(p)
    rng = np.random.default_rng(3)
    tface_np, tface_t = [None] * 6, {}
    for fc in range(6):
        if p["face_kind"][fc] != 0:
            a = p["face_T"][fc] * (1 + 0.01 * rng.standard_normal(ts.face_shape(fc)[::-1]).reshape(-1))
            tface_np[fc] = a
            tface_t[fc] = torch.tensor(a)
    o.set_face_T(tface_np)
    st, fo, go = o.step(f, g)
    assert st == 0
    ft, gt = ts.step(torch.tensor(f), torch.tensor(g), tface_t)
    ft, gt = ft.numpy(), gt.numpy()
    assert np.max(np.abs(ft - fo)) < 1e-12 * np.max(np.abs(fo))
    assert np.max(np.abs(gt - go)) < 1e-12 * np.max(np.abs(go))


def test_torch_step_matches_c_oracle_over_ten_steps(thermo):
    p, rho0, T0 = W.droplet(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], n=8, R=2.5, W=2.0, seed=4, amp=1e-3)
    p.update(lambda_l=0.4, lambda_v=0.2)
    f, g = Oracle(p).init_state(rho0, T0)
    st, fo, go = Oracle(p).run(f, g, 10)
    assert st == 0
    ts = TorchStep(p)
    ft, gt = torch.tensor(f), torch.tensor(g)
    for _ in range(10):
        ft, gt = ts.step(ft, gt, {})
    assert np.max(np.abs(ft.numpy() - fo)) < 1e-11 * np.max(np.abs(fo))
    assert np.max(np.abs(gt.numpy() - go)) < 1e-11 * np.max(np.abs(go))


def test_autograd_through_torch_step_matches_oracle_differences(thermo):
    """d(sum rho^2 at step 3)/d T0(c) and d/d T_face(bottom node) by autograd vs central
    differences of the C oracle (h = 1e-4 relative, FP64: the rounding of the difference
    quotient, eps |L| / h, stays below 1e-7 while the truncation error is O(h^2))."""
    p = _params("wall_bottom_open_top", thermo)
    ts = TorchStep(p)
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x, y, z = W.grid(nx, ny, nz)
    rho0 = W.tanh_profile(np.sqrt((x - 2) ** 2 + (y - 2) ** 2 + (z - 3) ** 2) - 1.5, thermo["rho_v"],
                          thermo["rho_l"], 2.0).reshape(-1)
    T0 = (thermo["Ts"] * (1 + 0.02 * np.cos(x + 2 * y + z))).reshape(-1)
    Tb = np.full(nx * ny, p["face_T"][4]) * (1 + 0.01 * np.arange(nx * ny) / (nx * ny))
    steps = 3

    def loss_torch(T0_t, Tb_t):
        f, g = ts.init_state(torch.tensor(rho0), T0_t)
        for _ in range(steps):
            f, g = ts.step(f, g, {4: Tb_t})
        return (f.sum(0) ** 2).sum() + 10 * g.sum(0).sum()

    T0_t = torch.tensor(T0, requires_grad=True)
    Tb_t = torch.tensor(Tb, requires_grad=True)
    L = loss_torch(T0_t, Tb_t)
    L.backward()

    def loss_oracle(T0v, Tbv):
        o = Oracle(p)
        o.set_face_T([None, None, None, None, Tbv, None])
        f, g = o.init_state(rho0, T0v)
        st, f, g = o.run(f, g, steps)
        assert st == 0
        return float((f.sum(0) ** 2).sum() + 10 * g.sum(0).sum())

    for c in (0, 17, 37, nx * ny * nz - 1):
        h = 1e-4 * T0[c]
        Tp, Tm = T0.copy(), T0.copy()
        Tp[c] += h
        Tm[c] -= h
        fd = (loss_oracle(Tp, Tb) - loss_oracle(Tm, Tb)) / (2 * h)
        assert abs(T0_t.grad[c].item() - fd) <= 1e-6 * max(1.0, abs(fd)), (c, T0_t.grad[c].item(), fd)
    for k in (0, 6, nx * ny - 1):
        h = 1e-4 * Tb[k]
        Bp, Bm = Tb.copy(), Tb.copy()
        Bp[k] += h
        Bm[k] -= h
        fd = (loss_oracle(T0, Bp) - loss_oracle(T0, Bm)) / (2 * h)
        assert abs(Tb_t.grad[k].item() - fd) <= 1e-6 * max(1.0, abs(fd)), (k, Tb_t.grad[k].item(), fd)
