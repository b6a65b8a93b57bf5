"""Physical behaviour of the CUDA path on the paper's own validation cases.

* d^2 law (Sec. 4.2): the droplet of the 128^3 open-face workload (radius 15,
  vapor at coexistence density, faces at T_c) shrinks with V^(2/3) linear in
  time once the heat from the faces has reached it.  The FP64 droplet volume
  comes from lbm_reduce every 200 steps over 20,000 steps; the fit window
  starts after 8,000 steps, the thermal transient of this geometry (vapor
  diffusivity lambda/(rho_v c_v) = 0.18, 49 cells from face to interface).
  The paper prints only a figure, so the rate K itself is not pinned.
"""
import numpy as np
import pytest

from paper_2206_00946_gb300 import lbm
from paper_2206_00946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()


def test_d2_law_is_linear_after_the_thermal_transient(thermo):
    p, rho0, T0 = W.droplet(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], n=128, R=15.0)
    p["schedule"] = lbm.SCHED_SLABS
    lat = lbm.Lattice(p, rho0.reshape(-1).astype(np.float32), T0.reshape(-1).astype(np.float32))
    t, V = [], []
    for k in range(101):
        st, red = lat.lbm_reduce()
        assert st == lbm.OK
        t.append(200 * k)
        V.append(red[2])
        if k < 100:
            lat.lbm_step(200)
    lat.close()
    t, V = np.array(t, dtype=float), np.array(V)
    sel = t >= 8000
    # evaporating: the volume falls monotonically in the window (before it, pressure
    # waves between the open faces make the volume integral oscillate by a few percent)
    assert V[-1] < 0.8 * V[0] and np.all(np.diff(V[sel]) < 0)
    y = V ** (2.0 / 3.0)
    a = np.polyfit(t[sel], y[sel], 1)
    r2 = 1 - np.sum((y[sel] - np.polyval(a, t[sel])) ** 2) / np.sum((y[sel] - y[sel].mean()) ** 2)
    print(f"d2 law: K = {-a[0]:.3e} per step (in V^(2/3)), R^2 = {r2:.5f}")
    assert a[0] < 0 and r2 >= 0.99, r2
