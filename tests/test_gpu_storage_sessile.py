"""Field errors of the population storage forms on the 256 x 256 x 128 droplet on a heated
surface (the headline workload), in FP32, FP16 and bfloat16 with one global shift, and FP16
with per-cell references.

* Short horizon against the FP64 oracle (its OpenMP build): 20 steps from the same FP32
  state.  FP32 stays within 1e-5 (max relative, rho and T); the 16-bit forms within their
  storage rounding over 20 steps.
* 10,000 steps against the FP32 run of the library (the oracle would take hours): the
  per-field max relative and relative L2 errors of each 16-bit form are printed for the
  record and must stay below their bounds.
"""
import numpy as np
import pytest

from cases import f32
from oracle import Oracle
from paper_2206_00946_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FORMS = {"f32": lbm.STORE_F32, "f16": lbm.STORE_F16_SHIFTED, "bf16": lbm.STORE_BF16_SHIFTED,
         "f16local": lbm.STORE_F16_LOCAL}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()


def _run(p, f0, g0, steps, storage):
    lat = lbm.Lattice(dict(p, storage=storage, schedule=lbm.SCHED_SLABS))
    lat.lbm_set_state(torch.from_numpy(f0).cuda(), torch.from_numpy(g0).cuda())
    lat.lbm_step(steps)
    rho = torch.empty(lat.N, device="cuda")
    T = torch.empty(lat.N, device="cuda")
    st = lat.lbm_macros(rho=rho, T=T)
    lat.close()
    assert st == lbm.OK
    return rho.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)


def _errs(a, r):
    return float(np.max(np.abs(a - r) / np.abs(r))), float(np.linalg.norm(a - r) / np.linalg.norm(r))


def test_storage_forms_on_the_sessile_workload(thermo):
    p, rho0, T0 = W.sessile(thermo["Tc"], thermo["rho_v"], thermo["rho_l"])
    o = Oracle(p, omp=True)
    f0, g0 = o.init_state(rho0, T0)
    f0, g0 = f32(f0), f32(g0)
    st, fo, go = o.run(f0.astype(np.float64), g0.astype(np.float64), 20)
    assert st == 0
    ro, To = fo.sum(0), go.sum(0)
    short = {}
    for name, storage in FORMS.items():
        r, T = _run(p, f0, g0, 20, storage)
        short[name] = (_errs(r, ro), _errs(T, To))
        print(f"sessile 256x256x128, 20 steps vs FP64 oracle, {name}: rho max {short[name][0][0]:.2e} "
              f"L2 {short[name][0][1]:.2e}; T max {short[name][1][0]:.2e} L2 {short[name][1][1]:.2e}")
    assert short["f32"][0][0] < 1e-5 and short["f32"][1][0] < 1e-5
    for name, half_ulp in (("f16", 2.0 ** -11), ("f16local", 2.0 ** -11), ("bf16", 2.0 ** -8)):
        # 20 roundings of deviations that are at most about rho_l / rho_v of the shift
        assert short[name][0][0] < 20 * half_ulp * 17 and short[name][1][0] < 20 * half_ulp, (name, short[name])
    ref = _run(p, f0, g0, 10000, lbm.STORE_F32)
    assert np.all(np.isfinite(ref[0])) and np.all(np.isfinite(ref[1]))
    long = {}
    for name in ("f16", "bf16", "f16local"):
        r, T = _run(p, f0, g0, 10000, FORMS[name])
        assert np.all(np.isfinite(r)) and np.all(np.isfinite(T)), name
        long[name] = (_errs(r, ref[0]), _errs(T, ref[1]))
        print(f"sessile 256x256x128, 10,000 steps vs FP32, {name}: rho max {long[name][0][0]:.2e} "
              f"L2 {long[name][0][1]:.2e}; T max {long[name][1][0]:.2e} L2 {long[name][1][1]:.2e}")
    # relative L2 bounds of rho and T, each a few times the measured error; the per-cell
    # references are the accurate form, one global shift drifts by 0.1 in rho over this run
    bounds = {"f16": (0.3, 3e-2), "bf16": (1.0, 0.1), "f16local": (3e-2, 3e-3)}
    for name, (bmax_rho, bmax_T) in bounds.items():
        assert long[name][0][1] < bmax_rho and long[name][1][1] < bmax_T, (name, long[name])
