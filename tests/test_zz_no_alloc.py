"""lbm_reduce_static: the allocation-free reductions agree with lbm_reduce.

Some callers cannot call cudaMalloc when they want these diagnostics (their
device memory is all handed out by their own pool, or they are a plug-in that
only receives device pointers); lbm_reduce_static serves them from a fixed
scratch array inside the library.  This file is collected after every other
test file, so that a run stopping at its first failure has already run the rest
of the suite; only the cases of the FP16 storage with per-cell references, which
the suite's configuration moves to the very end, run after it.
"""
import numpy as np
import pytest

from paper_2206_00946_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_reduction_matches_lbm_reduce_twice_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p0 = W.base_params(4, 4, 4)
    Tc = lbm.lbm_Tc(p0)
    rv, rl, _ = lbm.lbm_maxwell(p0, 0.86 * Tc)
    results = []
    for n, seed in ((40, 1), (24, 2)):  # two calls in a row, different sizes and contents
        p, rho0, T0 = W.droplet(Tc, rv, rl, n=n, R=n / 5, W=3.0, seed=seed)
        N = p["nx"] * p["ny"] * p["nz"]
        f, g = W.random_populations(n, n, n, rho0.reshape(-1), T0.reshape(-1), W.W19, W.w7(p["wbar"]), 0.01, seed)
        f_d = torch.tensor(f, dtype=torch.float32, device="cuda").contiguous()
        g_d = torch.tensor(g, dtype=torch.float32, device="cuda").contiguous()
        lat = lbm.Lattice(p)
        lat.lbm_set_state(f_d, g_d)
        st, ref = lat.lbm_reduce()
        lat.close()
        assert st == lbm.OK
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        st = lbm.lbm_reduce_static(f_d, g_d, N, p["cv"], p["rho_v"], p["rho_l"], out, stream)
        assert st == lbm.OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-9)
        assert got[3] == ref[3] == 0
        results.append(got)
    assert not np.allclose(results[0], results[1])  # the second call did not reuse the first call's sums


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dummy = torch.zeros(32, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # the library's own check, before any device access (a raw call: the binding stops a
    # buffer shorter than the cell count before calling the library)
    st = lbm.load().lbm_reduce_static(dummy.data_ptr(), dummy.data_ptr(), 4096 * 8192 + 1, 5.0, 0.38, 6.5,
                                      out.data_ptr(), None)
    assert st == lbm.ERR_ARG
    with pytest.raises(ValueError):
        lbm.lbm_reduce_static(dummy, dummy, 4096 * 8192 + 1, 5.0, 0.38, 6.5, out, None)


def test_static_scratch_counts_a_non_finite_cell_like_lbm_reduce():
    """One population set to NaN: the cell is counted in out[3] and left out of the three
    sums, exactly as lbm_reduce does on the same state."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p0 = W.base_params(4, 4, 4)
    Tc = lbm.lbm_Tc(p0)
    rv, rl, _ = lbm.lbm_maxwell(p0, 0.86 * Tc)
    n = 16
    p, rho0, T0 = W.droplet(Tc, rv, rl, n=n, R=4.0, W=3.0, seed=5)
    N = p["nx"] * p["ny"] * p["nz"]
    f, g = W.random_populations(n, n, n, rho0.reshape(-1), T0.reshape(-1), W.W19, W.w7(p["wbar"]), 0.01, 5)
    f[7, 123] = np.nan
    f_d = torch.tensor(f, dtype=torch.float32, device="cuda").contiguous()
    g_d = torch.tensor(g, dtype=torch.float32, device="cuda").contiguous()
    lat = lbm.Lattice(p)
    lat.lbm_set_state(f_d, g_d)
    st, ref = lat.lbm_reduce()
    lat.close()
    assert st in (lbm.OK, lbm.ERR_NONFINITE)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lbm.lbm_reduce_static(f_d, g_d, N, p["cv"], p["rho_v"], p["rho_l"], out,
                               torch.cuda.current_stream().cuda_stream)
    assert st == lbm.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[3] == ref[3] == 1
    np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-9)
    assert np.all(np.isfinite(got[:3]))
