"""Checkpoint / restore of the time-stepping state through the C ABI.

A restored image must continue bit-for-bit like the run it was taken from (the
step is deterministic: no atomics on the data path), in every storage mode and
schedule, from host and from device images; an image from a context with a
different lattice, storage mode or shift is rejected.
"""
import numpy as np
import pytest

from cases import F16_LOCAL
from paper_2206_00946_gb300 import lbm
from paper_2206_00946_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lbm.load()


def _droplet(thermo, n=16, storage=0, schedule=lbm.SCHED_PHASES):
    p, rho0, T0 = W.droplet(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], n=n, R=4.0, W=3.0, seed=7)
    p.update(storage=storage, schedule=schedule)
    return p, rho0.reshape(-1).astype(np.float32), T0.reshape(-1).astype(np.float32)


@pytest.mark.parametrize("storage", [lbm.STORE_F32, lbm.STORE_F16_SHIFTED, lbm.STORE_BF16_SHIFTED, F16_LOCAL])
@pytest.mark.parametrize("where", ["host", "device"])
def test_restore_continues_bit_exact(storage, where, thermo):
    import torch
    sched = lbm.SCHED_FUSED if storage == lbm.STORE_F32 else lbm.SCHED_SLABS
    p, rho0, T0 = _droplet(thermo, storage=storage, schedule=sched)
    lat = lbm.Lattice(p, rho0, T0)
    lat.lbm_step(7)
    nb = lat.lbm_checkpoint_bytes()
    refs = 8 * lat.N if storage == lbm.STORE_F16_LOCAL else 0  # per-cell rho_ref, T_ref
    assert nb == 256 + 26 * lat.N * (4 if storage == lbm.STORE_F32 else 2) + refs
    img = np.empty(nb, dtype=np.uint8) if where == "host" else torch.empty(nb, dtype=torch.uint8, device="cuda")
    assert lat.lbm_checkpoint(img) == lbm.OK
    lat.lbm_step(5)
    st, f1, g1 = lat.state()
    assert st == lbm.OK
    lat.lbm_restore(img)
    lat.lbm_step(5)
    st, f2, g2 = lat.state()
    assert st == lbm.OK
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    # a second context of the same problem continues from the same image identically
    lat2 = lbm.Lattice(p)
    lat2.lbm_restore(img)
    lat2.lbm_step(5)
    st, f3, g3 = lat2.state()
    assert st == lbm.OK
    assert np.array_equal(f1, f3) and np.array_equal(g1, g3)
    lat.close()
    lat2.close()


def test_restore_rejects_foreign_images(thermo):
    p, rho0, T0 = _droplet(thermo)
    lat = lbm.Lattice(p, rho0, T0)
    img = np.empty(lat.lbm_checkpoint_bytes(), dtype=np.uint8)
    assert lat.lbm_checkpoint(img) == lbm.OK
    q, _, _ = _droplet(thermo, storage=lbm.STORE_F16_SHIFTED, schedule=lbm.SCHED_PHASES)
    other = lbm.Lattice(q)
    with pytest.raises(lbm.LBMError) as e:
        other.lbm_restore(img)
    assert e.value.status == lbm.ERR_ARG
    r, _, _ = _droplet(thermo, n=18)
    bigger = lbm.Lattice(r)
    with pytest.raises(lbm.LBMError):
        bigger.lbm_restore(np.zeros(bigger.lbm_checkpoint_bytes(), dtype=np.uint8))  # no magic
    hdr_only = np.zeros(bigger.lbm_checkpoint_bytes(), dtype=np.uint8)
    hdr_only[:256] = img[:256]  # a valid header of the 16^3 lattice
    with pytest.raises(lbm.LBMError):
        bigger.lbm_restore(hdr_only)
    # checkpoint before any state: out of order
    empty = lbm.Lattice(p)
    assert empty.lbm_checkpoint(img) == lbm.ERR_STATE
    for x in (lat, other, bigger, empty):
        x.close()


def test_restore_continues_bit_exact_with_the_T_history(thermo):
    """vartheta = 1: the image carries the T history of the last two steps (8 B per cell),
    so a restored run continues with the same correction terms."""
    p, rho0, T0 = _droplet(thermo, schedule=lbm.SCHED_SLABS)
    p.update(vartheta=1)
    lat = lbm.Lattice(p, rho0, T0)
    lat.lbm_step(7)
    nb = lat.lbm_checkpoint_bytes()
    assert nb == 256 + 26 * lat.N * 4 + 8 * lat.N
    img = np.empty(nb, dtype=np.uint8)
    assert lat.lbm_checkpoint(img) == lbm.OK
    lat.lbm_step(5)
    st, f1, g1 = lat.state()
    lat.lbm_restore(img)
    lat.lbm_step(5)
    st2, f2, g2 = lat.state()
    assert st == st2 == lbm.OK
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    # an image of the same lattice without the history is not accepted
    q = dict(p, vartheta=0)
    other = lbm.Lattice(q, rho0, T0)
    img0 = np.empty(other.lbm_checkpoint_bytes(), dtype=np.uint8)
    assert other.lbm_checkpoint(img0) == lbm.OK
    with pytest.raises(lbm.LBMError):
        lat.lbm_restore(np.concatenate([img0, np.zeros(8 * lat.N, dtype=np.uint8)]))
    lat.close()
    other.close()
