"""Failure detection without a GPU fault.

The persistent schedule's work items wait, with a bound of about 2 s, for the planes they
read to be finished.  lbm_inject_stall clears the plane-completion counters while keeping
the step count, so that the next step's waits cannot be satisfied: the waits give up, the
launch aborts, and the host reads LBM_ERR_TIMEOUT.  The context stays usable.  The kernels
that stage their populations in shared memory wait on mbarriers with a bound of about 1 s;
there the injection makes one launch expect 16 bytes more than its copies bring.  The batched
persistent launch waits at grid barriers with the same bound; lbm_batch_inject_stall
fills the barrier's arrival counter so that it cannot complete, and after the timeout the
batch steps like a new one once the domains' states are set again.
"""
import time

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


def _droplet(thermo, schedule):
    p, rho0, T0 = W.droplet(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], n=16, R=4.0, W=3.0, seed=7)
    p.update(schedule=schedule)
    return p, rho0.reshape(-1).astype(np.float32), T0.reshape(-1).astype(np.float32)


def test_stalled_wait_times_out_and_the_context_recovers(thermo):
    p, rho0, T0 = _droplet(thermo, lbm.SCHED_FUSED)
    lat = lbm.Lattice(p, rho0, T0)
    assert lat.lbm_inject_stall() == lbm.ERR_STATE  # before the first step
    lat.lbm_step(2)
    st, f0, g0 = lat.state()
    assert st == lbm.OK
    assert lat.lbm_inject_stall() == lbm.OK
    t0 = time.perf_counter()
    lat.lbm_step(1)
    st = lat.lbm_sync()
    dt = time.perf_counter() - t0
    assert st == lbm.ERR_TIMEOUT
    assert 1.0 < dt < 60.0, dt  # the bound is about 2 s
    # the context stays usable: a state set again steps exactly like a fresh context
    lat.lbm_set_state(f0, g0)
    lat.lbm_step(3)
    st, f1, g1 = lat.state()
    assert st == lbm.OK
    ref = lbm.Lattice(p)
    ref.lbm_set_state(f0, g0)
    ref.lbm_step(3)
    st, f2, g2 = ref.state()
    assert st == lbm.OK
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    lat.close()
    ref.close()


def test_stall_injection_needs_a_bounded_wait(thermo):
    """A 16^3 slab-schedule lattice runs neither the persistent kernel nor the staged ones."""
    p, rho0, T0 = _droplet(thermo, lbm.SCHED_SLABS)
    lat = lbm.Lattice(p, rho0, T0)
    lat.lbm_step(1)
    assert lat.lbm_inject_stall() == lbm.ERR_ARG
    lat.close()


@pytest.mark.parametrize("schedule", [lbm.SCHED_SLABS, lbm.SCHED_PHASES])
def test_staged_wait_times_out_and_the_context_recovers(thermo, schedule):
    """96 x 96 x 72 (663,552 cells, planes of 36 tiles of 256 cells): large enough for the
    kernels that stage their populations."""
    p, rho0, T0 = W.droplet(thermo["Tc"], thermo["rho_v"], thermo["rho_l"], R=10.0, shape=(96, 96, 72), seed=7)
    p.update(schedule=schedule)
    rho0, T0 = rho0.reshape(-1).astype(np.float32), T0.reshape(-1).astype(np.float32)
    lat = lbm.Lattice(p, rho0, T0)
    lat.lbm_step(2)
    st, f0, g0 = lat.state()
    assert st == lbm.OK
    assert lat.lbm_inject_stall() == lbm.OK
    t0 = time.perf_counter()
    lat.lbm_step(1)
    st = lat.lbm_sync()
    dt = time.perf_counter() - t0
    assert st == lbm.ERR_TIMEOUT
    assert 0.5 < dt < 60.0, dt  # the bound is about 1 s, and the drain about 1 s more
    lat.lbm_set_state(f0, g0)
    lat.lbm_step(3)
    st, f1, g1 = lat.state()
    assert st == lbm.OK
    ref = lbm.Lattice(p)
    ref.lbm_set_state(f0, g0)
    ref.lbm_step(3)
    st, f2, g2 = ref.state()
    assert st == lbm.OK
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    lat.close()
    ref.close()


def test_batch_barrier_times_out_and_the_batch_recovers(thermo):
    doms = [_droplet(thermo, lbm.SCHED_PHASES) for _ in range(2)]
    lats = [lbm.Lattice(p, rho0, T0) for p, rho0, T0 in doms]
    b = lbm.Batch(lats)
    b.lbm_batch_step(2)
    assert b.lbm_batch_sync() == lbm.OK
    saved = [lat.state()[1:] for lat in lats]
    assert b.lbm_batch_inject_stall() == lbm.OK
    t0 = time.perf_counter()
    b.lbm_batch_step(1)
    st = b.lbm_batch_sync()
    dt = time.perf_counter() - t0
    assert st == lbm.ERR_TIMEOUT
    assert 1.0 < dt < 60.0, dt
    # states set again: the batch steps exactly like a new batch over the same states
    for lat, (f, g) in zip(lats, saved):
        lat.lbm_set_state(f, g)
    b.lbm_batch_step(3)
    assert b.lbm_batch_sync() == lbm.OK
    fresh = [lbm.Lattice(doms[0][0]) for _ in lats]
    for lat, (f, g) in zip(fresh, saved):
        lat.lbm_set_state(f, g)
    b2 = lbm.Batch(fresh)
    b2.lbm_batch_step(3)
    assert b2.lbm_batch_sync() == lbm.OK
    for x, y in zip(lats, fresh):
        _, f1, g1 = x.state()
        _, f2, g2 = y.state()
        assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    b.close()
    b2.close()
    for lat in lats + fresh:
        lat.close()
