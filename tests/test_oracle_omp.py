"""The OpenMP build of the oracle (the benchmark's all-core CPU baseline) computes exactly
what the serial build computes: its parallel loops over z write disjoint cells, so the
states after two steps are bit-identical for every boundary kind and for vartheta = 1."""
import numpy as np
import pytest

from cases import case_params, droplet_state
from oracle import Oracle


@pytest.mark.parametrize("name", ["open_all", "walls_xy_theta", "wall_bottom_open_top", "ragged_open_x"])
def test_openmp_build_is_bit_identical(name, thermo):
    p = case_params(name, thermo)
    f, g = (s.astype(np.float64) for s in droplet_state(p, thermo, seed=3, amp=0.005))
    a, b = Oracle(p), Oracle(p, omp=True)
    b.threads(4)
    ra, rb = a.run(f, g, 2), b.run(f, g, 2)
    assert ra[0] == rb[0] == 0
    assert np.array_equal(ra[1], rb[1]) and np.array_equal(ra[2], rb[2])
    pv = dict(p, vartheta=1)
    a, b = Oracle(pv), Oracle(pv, omp=True)
    ha, hb = a.run_hist(f, g, a.history(g), 2), b.run_hist(f, g, b.history(g), 2)
    assert ha[0] == hb[0] == 0
    assert all(np.array_equal(u, v) for u, v in zip(ha[1:], hb[1:]))
