import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built liblbm.so")
    config.addinivalue_line("markers", "slow: long CPU run (still part of the default suite)")
    config.addinivalue_line("markers", "per_cell_refs: the FP16 storage with per-cell references (run last)")


def pytest_collection_modifyitems(config, items):
    # the per-cell-reference storage form is the newest: its cases run after all others
    items.sort(key=lambda it: it.get_closest_marker("per_cell_refs") is not None)


@pytest.fixture(scope="session")
def thermo():
    """T_c and the Maxwell coexistence state at 0.86 T_c from the oracle (a = 2/49, b = 2/21)."""
    from oracle import Oracle
    from paper_2206_00946_gb300 import workloads as W

    o = Oracle(W.base_params(4, 4, 4))
    Tc = o.Tc()
    rv, rl, ps = o.maxwell(0.86 * Tc)
    return dict(Tc=Tc, Ts=0.86 * Tc, rho_v=rv, rho_l=rl, p_sat=ps)
