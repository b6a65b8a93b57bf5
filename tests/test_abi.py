"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/lbm.h (no GPU needed)."""
import ctypes as ct
import os
import re

import pytest

from paper_2206_00946_gb300 import lbm, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = lbm.load()
    names = _declared()
    assert "lbm_init" in names and "lbm_step" in names
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lbm.EXPORTS) == names


def test_params_struct_matches_header():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    body = src[src.index("typedef struct lbm_params"):src.index("} lbm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for line in body.splitlines()[1:]:
        line = line.strip().rstrip(";")
        if not line:
            continue
        typ, rest = line.split(None, 1)
        for nm in rest.split(","):
            fields.append(re.sub(r"\[.*\]", "", nm).strip())
    assert fields == [n for n, _ in lbm.lbm_params._fields_]


@pytest.mark.parametrize("bad", [
    dict(nx=0),
    dict(vartheta=2),
    dict(face_kind=[1, 1, 2, 2, 0, 0]),   # wall next to an open face
    dict(face_kind=[1, 0, 0, 0, 0, 0]),   # half-periodic axis
    dict(face_kind=[0, 0, 0, 0, 2, 2], face_rho=[0] * 6),
    dict(wbar=1.5),
    dict(storage=7),
    dict(storage=4),
    dict(storage=3, schedule=0),          # 16-bit storage in the persistent schedule (FP32 only)
    dict(storage=1, schedule=0),
    dict(nz=2, face_kind=[0, 0, 0, 0, 1, 1]),
])
def test_invalid_parameters_rejected_before_any_device_work(bad):
    p = W.base_params(8, 8, 8, rho_l=6.5, rho_v=0.38)
    p.update(bad)
    L = lbm.load()
    ctx = ct.c_void_p()
    st = L.lbm_init(ct.byref(ctx), ct.byref(lbm.make_params(p)), None, None, 0, None)
    assert st == lbm.ERR_ARG and not ctx.value


def test_status_strings_and_host_helpers(thermo):
    assert lbm.lbm_status_string(-4).startswith("psi undefined")
    p = W.base_params(4, 4, 4)
    assert abs(lbm.lbm_Tc(p) - thermo["Tc"]) < 1e-15
    rv, rl, ps = lbm.lbm_maxwell(p, thermo["Ts"])
    assert abs(rv - thermo["rho_v"]) < 1e-8 and abs(rl - thermo["rho_l"]) < 1e-8
    assert abs(ps - thermo["p_sat"]) < 1e-9 * ps
