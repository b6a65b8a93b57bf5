"""CPU check of the CUDA library's per-cell FP32 arithmetic against the FP64 oracle.

The hand-expanded D3Q19 transform and inverse, the closed-form equilibrium
moments and forcing increments, the D3Q7 collision, the open-face boundary
and the EOS of csrc/lbm_cell.cuh are compiled for the host by nvcc and
compared cell by cell, so that algebra mistakes show up before any GPU run.
"""
import ctypes as ct

import numpy as np
import pytest

import harness_build
from oracle import Oracle, feq19 as ofeq19
from paper_2206_00946_gb300 import workloads as W


@pytest.fixture(scope="module")
def H():
    if not harness_build.nvcc():
        pytest.skip("nvcc not available")
    return ct.CDLL(harness_build.build_harness("cell_harness"))


def _fp(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ct.POINTER(ct.c_float))


def _dk(p, o):
    kappa = 0.37464 + 1.54226 * p["omega"] - 0.26992 * p["omega"] ** 2
    d = np.array([p["a"], p["b"], p["R"], kappa, 1.0 / o.Tc(), p["G"], p["eos_c0"], p["s_e"], p["s_v"], p["s_q"],
                  p["s_pi"], p["cv"], p["wbar"], p["lambda_l"], p["lambda_v"], p["rho_l"], p["rho_v"]])
    k = np.array([p["meq_printed"], p["eos_kind"], p["vartheta"]], dtype=np.int32)
    return d, k


def _args(d, k):
    return d.ctypes.data_as(ct.POINTER(ct.c_double)), k.ctypes.data_as(ct.POINTER(ct.c_int))


@pytest.mark.parametrize("printed", [0, 1])
def test_collide19_matches_oracle(H, printed):
    p = W.base_params(2, 2, 2, meq_printed=printed, s_e=1.25, s_v=0.8, s_q=1.1, s_pi=0.9)
    o = Oracle(p)
    d, k = _dk(p, o)
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(200):
        rho = rng.uniform(0.3, 7.0)
        u = rng.uniform(-0.08, 0.08, 3)
        f = (ofeq19(rho, u) * (1 + 0.05 * rng.uniform(-1, 1, 19))).astype(np.float32).astype(np.float64)
        rho_f = f.sum()
        ueq = np.array([f @ np.array(c) for c in _C19T]) / rho_f
        F = rng.uniform(-0.02, 0.02, 3).astype(np.float32).astype(np.float64)
        ref = o.collide19(f, rho_f, ueq, F)
        fa, fp = _fp(f)
        ua, up = _fp(ueq)
        Fa, Fp = _fp(F)
        out = np.zeros(19, dtype=np.float32)
        H.h_collide19(*_args(d, k), fp, ct.c_float(rho_f), up, Fp, out.ctypes.data_as(ct.POINTER(ct.c_float)))
        worst = max(worst, np.max(np.abs(out - ref) / np.abs(ref)))
    assert worst < 2e-6, worst


_C19T = None


def setup_module(module):
    from oracle import tables
    global _C19T
    _C19T = tables()["c19"].T.astype(float)


@pytest.mark.parametrize("vartheta", [0, 1])
def test_collide7_matches_oracle(H, vartheta):
    p = W.base_params(2, 2, 2, lambda_l=0.4, lambda_v=0.2, rho_l=6.5, rho_v=0.38, vartheta=vartheta)
    o = Oracle(p)
    d, k = _dk(p, o)
    rng = np.random.default_rng(1)
    w7 = W.w7(p["wbar"])
    for _ in range(200):
        rho = rng.uniform(0.3, 7.0)
        g = (w7 * 0.06 * (1 + 0.02 * rng.uniform(-1, 1, 7))).astype(np.float32).astype(np.float64)
        T = g.sum()
        u = rng.uniform(-0.05, 0.05, 3).astype(np.float32).astype(np.float64)
        divu, dpdT = float(np.float32(rng.uniform(-1e-3, 1e-3))), float(np.float32(rng.uniform(0.1, 2)))
        d2T = float(np.float32(rng.uniform(-1e-3, 1e-3) * T))
        ref = o.collide7(g, rho, T, u, divu, dpdT, d2T)
        ga, gp = _fp(g)
        ua, up = _fp(u)
        out = np.zeros(7, dtype=np.float32)
        H.h_collide7(*_args(d, k), gp, ct.c_float(rho), ct.c_float(T), up, ct.c_float(divu), ct.c_float(dpdT),
                     ct.c_float(d2T), out.ctypes.data_as(ct.POINTER(ct.c_float)))
        np.testing.assert_allclose(out, ref, rtol=2e-6)


@pytest.mark.parametrize("face", range(6))
def test_zouhe_matches_oracle(H, face):
    p = W.base_params(3, 3, 3, face_kind=[2] * 6, face_rho=[0.41] * 6)
    o = Oracle(p)
    rng = np.random.default_rng(2 + face)
    f = (W.W19 * 0.4 * (1 + 0.2 * rng.uniform(-1, 1, 19))).astype(np.float32).astype(np.float64)
    F = rng.uniform(-0.02, 0.02, 3).astype(np.float32).astype(np.float64)
    ref = o.zouhe(face, f, F)
    fa, fp = _fp(f)
    Fa, Fp = _fp(F)
    H.h_zouhe(face, ct.c_float(0.41), Fp, fp)
    np.testing.assert_allclose(fa, ref, rtol=2e-6)


def test_eos_and_psi_match_oracle(H):
    p = W.base_params(2, 2, 2)
    o = Oracle(p)
    d, k = _dk(p, o)
    Tc = o.Tc()
    out = np.zeros(4, dtype=np.float32)
    for rho in (0.2, 0.38, 1.0, 3.0, 6.5, 7.2):
        for T in (0.8 * Tc, 0.86 * Tc, 0.96 * Tc, Tc):
            rho32, T32 = float(np.float32(rho)), float(np.float32(T))
            H.h_eos(*_args(d, k), ct.c_float(rho32), ct.c_float(T32), out.ctypes.data_as(ct.POINTER(ct.c_float)))
            pr, dp = o.p_eos(rho32, T32), o.dpdT(rho32, T32)
            psi = np.sqrt(2 * (rho32 / 3 - pr))
            assert out[3] == 1.0
            assert abs(out[0] - pr) < 2e-6 * (rho32 / 3)  # cancellation: error relative to rho c_s^2
            assert abs(out[1] - dp) < 1e-5 * abs(dp) + 1e-7
            assert abs(out[2] - psi) < 2e-6 * psi


@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 13, 16, 100, 128, 255, 256, 257, 384, 512, 1000, 4097])
def test_fast_division_of_cell_indices(H, d):
    """The multiply-shift division used for x, y, z of a cell index is exact below 2^31."""
    H.h_fdiv_check.restype = ct.c_uint
    assert H.h_fdiv_check(d, 1 << 31, 9973) == 0
    assert H.h_fdiv_check(d, 1 << 20, 1) == 0
