"""CPU check of the per-cell vector-Jacobian products of the discrete adjoint.

lbm_adjoint_cell.cuh is compiled for the host in double together with the
double instantiation of the forward cell functions; for random inputs and
random cotangents b and directions v, <b, J v> from central differences of
the forward must equal <VJP(b), v>.
"""
import ctypes as ct

import numpy as np
import pytest

import harness_build
from oracle import Oracle
from paper_2206_00946_gb300 import workloads as W

DP = ct.POINTER(ct.c_double)


@pytest.fixture(scope="module")
def H():
    if not harness_build.nvcc():
        pytest.skip("nvcc not available")
    L = ct.CDLL(harness_build.build_harness("adjoint_harness"))
    for n in ("a_eos", "a_eos_vjp"):
        getattr(L, n).argtypes = [DP, ct.POINTER(ct.c_int), ct.c_double, ct.c_double] + \
            ([DP] if n == "a_eos" else [ct.c_double, ct.c_double, DP])
    L.a_zouhe.argtypes = [ct.c_int, ct.c_double, DP, DP]
    L.a_zouhe_vjp.argtypes = [ct.c_int, ct.c_double, DP, DP]
    return L


def P_(a):
    return a.ctypes.data_as(DP)


def _dk(p):
    o = Oracle(p)
    kappa = 0.37464 + 1.54226 * p["omega"] - 0.26992 * p["omega"] ** 2
    d = np.array([p["a"], p["b"], p["R"], kappa, 1.0 / o.Tc(), p["G"], p["eos_c0"], p["s_e"], p["s_v"], p["s_q"],
                  p["s_pi"], p["cv"], p["wbar"], p["lambda_l"], p["lambda_v"], p["rho_l"], p["rho_v"]])
    k = np.array([p["meq_printed"], p["eos_kind"]], dtype=np.int32)
    return d, k


def _check(fwd, vjp, x, nout, rng, trials=4, h=1e-6, tol=1e-7):
    for _ in range(trials):
        b = rng.standard_normal(nout)
        v = rng.standard_normal(x.size) * np.maximum(np.abs(x), 1e-2)
        jv = (fwd(x + h * v) - fwd(x - h * v)) / (2 * h)
        lhs = float(b @ jv)
        rhs = float(vjp(x, b) @ v)
        assert abs(lhs - rhs) <= tol * max(1.0, abs(lhs)), (lhs, rhs)


@pytest.mark.parametrize("printed", [0, 1])
@pytest.mark.parametrize("ueq_from_f", [1, 0])
@pytest.mark.parametrize("rates", [(1.25, 0.8, 1.0, 1.0), (1.25, 0.8, 1.1, 0.9)])
def test_collide19_vjp(H, printed, ueq_from_f, rates):
    se, sv, sq, sp = rates
    p = W.base_params(2, 2, 2, meq_printed=printed, s_e=se, s_v=sv, s_q=sq, s_pi=sp)
    d, k = _dk(p)
    rng = np.random.default_rng(1 + printed + 2 * ueq_from_f)
    w = np.array(W.W19)
    for rho in (0.4, 6.3):
        f0 = w * rho * (1 + 0.1 * rng.standard_normal(19))
        F0 = 0.01 * rng.standard_normal(3)
        x = np.concatenate([f0, F0])

        def fwd(x):
            fs = np.empty(19)
            H.a_collide19(P_(d), k.ctypes.data_as(ct.POINTER(ct.c_int)), P_(np.ascontiguousarray(x[:19])),
                          ueq_from_f, P_(np.ascontiguousarray(x[19:])), P_(fs))
            return fs

        def vjp(x, b):
            fb, Fb = np.empty(19), np.empty(3)
            H.a_collide19_vjp(P_(d), k.ctypes.data_as(ct.POINTER(ct.c_int)), P_(np.ascontiguousarray(x[:19])),
                              ueq_from_f, P_(np.ascontiguousarray(x[19:])), P_(np.ascontiguousarray(b)), P_(fb),
                              P_(Fb))
            return np.concatenate([fb, Fb])

        _check(fwd, vjp, x, 19, rng)


@pytest.mark.parametrize("lam", [(0.4, 0.2), (1 / 3, 1 / 3)])
@pytest.mark.parametrize("rho", [0.5, 3.0, 6.6])
def test_collide7_vjp(H, lam, rho, thermo):
    p = W.base_params(2, 2, 2, lambda_l=lam[0], lambda_v=lam[1], rho_l=thermo["rho_l"], rho_v=thermo["rho_v"])
    d, k = _dk(p)
    rng = np.random.default_rng(int(rho * 10))
    w7 = np.array(W.w7(p["wbar"]))
    g0 = w7 * thermo["Ts"] * (1 + 0.05 * rng.standard_normal(7))
    x = np.concatenate([g0, [rho], 0.02 * rng.standard_normal(3), [0.003], [0.4]])
    ki = k.ctypes.data_as(ct.POINTER(ct.c_int))

    def fwd(x):
        gs = np.empty(7)
        H.a_collide7(P_(d), ki, P_(np.ascontiguousarray(x)), P_(gs))
        return gs

    def vjp(x, b):
        xb = np.empty(13)
        H.a_collide7_vjp(P_(d), ki, P_(np.ascontiguousarray(x)), P_(np.ascontiguousarray(b)), P_(xb))
        return xb

    _check(fwd, vjp, x, 7, rng)


@pytest.mark.parametrize("face", range(6))
def test_zouhe_vjp(H, face):
    rng = np.random.default_rng(face)
    w = np.array(W.W19)
    x = np.concatenate([w * 0.4 * (1 + 0.1 * rng.standard_normal(19)), 0.01 * rng.standard_normal(3)])
    rb = 0.39

    def fwd(x):
        fo = np.empty(19)
        H.a_zouhe(face, rb, P_(np.ascontiguousarray(x)), P_(fo))
        return fo

    def vjp(x, b):
        xb = np.empty(22)
        H.a_zouhe_vjp(face, rb, P_(np.ascontiguousarray(b)), P_(xb))
        return xb

    _check(fwd, vjp, x, 19, rng)


@pytest.mark.parametrize("eos_kind", [0, 1])
@pytest.mark.parametrize("rho", [0.38, 2.0, 6.5])
def test_psi_dpdT_vjp(H, eos_kind, rho, thermo):
    p = W.base_params(2, 2, 2, eos_kind=eos_kind, eos_c0=0.2)
    d, k = _dk(p)
    ki = k.ctypes.data_as(ct.POINTER(ct.c_int))
    rng = np.random.default_rng(7)
    x = np.array([rho, thermo["Ts"]])

    def fwd(x):
        out = np.empty(2)
        H.a_eos(P_(d), ki, x[0], x[1], P_(out))
        return out

    def vjp(x, b):
        out = np.empty(2)
        H.a_eos_vjp(P_(d), ki, x[0], x[1], b[0], b[1], P_(out))
        return out

    _check(fwd, vjp, x, 2, rng)


@pytest.mark.parametrize("ueq_from_f", [1, 0])
def test_closed_form_collision_equals_the_moment_form(H, ueq_from_f):
    """With s_q = s_pi = 1 and m^eq = M-hat f^eq the step uses the closed form
    f^eq(rho, u + F/rho) + relaxed second-order non-equilibrium; in double it must
    equal the moment-space collision to rounding, for any s_e, s_v."""
    for se, sv in ((1.25, 0.8), (0.6, 1.7)):
        p = W.base_params(2, 2, 2, s_e=se, s_v=sv, s_q=1.0, s_pi=1.0)
        d, k = _dk(p)
        ki = k.ctypes.data_as(ct.POINTER(ct.c_int))
        rng = np.random.default_rng(int(10 * se) + ueq_from_f)
        w = np.array(W.W19)
        for rho in (0.4, 6.3):
            for _ in range(20):
                f = np.ascontiguousarray(w * rho * (1 + 0.1 * rng.standard_normal(19)))
                F = np.ascontiguousarray(0.02 * rng.standard_normal(3))
                a, b = np.empty(19), np.empty(19)
                H.a_collide19(P_(d), ki, P_(f), ueq_from_f, P_(F), P_(a))
                H.a_collide19_fast(P_(d), ki, P_(f), ueq_from_f, P_(F), P_(b))
                assert np.max(np.abs(a - b)) <= 1e-13 * rho, np.max(np.abs(a - b))


@pytest.mark.parametrize("ueq_from_f", [1, 0])
def test_closed_form_collision_vjp(H, ueq_from_f):
    """The product of the closed form equals the general product (rate-1 case) and
    central differences of the forward."""
    for se, sv in ((1.25, 0.8), (0.6, 1.7)):
        p = W.base_params(2, 2, 2, s_e=se, s_v=sv, s_q=1.0, s_pi=1.0)
        d, k = _dk(p)
        ki = k.ctypes.data_as(ct.POINTER(ct.c_int))
        rng = np.random.default_rng(int(10 * sv) + 3 * ueq_from_f)
        w = np.array(W.W19)
        for rho in (0.4, 6.3):
            f = np.ascontiguousarray(w * rho * (1 + 0.1 * rng.standard_normal(19)))
            F = np.ascontiguousarray(0.02 * rng.standard_normal(3))
            x = np.concatenate([f, F])
            for _ in range(4):
                b = np.ascontiguousarray(rng.standard_normal(19))
                fb1, Fb1, fb2, Fb2 = np.empty(19), np.empty(3), np.empty(19), np.empty(3)
                H.a_collide19_vjp(P_(d), ki, P_(f), ueq_from_f, P_(F), P_(b), P_(fb1), P_(Fb1))
                H.a_collide19_fast_vjp(P_(d), ki, P_(f), ueq_from_f, P_(F), P_(b), P_(fb2), P_(Fb2))
                assert np.max(np.abs(fb1 - fb2)) <= 1e-12 * max(1.0, np.max(np.abs(fb1)))
                assert np.max(np.abs(Fb1 - Fb2)) <= 1e-12 * max(1.0, np.max(np.abs(Fb1)))

            def fwd(x):
                fs = np.empty(19)
                H.a_collide19_fast(P_(d), ki, P_(np.ascontiguousarray(x[:19])), ueq_from_f,
                                   P_(np.ascontiguousarray(x[19:])), P_(fs))
                return fs

            def vjp(x, b):
                fb, Fb = np.empty(19), np.empty(3)
                H.a_collide19_fast_vjp(P_(d), ki, P_(np.ascontiguousarray(x[:19])), ueq_from_f,
                                       P_(np.ascontiguousarray(x[19:])), P_(np.ascontiguousarray(b)), P_(fb),
                                       P_(Fb))
                return np.concatenate([fb, Fb])

            _check(fwd, vjp, x, 19, rng)
