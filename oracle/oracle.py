"""ctypes wrapper of the FP64 CPU oracle (oracle/lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py, never by the product path.  It imports nothing from the
CUDA package.

Arrays are numpy float64, populations in SoA layout f[i, z, y, x] (i.e. the
flat index i*N + x + nx*(y + ny*z)).
"""
import ctypes as ct
import os

import numpy as np

from .build import build_oracle

PERIODIC, WALL, OPEN = 0, 1, 2
OK, ERR_ARG, ERR_NONFINITE, ERR_PSI_DOMAIN = 0, -1, -3, -4

_D = ct.c_double
_PD = ct.POINTER(ct.c_double)


class OrcParams(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("a", _D), ("b", _D), ("R", _D), ("omega", _D), ("G", _D),
        ("s_e", _D), ("s_v", _D), ("s_q", _D), ("s_pi", _D),
        ("cv", _D), ("wbar", _D), ("lambda_l", _D), ("lambda_v", _D),
        ("rho_l", _D), ("rho_v", _D),
        ("vartheta", ct.c_int), ("meq_printed", ct.c_int), ("wall_ueq_zero", ct.c_int),
        ("eos_kind", ct.c_int), ("eos_c0", _D),
        ("face_kind", ct.c_int * 6), ("face_T", _D * 6), ("face_rho", _D * 6),
        ("face_theta_deg", _D * 6), ("face_T_fixed", ct.c_int * 6),
    ]


class OrcFields(ct.Structure):
    _fields_ = [(n, _PD) for n in ("rho", "T", "psi", "p", "dpdT", "ux", "uy", "uz", "Fx", "Fy", "Fz")]


_libs = {}


def lib(omp: bool = False):
    """The serial oracle library, or (omp=True) the same source built with OpenMP."""
    if omp not in _libs:
        path = build_oracle(omp=omp)
        L = ct.CDLL(path)
        P = ct.POINTER(OrcParams)
        L.orc_Tc.restype = _D
        L.orc_Tc.argtypes = [P]
        for fn in ("orc_p_eos", "orc_dpdT", "orc_dpdrho"):
            getattr(L, fn).restype = _D
            getattr(L, fn).argtypes = [P, _D, _D]
        L.orc_maxwell.argtypes = [P, _D, _PD, _PD, _PD]
        L.orc_tables.argtypes = [ct.c_void_p] * 7
        L.orc_tables.restype = None
        L.orc_feq19.argtypes = [_D, _PD, _PD]
        L.orc_feq19.restype = None
        L.orc_meq19.argtypes = [P, _D, _PD, _PD]
        L.orc_meq19.restype = None
        L.orc_collide19.argtypes = [P, _PD, _D, _PD, _PD, _PD]
        L.orc_collide19.restype = None
        L.orc_collide7.argtypes = [P, _PD, _D, _D, _PD, _D, _D, _D, _PD]
        L.orc_collide7.restype = None
        L.orc_zouhe.argtypes = [P, ct.c_int, _PD, _PD]
        L.orc_zouhe.restype = None
        L.orc_check.argtypes = [P]
        L.orc_macros.argtypes = [P, _PD, _PD, ct.POINTER(OrcFields)]
        L.orc_step.argtypes = [P, ct.POINTER(_PD), _PD, _PD, _PD, _PD, ct.POINTER(OrcFields)]
        L.orc_run.argtypes = [P, ct.POINTER(_PD), _PD, _PD, ct.c_int]
        L.orc_step_hist.argtypes = [P, ct.POINTER(_PD), _PD, _PD, _PD, _PD, _PD, _PD]
        L.orc_run_hist.argtypes = [P, ct.POINTER(_PD), _PD, _PD, _PD, ct.c_int]
        L.orc_stream_map19.argtypes = [P, ct.POINTER(ct.c_int)]
        L.orc_stream_map7.argtypes = [P, ct.POINTER(ct.c_int)]
        L.orc_node_class.argtypes = [P, ct.POINTER(ct.c_ubyte)]
        L.orc_init_state.argtypes = [P, _PD, _PD, _PD, _PD]
        L.orc_init_state.restype = None
        L.orc_threads.argtypes = [ct.c_int]
        _libs[omp] = L
    return _libs[omp]


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_PD)


def make_params(d: dict) -> OrcParams:
    """Builds the C struct from a plain dict (see workloads.base_params)."""
    p = OrcParams()
    for name, _ in OrcParams._fields_:
        if name not in d:
            continue
        v = d[name]
        if name.startswith("face_"):
            arr = getattr(p, name)
            for k in range(6):
                arr[k] = v[k]
        else:
            setattr(p, name, v)
    return p


def _tface_array(tface):
    arr = (_PD * 6)()
    keep = []
    for k in range(6):
        if tface is not None and tface[k] is not None:
            a = np.ascontiguousarray(tface[k], dtype=np.float64)
            keep.append(a)
            arr[k] = _ptr(a)
        else:
            arr[k] = _PD()
    return arr, keep


class Oracle:
    """FP64 reference lattice.  params: dict with the orc_params fields.  omp=True runs the
    OpenMP build (the same arithmetic on all host cores; threads() reports the count)."""

    def __init__(self, params: dict, omp: bool = False):
        self.omp = omp
        self.d = dict(params)
        self.p = make_params(self.d)
        self.shape = (self.p.nz, self.p.ny, self.p.nx)
        self.N = self.p.nx * self.p.ny * self.p.nz
        self.tface = None
        if lib(self.omp).orc_check(ct.byref(self.p)) != 0:
            raise ValueError("oracle rejects these parameters")

    # thermodynamics
    def Tc(self):
        return lib(self.omp).orc_Tc(ct.byref(self.p))

    def p_eos(self, rho, T):
        return lib(self.omp).orc_p_eos(ct.byref(self.p), rho, T)

    def dpdT(self, rho, T):
        return lib(self.omp).orc_dpdT(ct.byref(self.p), rho, T)

    def dpdrho(self, rho, T):
        return lib(self.omp).orc_dpdrho(ct.byref(self.p), rho, T)

    def maxwell(self, T):
        rv, rl, ps = _D(), _D(), _D()
        st = lib(self.omp).orc_maxwell(ct.byref(self.p), T, ct.byref(rv), ct.byref(rl), ct.byref(ps))
        if st != 0:
            raise ValueError("no coexistence at this temperature")
        return rv.value, rl.value, ps.value

    # lattice
    def set_face_T(self, tface):
        """tface: list of 6 arrays (or None) of per-node Dirichlet temperatures."""
        self.tface = tface

    def init_state(self, rho0, T0):
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64).reshape(-1)
        T0 = np.ascontiguousarray(T0, dtype=np.float64).reshape(-1)
        f = np.empty((19, self.N))
        g = np.empty((7, self.N))
        lib(self.omp).orc_init_state(ct.byref(self.p), _ptr(rho0), _ptr(T0), _ptr(f), _ptr(g))
        return f, g

    def step(self, f, g, diag=False):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(7, self.N)
        fo = np.empty_like(f)
        go = np.empty_like(g)
        tf, keep = _tface_array(self.tface)
        flds, out = self._fields_struct() if diag else (None, None)
        st = lib(self.omp).orc_step(ct.byref(self.p), tf, _ptr(f), _ptr(g), _ptr(fo), _ptr(go),
                            ct.byref(flds) if diag else None)
        del keep
        if diag:
            return st, fo, go, out
        return st, fo, go

    def run(self, f, g, nsteps):
        f = np.array(f, dtype=np.float64).reshape(19, self.N)
        g = np.array(g, dtype=np.float64).reshape(7, self.N)
        tf, keep = _tface_array(self.tface)
        st = lib(self.omp).orc_run(ct.byref(self.p), tf, _ptr(f), _ptr(g), int(nsteps))
        del keep
        return st, f, g

    def history(self, g):
        """T history of a state at rest before t = 0: T(t-1) = T(t-2) = T = sum g."""
        T = np.asarray(g, dtype=np.float64).reshape(7, self.N).sum(0)
        return np.stack([T, T])

    def step_hist(self, f, g, Th):
        """One step with the T history Th = [T(t-1), T(t-2)] (vartheta = 1 needs it);
        returns (status, f, g, [T(t), T(t-1)])."""
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(7, self.N)
        Th = np.ascontiguousarray(Th, dtype=np.float64).reshape(2, self.N)
        fo, go, Tho = np.empty_like(f), np.empty_like(g), np.empty_like(Th)
        tf, keep = _tface_array(self.tface)
        st = lib(self.omp).orc_step_hist(ct.byref(self.p), tf, _ptr(f), _ptr(g), _ptr(Th), _ptr(fo), _ptr(go), _ptr(Tho))
        del keep
        return st, fo, go, Tho

    def run_hist(self, f, g, Th, nsteps):
        f = np.array(f, dtype=np.float64).reshape(19, self.N)
        g = np.array(g, dtype=np.float64).reshape(7, self.N)
        Th = np.array(Th, dtype=np.float64).reshape(2, self.N)
        tf, keep = _tface_array(self.tface)
        st = lib(self.omp).orc_run_hist(ct.byref(self.p), tf, _ptr(f), _ptr(g), _ptr(Th), int(nsteps))
        del keep
        return st, f, g, Th

    def threads(self, n: int = 0):
        """Threads of the per-cell loops (n > 0 sets them; OpenMP build only)."""
        return lib(self.omp).orc_threads(int(n))

    def _fields_struct(self):
        out = {n: np.empty(self.N) for n, _ in OrcFields._fields_}
        s = OrcFields(*[_ptr(out[n]) for n, _ in OrcFields._fields_])
        return s, out

    def macros(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(7, self.N)
        s, out = self._fields_struct()
        st = lib(self.omp).orc_macros(ct.byref(self.p), _ptr(f), _ptr(g), ct.byref(s))
        return st, out

    def stream_map19(self):
        m = np.empty(19 * self.N, dtype=np.int32)
        lib(self.omp).orc_stream_map19(ct.byref(self.p), m.ctypes.data_as(ct.POINTER(ct.c_int)))
        return m

    def stream_map7(self):
        m = np.empty(7 * self.N, dtype=np.int32)
        lib(self.omp).orc_stream_map7(ct.byref(self.p), m.ctypes.data_as(ct.POINTER(ct.c_int)))
        return m

    def node_class(self):
        m = np.empty(self.N, dtype=np.uint8)
        lib(self.omp).orc_node_class(ct.byref(self.p), m.ctypes.data_as(ct.POINTER(ct.c_ubyte)))
        return m

    # per-cell pieces
    def collide19(self, f, rho, ueq, F):
        f = np.ascontiguousarray(f, dtype=np.float64)
        ueq = np.ascontiguousarray(ueq, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        out = np.empty(19)
        lib(self.omp).orc_collide19(ct.byref(self.p), _ptr(f), rho, _ptr(ueq), _ptr(F), _ptr(out))
        return out

    def collide7(self, g, rho, T, u, divu, dpdT, d2T=0.0):
        g = np.ascontiguousarray(g, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty(7)
        lib(self.omp).orc_collide7(ct.byref(self.p), _ptr(g), rho, T, _ptr(u), divu, dpdT, d2T, _ptr(out))
        return out

    def zouhe(self, face, f, F):
        f = np.array(f, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        lib(self.omp).orc_zouhe(ct.byref(self.p), int(face), _ptr(F), _ptr(f))
        return f

    def meq19(self, rho, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty(19)
        lib(self.omp).orc_meq19(ct.byref(self.p), rho, _ptr(u), _ptr(out))
        return out


def feq19(rho, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(19)
    lib().orc_feq19(rho, _ptr(u), _ptr(out))
    return out


def tables():
    c19 = np.empty((19, 3), dtype=np.int32)
    w19 = np.empty(19)
    c7 = np.empty((7, 3), dtype=np.int32)
    Mh = np.empty((19, 19))
    Mhi = np.empty((19, 19))
    M7 = np.empty((7, 7))
    M7i = np.empty((7, 7))
    lib().orc_tables(c19.ctypes.data, w19.ctypes.data, c7.ctypes.data, Mh.ctypes.data, Mhi.ctypes.data,
                     M7.ctypes.data, M7i.ctypes.data)
    return dict(c19=c19, w19=w19, c7=c7, Mhat=Mh, Mhat_inv=Mhi, M7=M7, M7_inv=M7i)
