"""Thin ctypes binding of liblbm.so (include/lbm.h): same function names,
argument marshalling only.  Every step of the lattice update runs in the
library's CUDA kernels; nothing here computes on the host.

Device arrays are passed as torch CUDA tensors (their data_ptr()) or raw
integer pointers; host arrays as numpy arrays.  The library must have been
built (``python -m paper_2206_00946_gb300.build``); loading fails loudly if it
is missing.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LBM_LIB") or os.path.join(_HERE, "_lib", "liblbm.so")

OK, ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_PSI_DOMAIN, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
FACE_PERIODIC, FACE_WALL, FACE_OPEN = 0, 1, 2
STORE_F32, STORE_F16_SHIFTED, STORE_BF16_SHIFTED, STORE_F16_LOCAL = 0, 1, 2, 3
MEM_DEVICE, MEM_HOST = 0, 1
SCHED_FUSED, SCHED_PHASES, SCHED_SLABS = 0, 1, 2

_D = ct.c_double


class lbm_params(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
        ("a", _D), ("b", _D), ("R", _D), ("omega", _D), ("G", _D),
        ("s_e", _D), ("s_v", _D), ("s_q", _D), ("s_pi", _D),
        ("cv", _D), ("wbar", _D), ("lambda_l", _D), ("lambda_v", _D),
        ("rho_l", _D), ("rho_v", _D),
        ("vartheta", ct.c_int), ("meq_printed", ct.c_int), ("wall_ueq_zero", ct.c_int),
        ("eos_kind", ct.c_int), ("eos_c0", _D),
        ("face_kind", ct.c_int * 6), ("face_T", _D * 6), ("face_rho", _D * 6), ("face_theta_deg", _D * 6),
        ("storage", ct.c_int), ("store_rho_ref", _D), ("store_T_ref", _D), ("schedule", ct.c_int),
        ("face_T_fixed", ct.c_int * 6),
    ]


# every symbol declared in include/lbm.h
EXPORTS = ["lbm_init", "lbm_set_state", "lbm_get_state", "lbm_set_face_T", "lbm_step", "lbm_macros",
           "lbm_reduce", "lbm_sync", "lbm_stream_map", "lbm_destroy", "lbm_status_string", "lbm_Tc",
           "lbm_maxwell", "lbm_launches_per_step", "lbm_step_launches", "lbm_profile", "lbm_profile_read", "lbm_reduce_static",
           "lbm_checkpoint_bytes", "lbm_checkpoint", "lbm_restore", "lbm_record", "lbm_adjoint_step",
           "lbm_adjoint_state", "lbm_batch_create", "lbm_batch_tune", "lbm_batch_step", "lbm_batch_sync",
           "lbm_batch_cells", "lbm_batch_destroy", "lbm_batch_inject_stall", "lbm_inject_stall"]
PROFILE_KINDS = ["phaseA", "phaseB", "phaseC", "phaseD", "fused", "phaseC7"]

_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {lbm_status_string(status)} ({status})")


def load(path: str = LIB_PATH):
    """Loads liblbm.so; raises if the CUDA library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbm.so not built at {path}; run python -m paper_2206_00946_gb300.build")
    L = ct.CDLL(path)
    vp, P = ct.c_void_p, ct.POINTER(lbm_params)
    L.lbm_init.argtypes = [ct.POINTER(vp), P, vp, vp, ct.c_int, vp]
    L.lbm_set_state.argtypes = [vp, vp, vp, ct.c_int]
    L.lbm_get_state.argtypes = [vp, vp, vp, ct.c_int]
    L.lbm_set_face_T.argtypes = [vp, ct.c_int, vp, ct.c_int]
    L.lbm_step.argtypes = [vp, ct.c_int]
    L.lbm_inject_stall.argtypes = [vp]
    L.lbm_macros.argtypes = [vp, vp, vp, vp, vp, vp, ct.c_int]
    L.lbm_reduce.argtypes = [vp, ct.POINTER(_D)]
    L.lbm_sync.argtypes = [vp]
    L.lbm_stream_map.argtypes = [vp, vp, vp, vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_status_string.argtypes = [ct.c_int]
    L.lbm_status_string.restype = ct.c_char_p
    L.lbm_Tc.argtypes = [P]
    L.lbm_Tc.restype = _D
    L.lbm_maxwell.argtypes = [P, _D, ct.POINTER(_D), ct.POINTER(_D), ct.POINTER(_D)]
    L.lbm_launches_per_step.argtypes = [vp]
    L.lbm_step_launches.argtypes = [vp, ct.c_int]
    L.lbm_step_launches.restype = ct.c_longlong
    L.lbm_profile.argtypes = [vp, ct.c_int]
    L.lbm_profile_read.argtypes = [vp, vp, vp, ct.c_int]
    L.lbm_reduce_static.argtypes = [vp, vp, ct.c_longlong, _D, _D, _D, vp, vp]
    L.lbm_checkpoint_bytes.argtypes = [vp]
    L.lbm_checkpoint_bytes.restype = ct.c_longlong
    L.lbm_checkpoint.argtypes = [vp, vp, ct.c_int]
    L.lbm_restore.argtypes = [vp, vp, ct.c_int]
    L.lbm_record.argtypes = [vp, ct.c_int, ct.c_int]
    L.lbm_adjoint_step.argtypes = [vp, ct.c_int, vp, vp, vp, vp]
    L.lbm_adjoint_state.argtypes = [vp, vp, vp, ct.c_int]
    L.lbm_batch_create.argtypes = [ct.POINTER(vp), ct.POINTER(vp), ct.c_int]
    L.lbm_batch_tune.argtypes = [vp, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    L.lbm_batch_step.argtypes = [vp, ct.c_int]
    L.lbm_batch_sync.argtypes = [vp]
    L.lbm_batch_cells.argtypes = [vp]
    L.lbm_batch_cells.restype = ct.c_longlong
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_inject_stall.argtypes = [vp]
    _lib = L
    return L


def make_params(d: dict) -> lbm_params:
    p = lbm_params()
    for name, _ in lbm_params._fields_:
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


def _ptr(x):
    """Device/host pointer of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array is not C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor is not contiguous")
        return x.data_ptr()
    raise TypeError(type(x))


def _is_device(x):
    return bool(getattr(x, "is_cuda", False))


def _mem_of(*xs):
    """LBM_MEM_HOST or LBM_MEM_DEVICE for the buffers of one call (all alike)."""
    kinds = {_is_device(x) for x in xs if x is not None and not isinstance(x, int)}
    if len(kinds) > 1:
        raise ValueError("the buffers of one call must be all host or all device memory")
    return MEM_DEVICE if (not kinds or kinds.pop()) else MEM_HOST


_DTYPES = {"f4": (np.float32, "float32"), "f8": (np.float64, "float64"), "i4": (np.int32, "int32"),
           "u1": (np.uint8, "uint8")}


def _arr(x, kind, count, what, device=None):
    """Checks a buffer before the library reads or writes `count` elements of it: the C ABI
    takes raw pointers, so a wrong type or a short buffer would be read or written past its
    end.  device: True / False requires device / host memory; None accepts either."""
    if x is None:
        return
    npdt, tname = _DTYPES[kind]
    if isinstance(x, np.ndarray):
        ok, contig, n = x.dtype == npdt, x.flags["C_CONTIGUOUS"], x.size
    elif hasattr(x, "data_ptr"):
        ok, contig, n = str(x.dtype) == "torch." + tname, x.is_contiguous(), x.numel()
    else:
        raise TypeError(f"{what}: a numpy array or a torch tensor is needed, not {type(x).__name__}")
    if not ok:
        raise TypeError(f"{what}: dtype {x.dtype}, {tname} needed")
    if not contig:
        raise ValueError(f"{what}: not contiguous")
    if n < count:
        raise ValueError(f"{what}: {n} elements, {count} needed")
    if device is not None and _is_device(x) != device:
        raise ValueError(f"{what}: {'device' if device else 'host'} memory needed")


def _check(st, where):
    if st != OK:
        raise LBMError(st, where)


def lbm_status_string(st: int) -> str:
    return load().lbm_status_string(int(st)).decode()


def lbm_Tc(params: dict) -> float:
    return load().lbm_Tc(ct.byref(make_params(params)))


def lbm_maxwell(params: dict, T: float):
    rv, rl, ps = _D(), _D(), _D()
    _check(load().lbm_maxwell(ct.byref(make_params(params)), T, ct.byref(rv), ct.byref(rl), ct.byref(ps)),
           "lbm_maxwell")
    return rv.value, rl.value, ps.value


def lbm_reduce_static(f, g, n_cells, cv, rho_v, rho_l, out, stream=None):
    """Reductions of caller-owned device populations into a device array of 4 doubles, with no
    device allocation (see include/lbm.h); returns the status code."""
    _arr(f, "f4", 19 * int(n_cells), "f", device=True)
    _arr(g, "f4", 7 * int(n_cells), "g", device=True)
    _arr(out, "f8", 4, "out", device=True)
    return load().lbm_reduce_static(_ptr(f), _ptr(g), int(n_cells), float(cv), float(rho_v), float(rho_l),
                                    _ptr(out), stream)


class Lattice:
    """Owns one lbm_ctx.  Methods mirror the C functions one to one."""

    def __init__(self, params: dict, rho0=None, T0=None, stream: int | None = None):
        self._ctx = ct.c_void_p()
        self.params = dict(params)
        self._p = make_params(self.params)
        self.N = self._p.nx * self._p.ny * self._p.nz
        _arr(rho0, "f4", self.N, "rho0")
        _arr(T0, "f4", self.N, "T0")
        mem = _mem_of(rho0, T0)
        L = load()
        self._keep = (rho0, T0)
        st = L.lbm_init(ct.byref(self._ctx), ct.byref(self._p), _ptr(rho0), _ptr(T0), mem, stream)
        _check(st, "lbm_init")

    def close(self):
        if self._ctx:
            load().lbm_destroy(self._ctx)
            self._ctx = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _face_len(self, face):
        n = (self._p.nx, self._p.ny, self._p.nz)
        a, b = [n[k] for k in range(3) if k != face // 2]
        return a * b

    def lbm_set_state(self, f, g):
        _arr(f, "f4", 19 * self.N, "f")
        _arr(g, "f4", 7 * self.N, "g")
        _check(load().lbm_set_state(self._ctx, _ptr(f), _ptr(g), _mem_of(f, g)), "lbm_set_state")

    def lbm_get_state(self, f, g):
        _arr(f, "f4", 19 * self.N, "f")
        _arr(g, "f4", 7 * self.N, "g")
        st = load().lbm_get_state(self._ctx, _ptr(f), _ptr(g), _mem_of(f, g))
        return st

    def lbm_checkpoint_bytes(self):
        return int(load().lbm_checkpoint_bytes(self._ctx))

    def lbm_checkpoint(self, dst):
        """Writes the state image into dst (uint8 numpy array or torch tensor of lbm_checkpoint_bytes())."""
        _arr(dst, "u1", self.lbm_checkpoint_bytes(), "dst")
        return load().lbm_checkpoint(self._ctx, _ptr(dst), _mem_of(dst))

    def lbm_restore(self, src):
        _arr(src, "u1", self.lbm_checkpoint_bytes(), "src")
        _check(load().lbm_restore(self._ctx, _ptr(src), _mem_of(src)), "lbm_restore")

    def lbm_record(self, n, K):
        """Advances n steps keeping a checkpoint every K steps for lbm_adjoint_step."""
        _check(load().lbm_record(self._ctx, int(n), int(K)), "lbm_record")

    def lbm_adjoint_step(self, n, dL_drho=None, dL_dT=None, dL_dTface=None, dL_dT0=None):
        """Adjoint of the n recorded steps; device tensors (float32 seeds, float64 outputs)."""
        nface = sum(self._face_len(f) for f in range(6) if self._p.face_kind[f] != 0)
        _arr(dL_drho, "f4", self.N, "dL_drho", device=True)
        _arr(dL_dT, "f4", self.N, "dL_dT", device=True)
        _arr(dL_dTface, "f8", nface, "dL_dTface", device=True)
        _arr(dL_dT0, "f8", self.N, "dL_dT0", device=True)
        _check(load().lbm_adjoint_step(self._ctx, int(n), _ptr(dL_drho), _ptr(dL_dT), _ptr(dL_dTface),
                                       _ptr(dL_dT0)), "lbm_adjoint_step")

    def lbm_adjoint_state(self, f_bar, g_bar):
        _arr(f_bar, "f4", 19 * self.N, "f_bar")
        _arr(g_bar, "f4", 7 * self.N, "g_bar")
        _check(load().lbm_adjoint_state(self._ctx, _ptr(f_bar), _ptr(g_bar), _mem_of(f_bar, g_bar)),
               "lbm_adjoint_state")

    def lbm_set_face_T(self, face, T_face):
        if not 0 <= int(face) < 6:
            raise ValueError(f"face {face}: 0..5 needed")
        _arr(T_face, "f4", self._face_len(int(face)), "T_face")
        _check(load().lbm_set_face_T(self._ctx, int(face), _ptr(T_face), _mem_of(T_face)), "lbm_set_face_T")

    def lbm_step(self, n=1):
        _check(load().lbm_step(self._ctx, int(n)), "lbm_step")

    def lbm_macros(self, rho=None, ux=None, uy=None, uz=None, T=None):
        for x, w in ((rho, "rho"), (ux, "ux"), (uy, "uy"), (uz, "uz"), (T, "T")):
            _arr(x, "f4", self.N, w)
        return load().lbm_macros(self._ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(T),
                                 _mem_of(rho, ux, uy, uz, T))

    def lbm_reduce(self):
        out = (_D * 4)()
        st = load().lbm_reduce(self._ctx, out)
        return st, [out[k] for k in range(4)]

    def lbm_sync(self):
        return load().lbm_sync(self._ctx)

    def lbm_inject_stall(self):
        return load().lbm_inject_stall(self._ctx)

    def lbm_stream_map(self, map19=None, map7=None, node_class=None):
        _arr(map19, "i4", 19 * self.N, "map19", device=False)
        _arr(map7, "i4", 7 * self.N, "map7", device=False)
        _arr(node_class, "u1", self.N, "node_class", device=False)
        return load().lbm_stream_map(self._ctx, _ptr(map19), _ptr(map7), _ptr(node_class))

    def lbm_launches_per_step(self):
        return load().lbm_launches_per_step(self._ctx)

    def lbm_step_launches(self, n):
        """Kernel launches of lbm_step(n)."""
        return load().lbm_step_launches(self._ctx, n)

    def lbm_profile(self, enable=True):
        _check(load().lbm_profile(self._ctx, int(bool(enable))), "lbm_profile")

    def lbm_profile_read(self):
        """{kind: (launches, total ms)} since the last lbm_profile(True)."""
        n = np.zeros(len(PROFILE_KINDS), dtype=np.int64)
        ms = np.zeros(len(PROFILE_KINDS), dtype=np.float64)
        _check(load().lbm_profile_read(self._ctx, n.ctypes.data, ms.ctypes.data, len(PROFILE_KINDS)),
               "lbm_profile_read")
        return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(PROFILE_KINDS) if n[i] > 0}

    # numpy conveniences (host copies through the same C calls)
    def state(self):
        f = np.empty((19, self.N), dtype=np.float32)
        g = np.empty((7, self.N), dtype=np.float32)
        st = self.lbm_get_state(f, g)
        return st, f, g

    def macros(self):
        out = {k: np.empty(self.N, dtype=np.float32) for k in ("rho", "ux", "uy", "uz", "T")}
        st = self.lbm_macros(**out)
        return st, out


class Batch:
    """Batched stepping of several Lattice objects (FP32, same stream) in one
    persistent launch per step.  The lattices must outlive the batch."""

    def __init__(self, lattices):
        L = load()
        self.lattices = list(lattices)
        arr = (ct.c_void_p * len(self.lattices))(*[lat._ctx.value for lat in self.lattices])
        self._b = ct.c_void_p()
        _check(L.lbm_batch_create(ct.byref(self._b), arr, len(self.lattices)), "lbm_batch_create")

    def lbm_batch_step(self, n=1):
        _check(load().lbm_batch_step(self._b, int(n)), "lbm_batch_step")

    def lbm_batch_sync(self):
        return load().lbm_batch_sync(self._b)

    def lbm_batch_inject_stall(self):
        return load().lbm_batch_inject_stall(self._b)

    def lbm_batch_tune(self):
        t, c, s = ct.c_int(), ct.c_int(), ct.c_int()
        _check(load().lbm_batch_tune(self._b, ct.byref(t), ct.byref(c), ct.byref(s)), "lbm_batch_tune")
        return t.value, c.value, s.value

    def lbm_batch_cells(self):
        return int(load().lbm_batch_cells(self._b))

    def close(self):
        if self._b:
            load().lbm_batch_destroy(self._b)
            self._b = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
