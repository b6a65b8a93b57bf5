"""The Python binding checks every buffer before the library reads or writes it.

The C ABI takes raw pointers and sizes implied by the lattice, so a buffer of the wrong
dtype, too short, non-contiguous, or in the wrong memory would be accessed past its end
(host memory, or device memory on the GPU).  These checks run on the host, before any call
into the library: here the library is replaced by a function that fails the test if it is
reached, and a Lattice is made without lbm_init.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2206_00946_gb300 import lbm
from paper_2206_00946_gb300 import workloads as W

torch = pytest.importorskip("torch")

NX, NY, NZ = 5, 4, 3
N = NX * NY * NZ


class _Reached(Exception):
    pass


@pytest.fixture
def lat(monkeypatch):
    def reached(*args, **kwargs):
        raise _Reached()

    monkeypatch.setattr(lbm, "load", reached)
    L = object.__new__(lbm.Lattice)
    L._ctx = ct.c_void_p()
    L.params = W.base_params(NX, NY, NZ, face_kind=[0, 0, 0, 0, 1, 2], face_T=[0, 0, 0, 0, 1.0, 1.0],
                             face_rho=[0, 0, 0, 0, 0, 1.0])
    L._p = lbm.make_params(L.params)
    L.N = N
    L.lbm_checkpoint_bytes = lambda: 256 + 104 * N
    return L


def f32(n):
    return np.zeros(n, dtype=np.float32)


def test_good_buffers_reach_the_library(lat):
    with pytest.raises(_Reached):
        lat.lbm_set_state(f32(19 * N), f32(7 * N))
    with pytest.raises(_Reached):
        lat.lbm_set_state(torch.zeros(19, N), torch.zeros(7, N))  # CPU tensors: host memory
    with pytest.raises(_Reached):
        lat.lbm_set_face_T(4, f32(NX * NY))
    with pytest.raises(_Reached):
        lat.lbm_macros(rho=f32(N), T=f32(N))
    with pytest.raises(_Reached):
        lat.lbm_stream_map(np.zeros(19 * N, np.int32), np.zeros(7 * N, np.int32), np.zeros(N, np.uint8))
    with pytest.raises(_Reached):
        lat.lbm_checkpoint(np.zeros(256 + 104 * N, np.uint8))


@pytest.mark.parametrize("call,exc", [
    (lambda L: L.lbm_set_state(np.zeros(19 * N), f32(7 * N)), TypeError),                 # float64
    (lambda L: L.lbm_set_state(f32(19 * N - 1), f32(7 * N)), ValueError),                  # short
    (lambda L: L.lbm_set_state(np.zeros((7 * N, 19), np.float32).T, f32(7 * N)), ValueError),  # strided
    (lambda L: L.lbm_set_state(np.zeros(19 * N, np.float16), f32(7 * N)), TypeError),      # half the bytes
    (lambda L: L.lbm_get_state(f32(19 * N), torch.zeros(7 * N, dtype=torch.float64)), TypeError),
    (lambda L: L.lbm_set_face_T(4, f32(NX * NY - 1)), ValueError),
    (lambda L: L.lbm_set_face_T(0, f32(NY * NZ - 1)), ValueError),
    (lambda L: L.lbm_set_face_T(6, f32(NX * NY)), ValueError),
    (lambda L: L.lbm_macros(rho=np.zeros(N, np.int32)), TypeError),
    (lambda L: L.lbm_macros(rho=f32(N), T=f32(N - 1)), ValueError),
    (lambda L: L.lbm_stream_map(np.zeros(19 * N, np.float32)), TypeError),
    (lambda L: L.lbm_stream_map(None, np.zeros(7 * N - 1, np.int32)), ValueError),
    (lambda L: L.lbm_checkpoint(np.zeros(256 + 104 * N - 1, np.uint8)), ValueError),
    (lambda L: L.lbm_restore(np.zeros(256 + 104 * N, np.int8)), TypeError),
    (lambda L: L.lbm_adjoint_step(3, f32(N)), ValueError),                                 # host seed
    (lambda L: L.lbm_adjoint_state(f32(19 * N), [0.0] * (7 * N)), TypeError),
    (lambda L: lbm.lbm_reduce_static(f32(19 * N), f32(7 * N), N, 5.0, 0.38, 6.5, np.zeros(4)), ValueError),
])
def test_bad_buffers_are_stopped_before_the_library(lat, call, exc):
    with pytest.raises(exc):
        call(lat)


def test_lattice_checks_its_initial_fields(monkeypatch):
    def reached(*args, **kwargs):
        raise _Reached()

    monkeypatch.setattr(lbm, "load", reached)
    p = W.base_params(NX, NY, NZ)
    with pytest.raises(TypeError):
        lbm.Lattice(p, np.ones(N), np.ones(N, np.float32))                  # float64 rho0
    with pytest.raises(ValueError):
        lbm.Lattice(p, np.ones(N - 1, np.float32), np.ones(N, np.float32))  # short
    with pytest.raises(_Reached):
        lbm.Lattice(p, np.ones(N, np.float32), np.ones(N, np.float32))
