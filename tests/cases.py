"""Shared inputs and error measures of the parity tests (GPU and host harness):
the small lattices with every boundary kind, seeded droplet states, the population
error relative to the workloads' smallest physical scale, and the rounding bound
of the 16-bit storage forms."""
import numpy as np
import pytest

from paper_2206_00946_gb300 import lbm, workloads as W

W7 = W.w7(0.75)
# the 16-bit forms; the per-cell-reference form runs after every other test (see conftest)
F16_LOCAL = pytest.param(lbm.STORE_F16_LOCAL, marks=pytest.mark.per_cell_refs, id="f16local")
STORAGES_16 = [lbm.STORE_F16_SHIFTED, lbm.STORE_BF16_SHIFTED, F16_LOCAL]


def f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def droplet_state(p, thermo, seed, amp=0.02, R=None):
    """Populations around a tanh droplet with seeded noise (non-zero force and velocity everywhere)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x, y, z = W.grid(nx, ny, nz)
    R = R if R is not None else 0.3 * min(nx, ny, nz) + 1.0
    r = np.sqrt((x - 0.45 * nx) ** 2 + (y - 0.55 * ny) ** 2 + (z - 0.5 * nz) ** 2)
    rho = W.tanh_profile(r - R, thermo["rho_v"], thermo["rho_l"], 3.0)
    Tm = thermo["Ts"] * (1 + 0.01 * np.sin(0.3 * x + 0.2 * y + 0.1 * z))
    f, g = W.random_populations(nx, ny, nz, rho.reshape(-1), Tm.reshape(-1), W.W19, W7, amp, seed)
    return f32(f), f32(g)


def relerr(a, b):
    return float(np.max(np.abs(a.astype(np.float64) - b) / np.abs(b)))


def pop_err(a, b, thermo):
    """Max population error relative to max(|b|, floor_i) (see the module docstring)."""
    q = a.shape[0]
    floor = (W.W19 * thermo["rho_v"]) if q == 19 else (W7 * 0.5 * thermo["Ts"])
    den = np.maximum(np.abs(b), floor[:, None])
    return float(np.max(np.abs(a.astype(np.float64) - b) / den))


CASES = {
    "periodic": dict(shape=(12, 10, 9), face_kind=[0] * 6),
    "walls_z": dict(shape=(8, 9, 10), face_kind=[0, 0, 0, 0, 1, 1]),
    "open_all": dict(shape=(9, 8, 10), face_kind=[2] * 6),
    "wall_bottom_open_top": dict(shape=(10, 9, 8), face_kind=[0, 0, 0, 0, 1, 2]),
    "walls_xy_theta": dict(shape=(7, 8, 9), face_kind=[1, 1, 1, 1, 0, 0], theta=[70, 110, 60, 120, 90, 90]),
    "ragged_open_x": dict(shape=(13, 7, 11), face_kind=[2, 2, 0, 0, 0, 0]),
    "column_1x1": dict(shape=(1, 1, 40), face_kind=[0, 0, 0, 0, 1, 1]),
    "multi_tile_plane": dict(shape=(40, 30, 6), face_kind=[0, 0, 2, 2, 0, 0]),
    # Sec. 4.2: periodic velocity field, every boundary node layer held at its face temperature
    "periodic_held_T": dict(shape=(9, 10, 11), face_kind=[0] * 6, held=[1] * 6),
}


def case_params(name, thermo):
    c = CASES[name]
    nx, ny, nz = c["shape"]
    Ts = thermo["Ts"]
    return W.base_params(nx, ny, nz, rho_l=thermo["rho_l"], rho_v=thermo["rho_v"], lambda_l=0.4, lambda_v=0.2,
                         face_kind=c["face_kind"], face_T=[Ts * (1 + 0.01 * k) for k in range(6)],
                         face_rho=[thermo["rho_v"] * (1 + 0.02 * k) for k in range(6)],
                         face_theta_deg=c.get("theta", [90] * 6), face_T_fixed=c.get("held", [0] * 6))


HALF_ULP = {lbm.STORE_F16_SHIFTED: 2.0 ** -11, lbm.STORE_BF16_SHIFTED: 2.0 ** -8, lbm.STORE_F16_LOCAL: 2.0 ** -11}


def _local_refs(f, g):
    """Per-cell shifts w_i rho(cell), w_i T(cell) of a state (19 x N, 7 x N)."""
    return (W.W19[:, None] * f.astype(np.float64).sum(0)[None, :],
            W7[:, None] * g.astype(np.float64).sum(0)[None, :])


def _face_nodes(p):
    """Cells on a non-periodic face or a held temperature layer (where Zou-He and the
    extrapolation rewrite populations)."""
    x, y, z = (a.reshape(-1) for a in W.grid(p["nx"], p["ny"], p["nz"]))
    n = (p["nx"], p["ny"], p["nz"])
    m = np.zeros(x.size, dtype=bool)
    held = p.get("face_T_fixed", [0] * 6)
    for face, kind in enumerate(p["face_kind"]):
        if kind != 0 or held[face]:
            coord = (x, y, z)[face // 2]
            m |= coord == (0 if face % 2 == 0 else n[face // 2] - 1)
    return m


def _storage_bound_ok(gpu, ora, ref, k, thermo, face):
    """Excess of |gpu - oracle| over the rounding bound.  Interior nodes: half an ulp of the
    stored deviation d.  Face nodes: their boundary rules combine up to ~10 populations that
    were already rounded when they were stored, so the bound there is linear propagation,
    half an ulp of (|d_i| + 2 max over cells of sum_j |d_j|)."""
    q = ora.shape[0]
    floor = (W.W19 * thermo["rho_v"]) if q == 19 else (W7 * 0.5 * thermo["Ts"])
    scale = np.maximum(np.abs(ora), floor[:, None])
    d = np.abs(ora - (ref if ref.ndim == 2 else ref[:, None]))
    prop = np.where(face[None, :], 2.0 * d.sum(0).max(), 0.0)
    bound = 1.02 * k * (d + prop) + 1e-5 * scale + 6e-8
    err = np.abs(gpu.astype(np.float64) - ora)
    return float((err - bound).max()), float((err / scale).max())
