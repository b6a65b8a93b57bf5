"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and bench.py.

This module holds no arithmetic of the method itself: thermodynamic quantities
(T_c, the Maxwell coexistence densities) are passed in by the caller, who gets
them either from the oracle (tests) or from the CUDA library's host helpers
(bench).  It only lays out initial fields, boundary settings and random
numbers.

Random numbers come from a counter-based generator, splitmix64(seed ^ index),
so any cell's value can be regenerated alone.
"""
from __future__ import annotations

import numpy as np

PERIODIC, WALL, OPEN = 0, 1, 2

# Parameters used by the paper's runs (Sec. 4: a, b, R, omega, relaxation
# settings) with a = 2/49 as in the workloads of this project.
DEFAULTS = dict(
    a=2.0 / 49.0, b=2.0 / 21.0, R=1.0, omega=0.344, G=-1.0,
    s_e=1.25, s_v=0.8, s_q=1.0, s_pi=1.0,
    cv=5.0, wbar=0.75, lambda_l=1.0 / 3.0, lambda_v=1.0 / 3.0,
    rho_l=1.0, rho_v=1.0,
    vartheta=0, meq_printed=0, wall_ueq_zero=1, eos_kind=0, eos_c0=0.0, storage=0,
    store_rho_ref=0.0, store_T_ref=0.0,
    face_kind=[PERIODIC] * 6, face_T=[0.0] * 6, face_rho=[0.0] * 6, face_theta_deg=[90.0] * 6,
    face_T_fixed=[0] * 6,
)


def base_params(nx: int, ny: int, nz: int, **kw) -> dict:
    d = {k: (list(v) if isinstance(v, list) else v) for k, v in DEFAULTS.items()}
    d.update(nx=nx, ny=ny, nz=nz)
    d.update(kw)
    return d


# ----------------------------------------------------------------- RNG ------

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """Steele, Lea & Flood's splitmix64 finaliser applied to a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from splitmix64(seed ^ (stream << 40) ^ index)."""
    idx = np.arange(n, dtype=np.uint64)
    key = np.uint64(seed) ^ (np.uint64(stream) << np.uint64(40))
    r = splitmix64(idx ^ key)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def perturb(field: np.ndarray, amp: float, seed: int, stream: int = 1) -> np.ndarray:
    """field * 1 + uniform(-amp, amp) additive perturbation, seeded."""
    r = uniform(seed, field.size, stream).reshape(field.shape)
    return field + amp * (2.0 * r - 1.0)


# ------------------------------------------------------------ geometry -------

def grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def tanh_profile(dist: np.ndarray, rho_v: float, rho_l: float, W: float) -> np.ndarray:
    """rho = (rho_l+rho_v)/2 - (rho_l-rho_v)/2 tanh(2 dist / W), dist > 0 outside the liquid (Sec. 4.2)."""
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * dist / W)


def liquid_fraction(rho, rho_v, rho_l):
    return np.clip((rho - rho_v) / (rho_l - rho_v), 0.0, 1.0)


# ------------------------------------------------------------- configs ------

def slab(Tc, rho_v, rho_l, nx=16, ny=16, nz=64, W=2.0, dT_bottom=0.02, lam=(0.4, 0.2), Ts_frac=0.86):
    """Flat liquid slab z in [nz/4, 3nz/4) between bounce-back walls at z = 0 and nz-1.

    Periodic in x, y; bottom wall at (Ts_frac + dT_bottom) Tc, top wall at Ts_frac Tc,
    everything initially at T_s.
    """
    Ts = Ts_frac * Tc
    x, y, z = grid(nx, ny, nz)
    z0, z1 = nz / 4.0, 3.0 * nz / 4.0
    # signed distance to the liquid slab [z0, z1) measured from cell centres
    dist = np.maximum(z0 - 0.5 - z, z - (z1 - 0.5))
    rho0 = tanh_profile(dist, rho_v, rho_l, W)
    T0 = np.full_like(rho0, Ts)
    p = base_params(nx, ny, nz, rho_l=rho_l, rho_v=rho_v, lambda_l=lam[0], lambda_v=lam[1],
                    face_kind=[PERIODIC, PERIODIC, PERIODIC, PERIODIC, WALL, WALL],
                    face_T=[0, 0, 0, 0, Ts + dT_bottom * Tc, Ts])
    return p, rho0, T0


def conduction_column(Tc, rho_v, rho_l, L=40, W=4.0, Th_frac=1.0, Ts_frac=0.86, lam=(0.4, 0.2), cv=5.0):
    """Saturated liquid-vapour column of Sec. 4.1, reduced to 1 x 1 x L (the paper's
    200 x 10 x 10 is periodic in the two short directions, so y,z-uniform data make it
    one-dimensional; the column runs along z here).

    Vapour fills z < L/2 next to the hot wall z = 0 (Th_frac Tc), liquid the upper half
    next to the wall at T_s; tanh profile of width W between the coexistence densities,
    everything initially at T_s; conductivities lam = (liquid, vapour).
    """
    Ts = Ts_frac * Tc
    z = np.arange(L, dtype=np.float64) + 0.5
    rho0 = tanh_profile(L / 2.0 - z, rho_v, rho_l, W).reshape(L, 1, 1)
    T0 = np.full_like(rho0, Ts)
    p = base_params(1, 1, L, rho_l=rho_l, rho_v=rho_v, lambda_l=lam[0], lambda_v=lam[1], cv=cv,
                    face_kind=[PERIODIC, PERIODIC, PERIODIC, PERIODIC, WALL, WALL],
                    face_T=[0, 0, 0, 0, Th_frac * Tc, Ts])
    return p, rho0, T0


def droplet(Tc, rho_v, rho_l, n=128, R=15.0, W=5.0, seed=2206, amp=1e-4, Ts_frac=0.86, Tg_frac=1.0,
            lam=1.0 / 3.0, faces=OPEN, shape=None):
    """Spherical droplet of radius R at the domain centre in vapor at coexistence density.

    faces=OPEN: constant-pressure faces (rho_b = rho_v) on all six sides with T = Tg;
    faces=PERIODIC: the paper's own setting of Sec. 4.2, a periodic velocity field with
    the boundary node layers held at Tg.  T0 = T_s inside the liquid, Tg outside,
    blended by the liquid fraction.  rho carries a seeded uniform(-amp, amp)
    perturbation.
    """
    nx, ny, nz = (n, n, n) if shape is None else shape
    Ts, Tg = Ts_frac * Tc, Tg_frac * Tc
    x, y, z = grid(nx, ny, nz)
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
    rho0 = tanh_profile(r - R, rho_v, rho_l, W)
    if amp:
        rho0 = perturb(rho0, amp, seed)
    phi = liquid_fraction(rho0, rho_v, rho_l)
    T0 = Ts + (Tg - Ts) * (1.0 - phi)
    kinds = [faces] * 6
    p = base_params(nx, ny, nz, rho_l=rho_l, rho_v=rho_v, lambda_l=lam, lambda_v=lam,
                    face_kind=kinds, face_T=[Tg] * 6, face_rho=[rho_v] * 6,
                    face_T_fixed=[1 if faces == PERIODIC else 0] * 6)
    return p, rho0, T0


def sessile(Tc, rho_v, rho_l, nx=256, ny=256, nz=128, R=30.0, W=5.0, dTw=0.1, Ts_frac=0.86, theta=90.0,
            lam=1.0 / 3.0, seed=2206, amp=0.0):
    """Hemispherical droplet of radius R centred on a heated bottom wall.

    Periodic in x, y; bounce-back wall at z = 0 held at (Ts_frac + dTw) Tc with
    contact angle theta; constant-pressure top face (rho_b = rho_v) at T_s.
    """
    Ts, Tw = Ts_frac * Tc, (Ts_frac + dTw) * Tc
    x, y, z = grid(nx, ny, nz)
    cx, cy = nx / 2.0, ny / 2.0
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + z ** 2)
    rho0 = tanh_profile(r - R, rho_v, rho_l, W)
    if amp:
        rho0 = perturb(rho0, amp, seed)
    T0 = np.full_like(rho0, Ts)
    T0[0] = Tw
    p = base_params(nx, ny, nz, rho_l=rho_l, rho_v=rho_v, lambda_l=lam, lambda_v=lam,
                    face_kind=[PERIODIC, PERIODIC, PERIODIC, PERIODIC, WALL, OPEN],
                    face_T=[0, 0, 0, 0, Tw, Ts], face_rho=[0, 0, 0, 0, 0, rho_v],
                    face_theta_deg=[90, 90, 90, 90, theta, 90])
    return p, rho0, T0


def heated_surface(Tc, rho_v, rho_l, nx=160, ny=160, nz=100, D=70.0, W=5.0, theta=120.0, Tw_frac=0.8931,
                   Ts_frac=0.86, lam=1.0 / 3.0):
    """Droplet evaporating on a heated surface as in Sec. 4.3: a droplet of diameter D on
    the bounce-back bottom wall (contact angle theta, held at Tw_frac Tc), constant-pressure
    top face (rho_b = rho_v at T_s), periodic in x and y, everything initially at T_s.  The
    droplet is the sphere of diameter D whose cap meets the wall layer at the angle theta:
    its centre lies R cos(pi - theta) above the wall layer.  The paper's a = 3/49 (with
    which its h_lv = 0.5032 and T_w = 0.8931 T_c hold); Tc and the coexistence densities
    are those of the caller (they depend on a only through Tc)."""
    Ts, Tw = Ts_frac * Tc, Tw_frac * Tc
    R = 0.5 * D
    x, y, z = grid(nx, ny, nz)
    zc = R * np.cos(np.pi - np.radians(theta))
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 + (z - zc) ** 2)
    rho0 = tanh_profile(r - R, rho_v, rho_l, W)
    T0 = np.full_like(rho0, Ts)
    T0[0] = Tw
    p = base_params(nx, ny, nz, a=3.0 / 49.0, rho_l=rho_l, rho_v=rho_v, lambda_l=lam, lambda_v=lam,
                    face_kind=[PERIODIC, PERIODIC, PERIODIC, PERIODIC, WALL, OPEN],
                    face_T=[0, 0, 0, 0, Tw, Ts], face_rho=[0, 0, 0, 0, 0, rho_v],
                    face_theta_deg=[90, 90, 90, 90, theta, 90])
    return p, rho0, T0


def pool_droplets(n=512, ndrop=64, Rmin=10.0, Rmax=25.0, W=5.0, seed=2206, shape=None, max_tries=100000):
    """Centres and radii of ndrop droplets by seeded rejection sampling: R uniform in
    [Rmin, Rmax), each surface at least W from every face, centre distances above
    R1 + R2 + W.  Candidate k draws (R, cx, cy, cz) from uniform(seed, ., stream=11)
    at indices 4k .. 4k+3.  Returns an array of rows (cx, cy, cz, R)."""
    nx, ny, nz = (n, n, n) if shape is None else shape
    u = uniform(seed, 4 * max_tries, stream=11).reshape(max_tries, 4)
    out = []
    for k in range(max_tries):
        R = Rmin + (Rmax - Rmin) * u[k, 0]
        m = R + W
        c = [m + (L - 1 - 2 * m) * u[k, 1 + a] for a, L in enumerate((nx, ny, nz))]
        if any(L - 1 - 2 * m <= 0 for L in (nx, ny, nz)):
            continue
        if all(np.sqrt(sum((c[a] - d[a]) ** 2 for a in range(3))) > R + d[3] + W for d in out):
            out.append((c[0], c[1], c[2], R))
            if len(out) == ndrop:
                return np.array(out)
    raise ValueError(f"only {len(out)} of {ndrop} droplets fit")


def pool(Tc, rho_v, rho_l, n=512, ndrop=64, Rmin=10.0, Rmax=25.0, W=5.0, Tw_frac=0.96, Ts_frac=0.86,
         lam=1.0 / 3.0, seed=2206, shape=None):
    """Heated-plate pool: ndrop droplets (pool_droplets) in vapour at coexistence density.

    Periodic in x, y; bounce-back wall at z = 0 held at Tw_frac Tc; constant-pressure
    top face (rho_b = rho_v) at T_s.  Each droplet has the tanh profile of width W
    out to 3W beyond its surface (the larger value is taken where two such shells
    meet; the gaps of at least W keep the liquid apart).  T0 = T_s, the
    wall layer at T_w.  Fields are FP32, z-major (nz, ny, nx).  Beyond 3W of every
    surface the density is rho_v exactly.
    """
    nx, ny, nz = (n, n, n) if shape is None else shape
    Ts, Tw = Ts_frac * Tc, Tw_frac * Tc
    rho0 = np.full((nz, ny, nx), rho_v, dtype=np.float32)
    for cx, cy, cz, R in pool_droplets(n, ndrop, Rmin, Rmax, W, seed, shape):
        h = R + 3 * W
        lo = [max(0, int(np.floor(c - h))) for c in (cx, cy, cz)]
        hi = [min(L, int(np.ceil(c + h)) + 1) for c, L in zip((cx, cy, cz), (nx, ny, nz))]
        z, y, x = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]),
                              indexing="ij")
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        box = rho0[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        prof = np.where(r - R <= 3 * W, tanh_profile(r - R, rho_v, rho_l, W), rho_v).astype(np.float32)
        np.maximum(box, prof, out=box)
    T0 = np.full((nz, ny, nx), Ts, dtype=np.float32)
    T0[0] = Tw
    p = base_params(nx, ny, nz, rho_l=rho_l, rho_v=rho_v, lambda_l=lam, lambda_v=lam,
                    face_kind=[PERIODIC, PERIODIC, PERIODIC, PERIODIC, WALL, OPEN],
                    face_T=[0, 0, 0, 0, Tw, Ts], face_rho=[0, 0, 0, 0, 0, rho_v],
                    storage=1)
    return p, rho0, T0


def random_populations(nx, ny, nz, rho_base, T_base, w19, w7, amp, seed):
    """Populations w_i * base * (1 + uniform(-amp, amp)), seeded; rho_base/T_base scalars or fields."""
    N = nx * ny * nz
    def field(v):
        v = np.asarray(v, dtype=np.float64)
        if v.size == N:
            return v.reshape(-1)
        return np.broadcast_to(v, (nz, ny, nx)).reshape(-1)

    rb, tb = field(rho_base), field(T_base)
    rf = uniform(seed, 19 * N, stream=7).reshape(19, N)
    rg = uniform(seed, 7 * N, stream=8).reshape(7, N)
    f = np.asarray(w19)[:, None] * rb[None, :] * (1.0 + amp * (2.0 * rf - 1.0))
    g = np.asarray(w7)[:, None] * tb[None, :] * (1.0 + amp * (2.0 * rg - 1.0))
    return f, g


# D3Q19 / D3Q7 weights as printed with Eqs. 2 and 14 (constants, used only to
# scale random populations to realistic magnitudes).
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def w7(wbar):
    return np.array([1.0 - wbar] + [wbar / 6.0] * 6)
