"""Seeded synthetic inputs: the placement rules and fields of the heated-plate pool
(512^3, 64 droplets with radii in [10, 25), FP16-shifted storage)."""
import numpy as np

from paper_2206_00946_gb300 import workloads as W


def test_pool_droplets_follow_the_placement_rules():
    d = W.pool_droplets()
    assert d.shape == (64, 4)
    c, R = d[:, :3], d[:, 3]
    assert np.all((R >= 10) & (R < 25))
    # every surface at least W = 5 from every face
    assert np.all(c - R[:, None] >= 5) and np.all(c + R[:, None] <= 511 - 5)
    # gaps between surfaces above W
    dist = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    gap = dist - R[:, None] - R[None, :]
    np.fill_diagonal(gap, np.inf)
    assert gap.min() > 5
    assert np.array_equal(d, W.pool_droplets())
    assert not np.array_equal(d, W.pool_droplets(seed=7))


def test_pool_fields():
    Tc, rv, rl = 0.07, 0.02, 0.3  # the generator takes the thermodynamics as given
    shape = (96, 80, 64)
    kw = dict(ndrop=6, Rmin=5.0, Rmax=9.0, shape=shape)
    p, rho, T = W.pool(Tc, rv, rl, **kw)
    d = W.pool_droplets(**kw)
    nx, ny, nz = shape
    assert rho.shape == (nz, ny, nx) and rho.dtype == np.float32 and T.dtype == np.float32
    assert rho.min() >= np.float32(rv) and rho.max() <= np.float32(rl)
    x, y, z = W.grid(nx, ny, nz)
    r = np.stack([np.sqrt((x - a) ** 2 + (y - b) ** 2 + (z - e) ** 2) - R for a, b, e, R in d])
    near = r.argmin(0)
    rmin = np.take_along_axis(r, near[None], 0)[0]
    # within 3W of the nearest surface: that droplet's tanh profile; beyond: vapour
    inside = rmin <= 15.0
    expect = W.tanh_profile(rmin, rv, rl, 5.0).astype(np.float32)
    assert np.array_equal(rho[inside], expect[inside])
    assert np.all(rho[~inside] == np.float32(rv))
    assert np.all(T[0] == np.float32(0.96 * Tc)) and np.all(T[1:] == np.float32(0.86 * Tc))
    assert p["face_kind"] == [W.PERIODIC] * 4 + [W.WALL, W.OPEN]
    assert p["face_T"][4] == 0.96 * Tc and p["face_rho"][5] == rv and p["storage"] == 1
