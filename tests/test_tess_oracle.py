"""Pins of the grid-triangle oracle (CPU): counts of full grids, the Euler
characteristic of the kept mesh against the topology of the region
(disc 1, annulus 0, cylinder 0, torus 0), orientation, vertices inside,
emission order."""
import numpy as np

from oracle.tess import grid_triangles


def euler(tris):
    """V - E + F of a triangle list (vertices: those used)."""
    if len(tris) == 0:
        return 0
    V = np.unique(tris).size
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    E = np.unique(e, axis=0).shape[0]
    return V - E + len(tris)


def centres(nu, nv):
    i, j = np.meshgrid(np.arange(nu), np.arange(nv))
    return (i.ravel() + 0.5) / nu, (j.ravel() + 0.5) / nv


def test_full_grids():
    for nu, nv in ((2, 2), (5, 3), (17, 11)):
        ins = np.ones(nu * nv, bool)
        t = grid_triangles(ins, nu, nv)
        assert len(t) == 2 * (nu - 1) * (nv - 1) and euler(t) == 1
        if nu < 3:
            continue                                                   # a wrap of 2 columns is degenerate
        t = grid_triangles(ins, nu, nv, wrap_u=True)
        assert len(t) == 2 * nu * (nv - 1) and euler(t) == 0          # cylinder
        if nv >= 3:
            t = grid_triangles(ins, nu, nv, wrap_u=True, wrap_v=True)
            assert len(t) == 2 * nu * nv and euler(t) == 0            # torus
    assert len(grid_triangles(np.zeros(30, bool), 6, 5)) == 0
    assert len(grid_triangles(np.ones(7, bool), 7, 1)) == 0            # one row: no quads


def test_region_topology():
    nu = nv = 64
    u, v = centres(nu, nv)
    r = np.hypot(u - 0.5, v - 0.5)
    disc = r < 0.4
    assert euler(grid_triangles(disc, nu, nv)) == 1
    annulus = disc & (r > 0.15)
    assert euler(grid_triangles(annulus, nu, nv)) == 0
    two_holes = disc & (np.hypot(u - 0.35, v - 0.5) > 0.08) & (np.hypot(u - 0.65, v - 0.5) > 0.08)
    assert euler(grid_triangles(two_holes, nu, nv)) == -1
    band = np.abs(v - 0.5) < 0.2                                        # a band around a cylinder
    assert euler(grid_triangles(band, nu, nv, wrap_u=True)) == 0


def test_orientation_inside_and_order():
    rng = np.random.default_rng(4)
    nu, nv = 23, 19
    ins = rng.random(nu * nv) < 0.7
    t = grid_triangles(ins, nu, nv)
    assert np.all(ins[t])
    x = (t % nu).astype(float)
    y = (t // nu).astype(float)
    area = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    assert np.all(area > 0)
    quad = (t[:, 0] // nu) * (nu - 1) + t[:, 0] % nu                   # lower-left vertex -> quad id
    assert np.all(np.diff(quad) >= 0)
    # every quad with four inside corners gives both triangles
    full = sum(ins[j * nu + i] and ins[j * nu + i + 1] and ins[(j + 1) * nu + i] and ins[(j + 1) * nu + i + 1]
               for j in range(nv - 1) for i in range(nu - 1))
    assert np.sum(np.bincount(quad) == 2) == full
