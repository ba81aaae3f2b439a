"""Multi-patch containment (OR over the faces of one surface) and midpoint
filtering of intersection-curve pieces (Sec. 5.4.2) on the GPU, against the
oracle per face and against closed forms."""
import numpy as np
import pytest

import wn_synth as ws
from oracle import query

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2510_25159_gb300 as wn
    return wn


def half_disc(c, r, lower):
    """Closed CCW half disc: two exact rational quarter arcs and the diameter."""
    a0 = np.pi if lower else 0.0
    arcs = [ws.rational_arc(c, r, a0, np.pi / 2), ws.rational_arc(c, r, a0 + np.pi / 2, np.pi / 2)]
    end, start = arcs[-1][0][-1], arcs[0][0][0]
    line = (np.array([end, start]), np.ones(2))
    return ws.make_domain([arcs + [line]], eps=1e-9)


def oracle_or(doms, pts):
    if not doms:
        return np.zeros(len(pts), np.uint8)
    return np.logical_or.reduce([query(d, pts)[1] != 0 for d in doms]).astype(np.uint8)


@pytest.mark.parametrize("prec", [1, 0])
def test_two_half_discs_make_a_disc(wn, prec):
    import torch
    c, r = np.array([0.45, 0.55]), 0.3
    doms = [half_disc(c, r, False), half_disc(c, r, True)]
    faces = [wn.Domain.from_dict(d) for d in doms]
    rng = np.random.default_rng(2)
    pts = rng.uniform(0, 1, (20001, 2))
    d = np.hypot(*(pts - c).T)
    got = wn.query_surfaces([faces], torch.from_numpy(pts).cuda(), [0, len(pts)], precision=prec).cpu().numpy()
    assert np.array_equal(got, oracle_or(doms, pts))
    far = np.abs(d - r) > 1e-6
    assert np.array_equal(got[far], (d[far] < r).astype(np.uint8))
    for f in faces:
        f.close()


def test_surfaces_with_0_1_3_faces(wn):
    import torch
    rng = np.random.default_rng(3)
    d2, _ = ws.config2(n_domains=64, n_uniform=64 * 10, n_near=0, domain_subset=[20, 21, 22, 23])
    groups = [[], [d2[0]], [d2[1], d2[2], d2[3]]]
    counts = [257, 1000, 3001]
    pts = [rng.uniform(0, 1, (n, 2)) for n in counts]
    faces = [[wn.Domain.from_dict(d) for d in g] for g in groups]
    allp = np.concatenate(pts)
    off = np.concatenate([[0], np.cumsum(counts)])
    got = wn.query_surfaces(faces, torch.from_numpy(allp).cuda(), off).cpu().numpy()
    for g, p, a, b in zip(groups, pts, off[:-1], off[1:]):
        assert np.array_equal(got[a:b], oracle_or(g, p))
    for g in faces:
        for f in g:
            f.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_intersection_piece_midpoints(wn, prec):
    import torch
    doms, _ = ws.config3(n_faces=256, n_queries=2560, face_subset=[7])
    dom = doms[0]
    rng = np.random.default_rng(5)
    # pieces of random polylines across the torus domain
    a = rng.uniform(0, ws.TWO_PI, (5000, 2))
    b = a + rng.normal(0, 0.05, (5000, 2))
    pieces = np.ascontiguousarray(np.concatenate([a, b], axis=1))
    h = wn.Domain.from_dict(dom)
    got = wn.query_midpoints(h, torch.from_numpy(pieces).cuda(), precision=prec).cpu().numpy()
    mid = np.stack([0.5 * (pieces[:, 0] + pieces[:, 2]), 0.5 * (pieces[:, 1] + pieces[:, 3])], axis=1)
    _, st = query(dom, mid)
    assert np.array_equal(got, st)
    h.close()
