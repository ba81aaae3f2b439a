"""Queries on the edges of the copy windows of periodic domains (GPU against
the FP64 oracle).

Which lattice copies of a loop a query sees is decided by exact FP64 window
tests: the control-point box of a contractible copy (Alg. 4-5 reading), the
slab of an extended curve's copies along its lattice vector (Eq. 9).  For an
open loop the window is the definition of the result, so a query just inside
and one just outside a window edge get different sums.  The mixed path
decides windows first in FP32 (an outer window that rejects, an inner one
that accepts) and runs the exact test only between them; these queries sit
within 0 to 1e-5 of the edges, so every branch of that decision runs."""
import numpy as np
import pytest

import oracle
import wn_synth as ws
from tests.gpu_util import TOL_MIXED, TOL_PLAIN, compare, run

pytestmark = pytest.mark.gpu

OFFSETS = np.array([0.0, 1e-15, -1e-15, 1e-12, -1e-12, 1e-9, -1e-9, 1e-7, -1e-7, 1e-5, -1e-5])


@pytest.fixture(scope="module")
def wn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2510_25159_gb300 as wn
    return wn


def edge_queries(dom, rng, per_edge=6):
    """Points on the box edges of every contractible loop and on the slab
    edges of every extended loop, at the offsets above, in several lattice
    tiles (the library and the oracle reduce them to the base tile)."""
    Pu, Pv = dom["period_u"], dom["period_v"]
    per = np.array([Pu, Pv])
    lifted, hom, _, _ = oracle.domain_info(dom)
    lo = dom["loop_offsets"]
    start = np.concatenate([[0], np.cumsum(dom["degrees"] + 1)])
    out = []
    for l in range(len(lo) - 1):
        cps = lifted[start[lo[l]]:start[lo[l + 1]]]
        if hom[l, 0] == 0 and hom[l, 1] == 0:
            x0, y0 = cps.min(axis=0)
            x1, y1 = cps.max(axis=0)
            for e in range(4):
                t = rng.uniform(0, 1, per_edge)
                d = rng.choice(OFFSETS, per_edge)
                shift = per * rng.integers(-2, 3, (per_edge, 2))
                if e < 2:
                    x = (x0 if e == 0 else x1) + d
                    y = y0 + t * (y1 - y0)
                else:
                    x = x0 + t * (x1 - x0)
                    y = (y0 if e == 2 else y1) + d
                out.append(np.stack([x, y], axis=1) + shift)
        else:
            v = np.array([hom[l, 0] * Pu, hom[l, 1] * Pv], dtype=np.float64)
            vv = float(v @ v)
            s = np.concatenate([cps, cps[:1] + v]) @ v / vv
            nrm = np.array([-v[1], v[0]]) / np.sqrt(vv)
            for edge in (s.min(), s.max()):
                k = rng.integers(-2, 3, per_edge)
                d = rng.choice(OFFSETS, per_edge)
                a = rng.uniform(-max(Pu, Pv), max(Pu, Pv), per_edge)
                out.append(((edge + k + d / np.sqrt(vv))[:, None] * v[None, :]) + a[:, None] * nrm[None, :])
    return np.ascontiguousarray(np.concatenate(out, axis=0))


@pytest.mark.parametrize("name,prec,tol", [("mixed", 1, TOL_MIXED), ("plain", 0, TOL_PLAIN)])
def test_cylinder_window_edges(wn, name, prec, tol):
    """The same on uni-periodic (cylinder) faces: box windows along the
    periodic axis only, extended curves winding once around it."""
    rng = ws.rng_for(41)
    doms = []
    for f in range(5):
        lps = ws.uniperiodic_face(rng, 3 + f, (6, 40), P=1.0, degrees=(1, 5))
        doms.append(ws.make_domain(lps, 1.0, 0.0, eps=1e-9))
    qr = np.random.default_rng(32)
    qs = [edge_queries(d, qr) for d in doms]
    assert sum(len(q) for q in qs) > 300
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


@pytest.mark.parametrize("name,prec,tol", [("mixed", 1, TOL_MIXED), ("plain", 0, TOL_PLAIN)])
def test_periodic_window_edges(wn, name, prec, tol):
    doms, _ = ws.config3(n_faces=256, n_queries=256, face_subset=range(6))
    rng = np.random.default_rng(31)
    qs = [edge_queries(d, rng) for d in doms]
    assert sum(len(q) for q in qs) > 500
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)
