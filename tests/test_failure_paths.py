"""Failure and tuning paths of the mixed query, on the GPU, made on the host
side: queues capped from the host (a pair that does not fit sends its query
to the FP64 recomputation), the FP32 near walk at its extreme depth caps and
draw sizes, the escalated-query readback, and the gap angle of the sweep
against the library's atan2 (the chord angle of Eq. 3 in the crossing form)."""
import numpy as np
import pytest

import wn_synth as ws
from tests.gpu_util import TOL_MIXED, compare, run

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


def _batch():
    d2, q2 = ws.config2(n_domains=64, n_uniform=64 * 5000, n_near=64 * 1500, domain_subset=[1, 2])
    d3, q3 = ws.config3(n_faces=256, n_queries=256 * 2000, face_subset=[5, 6])
    return d2 + d3, q2 + q3


@pytest.mark.parametrize("near_cap,f64_cap", [(2000, 0), (0, 40), (300, 10)])
def test_queue_overflow_recomputes_in_fp64(wn, near_cap, f64_cap):
    """Pairs beyond a capped near or FP64 queue flag their queries for the
    FP64 recomputation: results still match the oracle, and the stats count
    the pairs that did not fit."""
    doms, qs = _batch()
    wn.set_queue_limits(near_cap, f64_cap)
    try:
        res = run(wn, doms, qs, 1)
        st = wn.stats()
    finally:
        wn.set_queue_limits(0, 0)
    assert st["overflow"] > 0
    assert st["fp64_queries"] > 0
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, TOL_MIXED)
    run(wn, doms[:1], qs[:1], 1)
    assert wn.stats()["overflow"] == 0


@pytest.mark.parametrize("depth,chunk,refill", [(12, 32, 1), (30, 1024, 32), (16, 64, 8)])
def test_near_tuning_extremes(wn, depth, chunk, refill):
    """The FP32 near walk's depth cap (Lemma 2 bounds the depth a pair
    needs) and its queue draws only move work between FP32 and FP64: results
    match the oracle at the extreme settings."""
    doms, qs = _batch()
    saved = wn.get_tuning()
    wn.set_near_tuning(depth, chunk, refill)
    try:
        assert wn.get_tuning()["near_depth"] == depth
        res = run(wn, doms, qs, 1)
        st = wn.stats()
    finally:
        wn.set_near_tuning(saved["near_depth"], saved["near_chunk"], saved["near_refill"])
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, TOL_MIXED)
    assert st["near_pairs"] > 0


def test_last_escalated_lists_fp64_queries(wn):
    """The queries within the classification band are recomputed in FP64 and
    listed by wn_last_escalated."""
    arcs = ws.circle_loop((0.5, 0.5), 0.3, n_arcs=16)[:8]
    dom = ws.make_domain([arcs], eps=1e-9)
    rng = np.random.default_rng(4)
    near_c = 0.5 + rng.uniform(-1e-6, 1e-6, (300, 2))
    far = rng.uniform(0.0, 0.2, (700, 2))
    q = np.concatenate([near_c, far])
    (w, s), = run(wn, [dom], [q], 1)
    compare(dom, q, w, s, TOL_MIXED)
    esc = np.sort(wn.last_escalated())
    assert len(esc) == wn.stats()["fp64_queries"]
    assert set(range(300)) <= set(esc.tolist())
    assert np.all(esc < len(q))


def test_gap_angle_against_atan2(wn):
    """The sweep's gap angle: odd series of atan(y/x) for |y| <= x/4 (error
    below |t|^13/13 plus FP32 rounding of a few ulp), atan2f elsewhere;
    compared with FP64 atan2 over the series' domain, its edge and the
    other quadrants."""
    import torch
    rng = np.random.default_rng(17)
    n = 400_000
    t = np.concatenate([rng.uniform(-0.25, 0.25, n), np.array([0.25, -0.25, 0.0, 1e-30, -1e-30]),
                        rng.uniform(-0.2500001, -0.2499999, 1000), rng.uniform(0.2499999, 0.2500001, 1000)])
    x = np.exp(rng.uniform(np.log(1e-12), np.log(1e3), t.size))
    y = (t * x).astype(np.float32)
    x = x.astype(np.float32)
    # every direction, for the atan2f branch
    ang = rng.uniform(-np.pi, np.pi, 100_000)
    r = np.exp(rng.uniform(np.log(1e-6), np.log(1e2), ang.size))
    y = np.concatenate([y, (r * np.sin(ang)).astype(np.float32)])
    x = np.concatenate([x, (r * np.cos(ang)).astype(np.float32)])
    got = wn.eval_gap_angle(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    series = np.abs(y.astype(np.float64)) <= 0.25 * x.astype(np.float64)
    assert series.sum() > n
    err = np.abs(got - ref)
    tt = np.abs(y.astype(np.float64) / x.astype(np.float64))
    # the series: truncation |t|^13/13 and a few FP32 ulps of the result
    bound_s = tt ** 13 / 13 + 6 * 2.0 ** -24 * np.abs(ref) + 1e-36
    assert np.all(err[series] <= bound_s[series]), float(np.max(err[series] / bound_s[series]))
    # atan2f: within a few ulps of the result (and of pi at the cut)
    bound_w = 4 * 2.0 ** -24 * np.maximum(np.abs(ref), 1e-30)
    assert np.all(err[~series] <= bound_w[~series]), float(np.max(err[~series] / bound_w[~series]))
