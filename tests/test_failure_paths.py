"""Failure and tuning paths of the mixed query, on the GPU, made on the host
side: queues capped from the host (a pair that does not fit sends its query
to the FP64 recomputation), the FP32 near walk at its extreme depth caps and
draw sizes, the escalated-query readback, output buffers of any alignment
(the vectorised and the scalar finalize), and the gap angle of the sweep
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


def test_unaligned_outputs_same_results(wn):
    """Outputs 16-byte aligned take the four-query finalize, outputs one
    element off take the scalar one: the same windings (bit for bit) and
    states, escalated queries (next to a circle's centre) included, on a
    ragged batch."""
    import torch
    doms, qs = _batch()
    arcs = ws.circle_loop((0.5, 0.5), 0.3, n_arcs=16)[:8]
    doms = doms + [ws.make_domain([arcs], eps=1e-9)]
    rng = np.random.default_rng(5)
    qs = qs + [np.concatenate([0.5 + rng.uniform(-1e-6, 1e-6, (301, 2)), rng.uniform(0.0, 1.0, (2000, 2))])]
    handles = [wn.Domain.from_dict(d) for d in doms]
    pts = torch.from_numpy(np.ascontiguousarray(np.concatenate(qs))).cuda()
    off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
    n = int(off[-1])
    assert n % 4 != 0
    w_a = torch.empty(n, dtype=torch.float64, device="cuda")
    s_a = torch.empty(n, dtype=torch.uint8, device="cuda")
    wn.query_batched(handles, pts, off, out_winding=w_a, out_inside=s_a)
    torch.cuda.synchronize()
    assert wn.stats()["fp64_queries"] >= 301
    W = torch.full((n + 1,), 7.0, dtype=torch.float64, device="cuda")
    S = torch.full((n + 1,), 9, dtype=torch.uint8, device="cuda")
    w_u, s_u = W[1:], S[1:]
    assert w_u.data_ptr() % 16 == 8 and s_u.data_ptr() % 4 == 1
    wn.query_batched(handles, pts, off, out_winding=w_u, out_inside=s_u)
    torch.cuda.synchronize()
    for h in handles:
        h.close()
    assert torch.equal(w_a.view(torch.int64), w_u.view(torch.int64))
    assert torch.equal(s_a, s_u)
    assert W[0].item() == 7.0 and S[0].item() == 9
    wa, sa = w_a.cpu().numpy(), s_a.cpu().numpy()
    for d, q, a, b in zip(doms, qs, off[:-1], off[1:]):
        compare(d, q, wa[a:b], sa[a:b], TOL_MIXED)


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
