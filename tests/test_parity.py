"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Sizes span several sweep tiles (512 queries) and ragged tails.  States must
match exactly except oracle ties (decision margin < 1e-12 * domain scale);
omega within 1e-9 (plain FP64) / 1e-5 (mixed); closed-loop workloads must
also match rounded omega exactly."""
import numpy as np
import pytest

import wn_synth as ws
from tests.gpu_util import TOL_MIXED, TOL_PLAIN, compare, run

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


PRECS = [("mixed", 1, TOL_MIXED), ("plain", 0, TOL_PLAIN)]


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_workload1_closed(wn, name, prec, tol):
    dom, q = ws.config1()
    (w, s), = run(wn, [dom], [q], prec)
    r = compare(dom, q, w, s, tol, closed=True)
    assert r["boundary"] == 0


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_workload2_open_noisy(wn, name, prec, tol):
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 12000, n_near=64 * 1500,
                          domain_subset=range(6))
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


def test_workload2_full_size_sampled(wn):
    """The benchmark configuration (64 domains, 10M + 1M queries) in one
    mixed batched call; the oracle checks a stratified sample of every
    domain's uniform and near-curve queries."""
    doms, qs = ws.config2()
    res = run(wn, doms, qs, 1)
    rng = np.random.default_rng(7)
    for i, (d, q, (w, s)) in enumerate(zip(doms, qs, res)):
        n = len(q)
        nu = n - (1_000_000 // 64 + (1 if i < 1_000_000 % 64 else 0))
        idx = np.concatenate([rng.choice(nu, 150, replace=False), nu + rng.choice(n - nu, 100, replace=False),
                              [0, n - 1]])
        compare(d, q[idx], w[idx], s[idx], TOL_MIXED)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_workload3_biperiodic(wn, name, prec, tol):
    doms, qs = ws.config3(n_faces=256, n_queries=256 * 3000, face_subset=range(8))
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_rational_open_noisy(wn, name, prec, tol):
    """Rational segments (every weight log-uniform in [1/2, 2]) on open,
    noisy loops, plus exact circles of rational arcs."""
    doms, qs = ws.config6(n_domains=64, n_uniform=64 * 8000, n_near=64 * 1500, domain_subset=range(5))
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_rational_exact_circles_closed(wn, name, prec, tol):
    """Closed loops of exact rational arcs: rounded omega and states exact,
    also for points 1e-7..1e-3 from the circles and on a ragged query count."""
    rng = np.random.default_rng(8)
    outer = ws.rational_circle_loop((0.5, 0.5), 0.4, [1.0, 2.0, 1.5, 2 * np.pi - 4.5])
    holes = [ws.rational_circle_loop((0.35, 0.5), 0.08, [2.5, 2.5, 2 * np.pi - 5.0], ccw=False),
             ws.rational_circle_loop((0.65, 0.55), 0.1, [np.pi / 2] * 4, ccw=False)]
    dom = ws.make_domain([outer] + holes, eps=1e-9)
    r = np.concatenate([0.4 + rng.choice([-1, 1], 3000) * np.exp(rng.uniform(np.log(1e-7), np.log(1e-3), 3000)),
                        rng.uniform(0, 0.5, 2001)])
    ph = rng.uniform(0, 2 * np.pi, r.size)
    q = np.stack([0.5 + r * np.cos(ph), 0.5 + r * np.sin(ph)], axis=1)
    (w, s), = run(wn, [dom], [q], prec)
    compare(dom, q, w, s, tol, closed=True)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_rational_wide_arcs_near(wn, name, prec, tol):
    """Circles of wide rational arcs (up to 3 radians: middle weight down to
    cos(1.5) = 0.07, where App. A.1's segment bound is loosest and the walks
    also use the bounds of the segments' eighths): points 3e-9..1e-3 from
    the arcs (states and rounded omega exact) and points on them (boundary)."""
    rng = np.random.default_rng(11)
    centres = np.array([[0.5, 0.5], [0.45, 0.55]])
    radii = np.array([0.4, 0.15])
    outer = ws.rational_circle_loop(tuple(centres[0]), radii[0], [3.0, 3.0, 2 * np.pi - 6.0])
    hole = ws.rational_circle_loop(tuple(centres[1]), radii[1], [2.9, 2.2, 2 * np.pi - 5.1], ccw=False)
    dom = ws.make_domain([outer, hole], eps=1e-9)
    n, n_on = 4001, 300
    which = rng.integers(0, 2, n + n_on)
    off = rng.choice([-1, 1], n) * np.exp(rng.uniform(np.log(3e-9), np.log(1e-3), n))
    r = radii[which] + np.concatenate([off, np.zeros(n_on)])
    ph = rng.uniform(0, 2 * np.pi, n + n_on)
    q = centres[which] + r[:, None] * np.stack([np.cos(ph), np.sin(ph)], axis=1)
    (w, s), = run(wn, [dom], [q], prec)
    compare(dom, q, w, s, tol, closed=True)
    assert np.all(s[n:] == 2)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_uniperiodic_cylinders(wn, name, prec, tol):
    rng = ws.rng_for(40)
    doms, qs = [], []
    for f in range(5):
        lps = ws.uniperiodic_face(rng, 3 + f, (6, 40), P=1.0, degrees=(1, 5))
        doms.append(ws.make_domain(lps, 1.0, 0.0, eps=1e-9))
        q = np.stack([rng.uniform(-2, 3, 2500), rng.uniform(-0.1, 1.1, 2500)], axis=1)
        qs.append(q)
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_uniperiodic_v_cylinders(wn, name, prec, tol):
    """Faces periodic in v only (the cylinder case of Sec. 4.3 along the
    other axis): workload-4-style cylinder faces with u and v exchanged,
    separation loops along v, contractible stars across the v seam, queries
    outside the base tile on both axes."""
    rng = ws.rng_for(41)
    doms, qs = [], []
    for f in range(4):
        lps = ws.uniperiodic_face(rng, 3 + f, (6, 40), P=1.0, degrees=(1, 5))
        lps = [ws._wrap_segments(lp, 0.0, 1.0) for lp in ws.swap_axes_loops(lps)]
        doms.append(ws.make_domain(lps, 0.0, 1.0, eps=1e-9))
        q = np.stack([rng.uniform(-0.1, 1.1, 2300 + 37 * f), rng.uniform(-2, 3, 2300 + 37 * f)], axis=1)
        qs.append(q)
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_workload4_batched_mixed_kinds(wn, name, prec, tol):
    S, Q, kind = ws.config4_sizes()
    pick = list(np.nonzero(kind < 0.1)[0][:6]) + list(np.nonzero((kind >= 0.1) & (kind < 0.2))[0][:6]) + \
        list(np.nonzero(kind >= 0.2)[0][:20])
    doms, qs = ws.config4(face_subset=pick, query_scale=0.05)
    res = run(wn, doms, qs, prec)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, tol)


@pytest.mark.parametrize("nu,nv,tile", [(200, 137, 8), (203, 61, 8), (1, 9, 8), (8, 8, 8), (203, 61, 64),
                                         (131, 70, 16), (65, 3, 32)])
def test_grid_bitmask(wn, nu, nv, tile):
    """Cell-centre grids (ragged against the tiles of the tree sweep, of
    every width), mixed and plain, bit for bit against the oracle."""
    import torch
    dom = ws.config5_face(0, levels=8, n_holes=25, hole_segs=24)
    pts = ws.grid_points(nu, nv)
    from oracle import query
    ow, osd = query(dom, pts)
    saved = wn.get_tuning()["grid_tile_w"]
    wn.set_grid_tile(tile)
    for prec in (1, 0):
        h = wn.Domain.from_dict(dom)
        bits, nb = wn.query_grid_bitmask(h, nu, nv, precision=prec)
        torch.cuda.synchronize()
        b = bits.cpu().numpy().view(np.uint32)
        k = np.arange(nu * nv)
        got = (b[k >> 5] >> (k & 31).astype(np.uint32)) & 1
        assert np.array_equal(got, (osd != 0).astype(np.uint32))
        assert int(nb.item()) == int((osd == 2).sum())
        h.close()
    wn.set_grid_tile(saved)


def test_workload5_full_face_sampled(wn):
    """Faces of the tessellation workload at full size (~100k cubics,
    4096 x 4096 cells): the bitmask against the oracle on stratified cells,
    on every cell the GPU recomputed in FP64, on cells next to a change of
    state (the cells nearest the curves) and on cells around control
    points; the boundary count is consistent."""
    import torch
    from oracle import query
    G = 4096
    rng = np.random.default_rng(11)
    for face in (3, 17):
        dom = ws.config5_face(face)
        h = wn.Domain.from_dict(dom)
        bits, nb = wn.query_grid_bitmask(h, G, G, precision=1)
        torch.cuda.synchronize()
        esc = wn.last_escalated()
        b = bits.cpu().numpy().view(np.uint32)
        h.close()
        k = np.arange(G * G, dtype=np.int64)
        v = ((b[k >> 5] >> (k & 31).astype(np.uint32)) & 1).reshape(G, G)
        edge = np.zeros_like(v, dtype=bool)
        edge[:, :-1] |= v[:, 1:] != v[:, :-1]
        edge[:-1, :] |= v[1:, :] != v[:-1, :]
        cand = np.flatnonzero(edge)
        rows = (np.arange(512) * G) // 512 + rng.integers(0, G // 512, 512)
        strat = rows * G + rng.integers(0, G, 512)
        cp = dom["cps"][rng.choice(len(dom["cps"]), 200, replace=False)]
        ij = np.clip(np.floor(cp * G).astype(np.int64) + rng.integers(-2, 3, cp.shape), 0, G - 1)
        cells = np.unique(np.concatenate([strat, ij[:, 1] * G + ij[:, 0], esc[:2000],
                                          rng.choice(cand, min(len(cand), 600), replace=False)]))
        pts = np.stack([((cells % G) + 0.5) / G, ((cells // G) + 0.5) / G], axis=1)
        ow, osd, om = query(dom, pts, margins=True)
        got = (b[cells >> 5] >> (cells & 31).astype(np.uint32)) & 1
        bad = (got != (osd != 0).astype(np.uint32)) & (om >= 1e-12)
        assert not bad.any(), (face, int(bad.sum()))
        assert 0 <= int(nb.item()) < G * G


def test_edge_cases(wn):
    import torch
    # empty query set, single query, ragged tile tails
    dom, q = ws.config1(n_uniform=1500, n_near=1)
    h = wn.Domain.from_dict(dom)
    for n in (0, 1, 511, 512, 513, 1501):
        pts = torch.from_numpy(q[:n].copy()).cuda()
        w, s = wn.query(h, pts, precision=1)
        torch.cuda.synchronize()
        if n:
            compare(dom, q[:n], w.cpu().numpy(), s.cpu().numpy(), TOL_MIXED)
    # points exactly on control points are BOUNDARY, far-away points escalate
    seg_ends = dom["cps"][::4][:40]
    far = np.array([[50.0, -30.0], [1e6, 1e6], [-3.0, 0.5]])
    pts = np.concatenate([seg_ends, far])
    for prec in (1, 0):
        w, s = wn.query(h, torch.from_numpy(pts).cuda(), precision=prec)
        torch.cuda.synchronize()
        s = s.cpu().numpy()
        assert np.all(s[:40] == 2)
        compare(dom, pts, w.cpu().numpy(), s, TOL_MIXED)
    h.close()
    # domain without loops: everything outside
    empty = ws.make_domain([], eps=1e-9)
    empty["cps"] = np.zeros((0, 2))
    he = wn.Domain.from_dict(empty)
    w, s = wn.query(he, torch.rand(700, 2, dtype=torch.float64, device="cuda"), precision=1)
    assert torch.all(s == 0) and torch.all(w == 0)
    he.close()


def test_max_degree_and_periodic_outside_tile(wn):
    rng = np.random.default_rng(3)
    loop = ws.star_loop(rng, (0.5, 0.5), 0.3, 30, 7, ccw=True, bend=0.2)
    dom = ws.make_domain([loop], eps=1e-9)
    q = rng.uniform(0, 1, (3000, 2))
    (w, s), = run(wn, [dom], [q], 1)
    compare(dom, q, w, s, TOL_MIXED, closed=True)
    doms, qs = ws.config3(n_faces=256, n_queries=256 * 2000, face_subset=[9, 10])
    qs = [q + rng.integers(-3, 4, q.shape) * ws.TWO_PI for q in qs]
    res = run(wn, doms, qs, 1)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, TOL_MIXED)


def test_host_buffers_match_device(wn):
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 3000, n_near=64 * 300, domain_subset=range(3))
    a = run(wn, doms, qs, 1, host=False)
    b = run(wn, doms, qs, 1, host=True)
    for (w1, s1), (w2, s2) in zip(a, b):
        # every query's arithmetic is its own (series lengths per query), so
        # staging and grouping change nothing, bit for bit
        assert np.array_equal(s1, s2)
        assert np.array_equal(w1, w2, equal_nan=True)


def test_host_buffers_grouped_match_device(wn):
    """A large mixed batch of host buffers (here 6M queries: two groups) runs
    as groups of domains whose copies overlap the other groups' kernels; it
    must give the results of the same batch from device buffers."""
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 1_100_000, n_near=64 * 100_000, domain_subset=range(5))
    assert sum(len(q) for q in qs) >= 6_000_000
    a = run(wn, doms, qs, 1, host=False)
    b = run(wn, doms, qs, 1, host=True)
    for (w1, s1), (w2, s2) in zip(a, b):
        # the groups' warps hold other queries than the single batch's; each
        # query's series lengths are its own, so the results are identical
        assert np.array_equal(s1, s2)
        assert np.array_equal(w1, w2, equal_nan=True)
    st = wn.stats()
    assert st["queries"] == sum(len(q) for q in qs)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_half_band_escalation(wn, name, prec, tol):
    """An open semicircle: its centre sees omega = 1/2 exactly, so queries
    within 1e-5 of it fall in the mixed path's classification band and are
    recomputed in FP64; their states hang on the sign of omega - 1/2 at the
    1e-7 level and must match the oracle's."""
    arcs = ws.circle_loop((0.5, 0.5), 0.3, n_arcs=16)[:8]
    dom = ws.make_domain([arcs], eps=1e-9)
    rng = np.random.default_rng(12)
    r = np.exp(rng.uniform(np.log(1e-9), np.log(1e-5), 1500))
    ph = rng.uniform(0, 2 * np.pi, r.size)
    q = np.stack([0.5 + r * np.cos(ph), 0.5 + r * np.sin(ph)], axis=1)
    (w, s), = run(wn, [dom], [q], prec)
    res = compare(dom, q, w, s, tol)
    assert res["n"] == 1500
    if prec == 1:
        assert wn.stats()["fp64_queries"] >= 1000


def test_stats_and_profiling(wn):
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 2000, n_near=64 * 500, domain_subset=range(2))
    wn.set_profiling(True)
    run(wn, doms, qs, 1)
    t, n = wn.kernel_times()
    wn.set_profiling(False)
    st = wn.stats()
    assert n == 1 and t["sweep"] > 0 and t["bucket"] >= 0
    assert st["queries"] == sum(len(q) for q in qs)
    assert st["overflow"] == 0 and st["depth_cap"] == 0


def test_work_counting_build(wn):
    """The counting build of the tree sweep decides and computes as the plain
    build (identical results) and its tallies are consistent: every
    telescoped node and expansion sum follows a node test, and records are
    tested."""
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 4000, n_near=64 * 500, domain_subset=[3, 4])
    a = run(wn, doms, qs, 1)
    wn.set_work_counting(True)
    try:
        b = run(wn, doms, qs, 1)
        work = wn.sweep_work()
    finally:
        wn.set_work_counting(False)
    for (w1, s1), (w2, s2) in zip(a, b):
        assert np.array_equal(s1, s2)
        assert np.array_equal(w1, w2, equal_nan=True)
    n_q = sum(len(q) for q in qs)
    assert work["node_tests"] >= n_q
    assert work["telescoped_nodes"] + work["expansions"] <= 2 * work["node_tests"]
    assert 4 * work["expansions"] <= work["expansion_terms"] <= 32 * work["expansions"]
    assert work["record_tests_near"] > 0 and work["telescoped_nodes"] > 0
    assert 0 < work["ellipse_tests"] <= work["record_tests_near"]
    assert 0 < work["box_tests"] <= work["ellipse_tests"]
    assert wn.sweep_work()["node_tests"] == 0      # read clears


@pytest.mark.parametrize("tree,bucket", [(0, 0), (1, 0), (1, 1)])
def test_sweep_modes(wn, tree, bucket):
    """Flat sweep, cluster sweep without and with spatial bucketing: all
    against the oracle on open planar, bi-periodic and mixed batched faces."""
    wn.set_tuning(tree=tree, bucket=bucket)
    try:
        d2, q2 = ws.config2(n_domains=64, n_uniform=64 * 9000, n_near=64 * 1500, domain_subset=[7, 8, 9])
        d3, q3 = ws.config3(n_faces=256, n_queries=256 * 3000, face_subset=[20, 21, 22, 23])
        S, Q, kind = ws.config4_sizes()
        pick = list(np.nonzero(kind < 0.1)[0][6:9]) + list(np.nonzero(kind >= 0.2)[0][20:30])
        d4, q4 = ws.config4(face_subset=pick, query_scale=0.05)
        doms, qs = d2 + d3 + d4, q2 + q3 + q4
        res = run(wn, doms, qs, 1)
        for d, q, (w, s) in zip(doms, qs, res):
            compare(d, q, w, s, TOL_MIXED)
    finally:
        wn.set_tuning(tree=1, bucket=1)


def test_graph_replay_and_autotune(wn):
    """Autotuning keeps results within tolerance; a captured graph replays the
    same launches on new contents of the same buffers."""
    import torch
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 6000, n_near=64 * 600, domain_subset=[11, 12, 13])
    handles = [wn.Domain.from_dict(d) for d in doms]
    pts_h = np.concatenate(qs)
    off = np.concatenate([[0], np.cumsum([len(q) for q in qs])]).astype(np.int64)
    stream = torch.cuda.Stream()
    saved = wn.get_tuning()
    try:
        with torch.cuda.stream(stream):
            pts = torch.from_numpy(pts_h).cuda()
            ms, tun = wn.autotune(handles, pts, off, iterations=1)
            assert ms > 0 and tun["qpt"] in (1, 2)
            wn.set_tuning(use_graph=1)
            w = torch.empty(len(pts_h), dtype=torch.float64, device="cuda")
            s = torch.empty(len(pts_h), dtype=torch.uint8, device="cuda")
            rng = np.random.default_rng(5)
            for rep in range(3):
                new = pts_h if rep == 0 else np.concatenate(
                    [rng.uniform(0, 1, (len(q), 2)) for q in qs])
                pts.copy_(torch.from_numpy(new))
                wn.query_batched(handles, pts, off, out_winding=w, out_inside=s)
                stream.synchronize()
                wh, sh = w.cpu().numpy(), s.cpu().numpy()
                for d, a, b in zip(doms, off[:-1], off[1:]):
                    compare(d, new[a:b], wh[a:b], sh[a:b], TOL_MIXED)
    finally:
        wn.set_tuning(qpt=saved["qpt"], sweep_ctas_per_sm=saved["sweep_ctas_per_sm"],
                      near_ctas_per_sm=saved["near_ctas_per_sm"], use_graph=0)
        for h in handles:
            h.close()


@pytest.mark.parametrize("flat", [0, 32, 4096])
def test_flat_sweep_for_small_planar_faces(wn, flat):
    """Planar faces up to the record limit take the flat sweep beside the
    tree sweep of the others (one batch, two kernels): every face against
    the oracle, for no flat face, the small ones, and every planar face."""
    S, Q, kind = ws.config4_sizes()
    pick = list(np.nonzero((kind >= 0.2) & (S <= 32))[0][:8]) + list(np.nonzero((kind >= 0.2) & (S > 200))[0][:4]) + \
        list(np.nonzero(kind < 0.2)[0][:4])
    doms, qs = ws.config4(face_subset=pick, query_scale=0.04)
    saved = wn.get_tuning()["flat_max"]
    wn.set_flat_records(flat)
    try:
        res = run(wn, doms, qs, 1)
    finally:
        wn.set_flat_records(saved)
    for d, q, (w, s) in zip(doms, qs, res):
        compare(d, q, w, s, TOL_MIXED, closed=True)


@pytest.mark.parametrize("name,prec,tol", PRECS)
def test_sphere_cone_punctured(wn, name, prec, tol):
    """Sphere and cone faces with their singular points punctured (Sec. 4.3):
    cylinders in the parameter domain, each removed point passed as the
    degenerate boundary loop B-Rep models store; queries sampled on the
    surfaces, against the oracle and the faces' closed forms."""
    rng = np.random.default_rng(30)
    loops, hc, hr = ws.sphere_cap_face(rng)
    sphere = ws.make_domain(loops, ws.TWO_PI, 0.0, eps=1e-9)
    cone = ws.make_domain(ws.cone_face(), ws.TWO_PI, 0.0, eps=1e-9)
    ps = ws.sphere_points(rng, 20011)
    pc = np.stack([rng.uniform(0, ws.TWO_PI, 15013), np.sqrt(rng.uniform(1e-6, 1, 15013))], axis=1)
    res = run(wn, [sphere, cone], [ps, pc], prec)
    for d, q, (w, s) in zip([sphere, cone], [ps, pc], res):
        compare(d, q, w, s, tol, closed=True)
    (ws_, ss), (wc, sc) = res
    curve = 0.35 + 0.15 * np.sin(3 * ps[:, 0])
    du = np.mod(ps[:, 0] - hc[0] + np.pi, ws.TWO_PI) - np.pi
    dh = np.hypot(du, ps[:, 1] - hc[1])
    far = (np.abs(ps[:, 1] - curve) > 1e-3) & (np.abs(dh - hr) > 1e-3) & (ps[:, 1] < 0.5 * np.pi - 1e-3)
    assert np.array_equal(ss[far], ((ps[far, 1] > curve[far]) & (dh[far] > hr)).astype(np.uint8))
    t0 = 0.3 + 0.05 * np.sin(2 * pc[:, 0])
    far = (np.abs(pc[:, 1] - t0) > 1e-3) & (np.abs(pc[:, 1] - 0.8) > 1e-3) & (np.abs(pc[:, 1] - 1.0) > 1e-3) & \
        (pc[:, 1] > 1e-3)
    exp = (pc[far, 1] < t0[far]) | ((pc[far, 1] > 0.8) & (pc[far, 1] < 1.0))
    assert np.array_equal(sc[far], exp.astype(np.uint8))


def _sampled_full_size(wn, doms, qs, per_dom, big_extra, seed):
    """One mixed batched call over a whole workload; the oracle checks
    per_dom stratified queries of every domain and big_extra more of every
    large domain (1000+ segments or 2^18+ queries)."""
    res = run(wn, doms, qs, 1)
    rng = np.random.default_rng(seed)
    for d, q, (w, s) in zip(doms, qs, res):
        big = ws.n_segments(d) >= 1000 or len(q) >= (1 << 18)
        m = min(len(q), per_dom + (big_extra if big else 0))
        idx = np.sort(rng.choice(len(q), m, replace=False))
        compare(d, q[idx], w[idx], s[idx], TOL_MIXED, threads=1)


def test_workload3_full_size_sampled(wn):
    """All 256 tori with their 20M queries in one call; every face checked."""
    doms, qs = ws.config3()
    _sampled_full_size(wn, doms, qs, 40, 200, 31)


def test_workload4_full_size_sampled(wn):
    """The batched B-Rep workload at full size (10k faces, 2e8 queries) in
    one call; every face checked, the large ones (up to 4000 segments or 1M
    queries) more."""
    doms, qs = ws.config4()
    _sampled_full_size(wn, doms, qs, 6, 150, 32)
