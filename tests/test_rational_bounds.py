"""The derivative bounds of rational segments that the walks of Algorithm 1
use (App. A.1; host code of the C library, no GPU): the whole segment's B
and the bounds on its eighths must bound |gamma'(t)|, which the test
computes independently by the quotient rule from the Bernstein derivatives
of the homogeneous curve, densely sampled on every eighth.  A bound below
a sampled speed would let a walk call a node far while the curve leaves
the node's ellipse, so a crossing could be lost."""
from math import comb

import numpy as np
import pytest

import wn_synth as ws


@pytest.fixture(scope="module")
def wn():
    import __graft_entry__ as g
    g.build()
    import paper_2510_25159_gb300 as wn
    return wn


def speeds(cps, w, t):
    """|gamma'(t)| of the rational Bezier curve (control points cps, weights
    w) at the parameters t: gamma = Q / W, gamma' = (Q' W - Q W') / W^2."""
    n = len(w) - 1
    cps = cps - cps[0]          # gamma' is translation-invariant; this keeps the quotient rule from cancelling
    H = np.concatenate([cps * w[:, None], w[:, None]], axis=1)          # (n+1, 3)
    B = np.stack([comb(n, k) * t ** k * (1 - t) ** (n - k) for k in range(n + 1)], axis=1)
    D = np.zeros_like(B)
    for k in range(n + 1):
        # d/dt of C(n,k) t^k (1-t)^(n-k) = n (B_{k-1}^{n-1} - B_k^{n-1})
        a = comb(n - 1, k - 1) * t ** (k - 1) * (1 - t) ** (n - k) if k >= 1 else 0.0
        b = comb(n - 1, k) * t ** k * (1 - t) ** (n - 1 - k) if k <= n - 1 else 0.0
        D[:, k] = n * (a - b)
    Hv, Hd = B @ H, D @ H
    Wv, Wd = Hv[:, 2:3], Hd[:, 2:3]
    g1 = (Hd[:, :2] * Wv - Hv[:, :2] * Wd) / Wv ** 2
    return np.hypot(g1[:, 0], g1[:, 1])


def check(wn, cps, w, samples=4001):
    out = wn.rational_bounds(cps, w)
    B, Bj = out[0], out[1:]
    assert np.all(Bj <= B) and np.all(Bj > 0)
    worst = 0.0
    for j in range(8):
        t = np.linspace(j / 8, (j + 1) / 8, samples)
        s = speeds(cps, w, t)
        assert s.max() <= Bj[j] * (1 + 1e-12), (j, s.max(), Bj[j])
        assert s.max() <= B * (1 + 1e-12)
        worst = max(worst, Bj[j] / max(s.max(), 1e-300))
    return B, Bj, worst


def test_random_rational_segments(wn):
    rng = np.random.default_rng(20251025)
    for trial in range(300):
        n = int(rng.integers(1, 8))
        cps = rng.uniform(-1.0, 1.0, (n + 1, 2)) * 10.0 ** rng.uniform(-3, 1)
        w = np.exp(rng.uniform(np.log(0.05), np.log(20.0), n + 1))
        check(wn, cps, w, samples=1001)


def test_equal_weights_is_polynomial(wn):
    """Equal weights give the polynomial curve, whose speed the hodograph
    bound n max |P_i - P_{i-1}| (Lemma 1) also bounds."""
    rng = np.random.default_rng(3)
    for n in range(1, 8):
        cps = rng.uniform(-1.0, 1.0, (n + 1, 2))
        B, Bj, _ = check(wn, cps, np.full(n + 1, 2.5))
        lemma1 = n * np.max(np.hypot(*np.diff(cps, axis=0).T))
        assert B <= lemma1 * (1 + 1e-12)


@pytest.mark.parametrize("theta", [0.1, 1.0, 2.0, 2.6, 3.0, 3.1])
def test_circular_arcs(wn, theta):
    """Exact arcs (weights 1, cos(theta/2), 1): the segment's bound grows
    like 1 / cos(theta/2) (the looseness that slows walks next to wide
    arcs), the eighths' bounds stay within a small factor of the speed."""
    cps, w = ws.rational_arc((0.5, 0.5), 0.3, 0.4, theta)
    B, Bj, worst = check(wn, cps, w)
    smax = speeds(cps, w, np.linspace(0.0, 1.0, 20001)).max()
    assert worst < 3.0
    if theta >= 3.0:
        assert B > 30.0 * smax
    assert Bj.max() < 3.0 * smax


def test_subdivision_rounding_far_from_origin(wn):
    """Control points far from the origin relative to the segment's size
    (the subdivision's rounding is then largest relative to the speeds)."""
    cps, w = ws.rational_arc((1000.0, -2000.0), 1e-3, 0.0, 2.5)
    check(wn, cps, w)
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = int(rng.integers(1, 8))
        cps = 5e3 + rng.uniform(-1e-3, 1e-3, (n + 1, 2))
        w = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n + 1))
        check(wn, cps, w, samples=1001)


def test_bad_arguments(wn):
    with pytest.raises(wn.WnError):
        wn.rational_bounds(np.zeros((1, 2)), np.ones(1))              # degree 0
    with pytest.raises(wn.WnError):
        wn.rational_bounds(np.zeros((9, 2)), np.ones(9))              # degree 8
    with pytest.raises(wn.WnError):
        wn.rational_bounds(np.zeros((3, 2)), np.array([1.0, -1.0, 1.0]))
    with pytest.raises(wn.WnError):
        wn.rational_bounds(np.array([[0.0, 0.0], [np.nan, 1.0]]), np.ones(2))
