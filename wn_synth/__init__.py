"""Seeded synthetic inputs for the trimmed-surface containment workloads.

This module is shared by the oracle tests, the CUDA-path tests and ``bench.py``.
It only *places geometry*: it draws trimming loops made of Bezier segments and
query points.  It contains none of the winding-number arithmetic (no bounds, no
chord angles, no recursion, no lifting); the one curve evaluation it does (the
Bernstein sum in :func:`bezier_point`) is used only to put query points next to
a curve.

A domain is a plain dict::

    {"loop_offsets": int32[n_loops+1],   # CSR of loops into segments
     "degrees":      int32[n_segs],      # 1..7
     "cps":          float64[sum(deg+1), 2],  # control points, segment-major
     "period_u": float, "period_v": float,    # 0 = not periodic on that axis
     "eps": float}                             # boundary tolerance

Workload shapes follow the synthetic stand-ins for the paper's datasets:
closed C0 cubic loops (BG dataset A style, Sec. 5.1.1), Gaussian control-point
noise and open joins (the robustness study of Sec. 5.1.2), periodic loops with
non-contractible pairs (the periodic datasets of Sec. 5.2) and dense uv grids
(the tessellation application of Sec. 5.4.3).  Seeds are ``20251025 + index``.
"""
from __future__ import annotations

import math
from math import comb

import numpy as np

SEED_BASE = 20251025
TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# small helpers
# --------------------------------------------------------------------------
def rng_for(index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index + 1000003 * salt))


def bezier_point(cps: np.ndarray, t):
    """Point and derivative of a Bezier segment (Bernstein sum), for placing
    query points only.  ``cps`` is (n+1, 2); ``t`` scalar or array."""
    t = np.asarray(t, dtype=np.float64)
    n = cps.shape[0] - 1
    pt = np.zeros(t.shape + (2,))
    dv = np.zeros(t.shape + (2,))
    for k in range(n + 1):
        bk = comb(n, k) * t ** k * (1 - t) ** (n - k)
        pt += bk[..., None] * cps[k]
    for k in range(n):
        bk = comb(n - 1, k) * t ** k * (1 - t) ** (n - 1 - k)
        dv += (n * bk)[..., None] * (cps[k + 1] - cps[k])
    return pt, dv


def make_domain(loops, period_u=0.0, period_v=0.0, eps=1e-9):
    """Pack a list of loops (each a list of (n+1,2) control-point arrays).
    A segment may also be a pair (control points, weights) of a rational
    segment; a domain with any rational segment carries "weights", one per
    control point (1 for the polynomial segments)."""
    degs, cps, wts, offs = [], [], [], [0]
    rational = False
    for loop in loops:
        for seg in loop:
            if isinstance(seg, tuple):
                seg, w = np.asarray(seg[0], dtype=np.float64), np.asarray(seg[1], dtype=np.float64)
                rational = True
            else:
                seg = np.asarray(seg, dtype=np.float64)
                w = np.ones(seg.shape[0])
            degs.append(seg.shape[0] - 1)
            cps.append(seg)
            wts.append(w)
        offs.append(offs[-1] + len(loop))
    dom = {
        "loop_offsets": np.asarray(offs, dtype=np.int32),
        "degrees": np.asarray(degs, dtype=np.int32),
        "cps": np.ascontiguousarray(np.concatenate(cps, axis=0)) if cps else np.zeros((0, 2)),
        "period_u": float(period_u),
        "period_v": float(period_v),
        "eps": float(eps),
    }
    if rational:
        dom["weights"] = np.ascontiguousarray(np.concatenate(wts))
    return dom


def domain_weights(dom):
    """Per-segment weight arrays (None for a polynomial domain)."""
    if "weights" not in dom:
        return None
    out, off = [], 0
    for d in dom["degrees"]:
        out.append(dom["weights"][off:off + d + 1])
        off += d + 1
    return out


def rational_arc(center, radius, a0, theta):
    """Exact circular arc of angle theta (|theta| < pi) from angle a0, as a
    rational quadratic: middle point on the tangents' intersection, weight
    cos(theta/2)."""
    c = np.asarray(center, dtype=np.float64)
    h = abs(theta) / 2.0
    p0 = c + radius * np.array([math.cos(a0), math.sin(a0)])
    p2 = c + radius * np.array([math.cos(a0 + theta), math.sin(a0 + theta)])
    am = a0 + theta / 2.0
    p1 = c + radius / math.cos(h) * np.array([math.cos(am), math.sin(am)])
    return np.array([p0, p1, p2]), np.array([1.0, math.cos(h), 1.0])


def rational_circle_loop(center, radius, angles, ccw=True):
    """Closed loop of exact rational arcs whose angles (radians, each below
    pi) sum to 2 pi; CW when ccw is False."""
    a = 0.0
    sgn = 1.0 if ccw else -1.0
    segs = []
    for th in angles:
        cps, w = rational_arc(center, radius, sgn * a, sgn * th)
        segs.append((cps, w))
        a += th
    # close exactly: the last end is the first start
    last = segs[-1][0].copy()
    last[-1] = segs[0][0][0]
    segs[-1] = (last, segs[-1][1])
    return segs


def domain_segments(dom):
    """List of (n+1,2) arrays, one per segment (views into dom['cps'])."""
    out, off = [], 0
    for d in dom["degrees"]:
        out.append(dom["cps"][off:off + d + 1])
        off += d + 1
    return out


def domain_loops(dom):
    segs = domain_segments(dom)
    lo = dom["loop_offsets"]
    return [segs[lo[i]:lo[i + 1]] for i in range(len(lo) - 1)]


def n_segments(dom):
    return int(dom["degrees"].shape[0])


# --------------------------------------------------------------------------
# loop builders
# --------------------------------------------------------------------------
def _elevate_line(p0, p1, n, rng, bend):
    """Degree-n segment from p0 to p1 with interior points on the chord at
    i/n, each pushed along the chord normal by U(-bend, bend) * |chord|."""
    d = p1 - p0
    L = math.hypot(d[0], d[1])
    nrm = np.array([-d[1], d[0]]) / (L if L > 0 else 1.0)
    pts = [p0]
    for i in range(1, n):
        q = p0 + d * (i / n) + nrm * rng.uniform(-bend, bend) * L
        pts.append(q)
    pts.append(p1)
    return np.array(pts)


def circle_loop(center, radius, n_arcs=16, ccw=True):
    """Closed C1 loop of cubic arcs approximating a circle; handle length
    (4/3) tan(theta/4) for an arc of angle theta."""
    c = np.asarray(center, dtype=np.float64)
    th = TWO_PI / n_arcs
    h = 4.0 / 3.0 * math.tan(th / 4.0) * radius
    sgn = 1.0 if ccw else -1.0
    angs = [sgn * th * k for k in range(n_arcs + 1)]
    verts = [c + radius * np.array([math.cos(a), math.sin(a)]) for a in angs]
    verts[-1] = verts[0].copy()
    segs = []
    for k in range(n_arcs):
        a0, a1 = angs[k], angs[k + 1]
        t0 = sgn * np.array([-math.sin(a0), math.cos(a0)])
        t1 = sgn * np.array([-math.sin(a1), math.cos(a1)])
        p0, p3 = verts[k], verts[k + 1]
        segs.append(np.array([p0, p0 + h * t0, p3 - h * t1, p3]))
    return segs


def star_loop(rng, center, radius, n_seg, degrees, noise=0.0, ccw=True,
              bend=0.01, gap_lo=0.0, gap_hi=0.0, radial_noise=0.125):
    """Star-shaped loop: vertices at equal angles with radius r(1+U(-a,a)).
    ``degrees`` is an int or an array of per-segment degrees.  With
    gap_hi > 0 every join (the closing one included) is opened by a gap of
    log-uniform length in [gap_lo, gap_hi] in a random direction.  ``noise``
    adds N(0, noise^2) to every control point coordinate."""
    c = np.asarray(center, dtype=np.float64)
    ang = TWO_PI * np.arange(n_seg) / n_seg
    if not ccw:
        ang = -ang
    rad = radius * (1.0 + rng.uniform(-radial_noise, radial_noise, n_seg))
    verts = c + np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    if np.isscalar(degrees):
        degrees = np.full(n_seg, int(degrees))
    starts = verts.copy()
    if gap_hi > 0:
        g = np.exp(rng.uniform(math.log(gap_lo), math.log(gap_hi), n_seg))
        phi = rng.uniform(0, TWO_PI, n_seg)
        starts = verts + np.stack([g * np.cos(phi), g * np.sin(phi)], axis=1)
    segs = []
    for k in range(n_seg):
        p0 = starts[k]
        p1 = verts[(k + 1) % n_seg]
        segs.append(_elevate_line(p0, p1, int(degrees[k]), rng, bend))
    if noise > 0:
        segs = [s + rng.normal(0.0, noise, s.shape) for s in segs]
    return segs


def _near_points(rng, dom, count, off_lo, off_hi=None):
    """``count`` points at gamma(t) + s * off * nhat(t) for random segments,
    t ~ U(0,1), s = +-1; off fixed (off_hi None) or log-uniform."""
    nseg = n_segments(dom)
    if count == 0 or nseg == 0:
        return np.zeros((0, 2))
    which = rng.integers(0, nseg, count)
    t = rng.uniform(0.0, 1.0, count)
    side = rng.choice([-1.0, 1.0], count)
    if off_hi is None:
        off = np.full(count, off_lo)
    else:
        off = np.exp(rng.uniform(math.log(off_lo), math.log(off_hi), count))
    degs = dom["degrees"].astype(np.int64)
    start = np.concatenate([[0], np.cumsum(degs + 1)[:-1]])
    wall = dom.get("weights")
    out = np.empty((count, 2))
    for n in np.unique(degs[which]):
        sel = np.nonzero(degs[which] == n)[0]
        base = start[which[sel]]
        idx = base[:, None] + np.arange(n + 1)[None, :]
        cps = dom["cps"][idx]      # (k, n+1, 2)
        wt = np.ones((sel.size, n + 1)) if wall is None else wall[idx]
        tt = t[sel][:, None]
        # placement only: homogeneous Bernstein sums (x w, y w, w) and their
        # derivative give the point and the tangent direction
        hp = np.zeros((sel.size, 3))
        hd = np.zeros((sel.size, 3))
        H = np.concatenate([cps * wt[:, :, None], wt[:, :, None]], axis=2)
        for k in range(n + 1):
            hp += comb(n, k) * tt ** k * (1 - tt) ** (n - k) * H[:, k]
        for k in range(n):
            hd += n * comb(n - 1, k) * tt ** k * (1 - tt) ** (n - 1 - k) * (H[:, k + 1] - H[:, k])
        if wall is None:        # polynomial: the Bernstein sums themselves
            pt = hp[:, :2]
            dv = hd[:, :2]
        else:
            pt = hp[:, :2] / hp[:, 2:3]
            dv = (hd[:, :2] * hp[:, 2:3] - hp[:, :2] * hd[:, 2:3])
        L = np.hypot(dv[:, 0], dv[:, 1])
        ok = L > 0
        nh = np.zeros((sel.size, 2))
        nh[:, 1] = 1.0
        nh[ok] = np.stack([-dv[ok, 1], dv[ok, 0]], axis=1) / L[ok, None]
        out[sel] = pt + (side[sel] * off[sel])[:, None] * nh
    return out


# --------------------------------------------------------------------------
# workload 1: plain FP64, one planar domain
# --------------------------------------------------------------------------
def config1(n_uniform=100_000, n_near=10_000, seed_index=1):
    """One outer CCW loop of 64 cubics (radius 0.4 +- 0.05, C0) and two CW
    circular holes of 16 cubics (radius 0.08 at (0.35,.5), (0.65,.5))."""
    rng = rng_for(seed_index)
    c = np.array([0.5, 0.5])
    m = 64
    ang = TWO_PI * np.arange(m) / m
    r = 0.4 + rng.uniform(-0.05, 0.05, m)
    verts = c + np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
    # inner control points at 1/3 and 2/3 of the chord, each displaced by
    # U(-0.01,0.01) (absolute units) along the chord normal
    outer = []
    for k in range(m):
        p0, p3 = verts[k], verts[(k + 1) % m]
        d = p3 - p0
        L = math.hypot(*d)
        nrm = np.array([-d[1], d[0]]) / L
        p1 = p0 + d / 3 + nrm * rng.uniform(-0.01, 0.01)
        p2 = p0 + 2 * d / 3 + nrm * rng.uniform(-0.01, 0.01)
        outer.append(np.array([p0, p1, p2, p3]))
    holes = [circle_loop((0.35, 0.5), 0.08, 16, ccw=False),
             circle_loop((0.65, 0.5), 0.08, 16, ccw=False)]
    dom = make_domain([outer] + holes, eps=1e-9)
    q = [rng.uniform(0.0, 1.0, (n_uniform, 2)), _near_points(rng, dom, n_near, 1e-6)]
    return dom, np.ascontiguousarray(np.concatenate(q, axis=0))


# --------------------------------------------------------------------------
# workload 2: open / noisy boundaries, 64 planar domains
# --------------------------------------------------------------------------
def config2(n_domains=64, n_uniform=10_000_000, n_near=1_000_000, seed_index=2,
            loops=(4, 12), segs=(32, 512), domain_subset=None):
    """Per domain 4-12 star loops of 32-512 segments of degree U{1..5}, every
    join opened by a log-uniform 1e-4..1e-2 gap, control-point noise
    N(0,1e-4); queries split evenly over domains: uniform in [0,1]^2 plus
    near-curve points offset log-uniform 1e-7..1e-3 along the normal.
    Returns (list of domains, list of per-domain query arrays)."""
    doms, qs = [], []
    nu = [n_uniform // n_domains + (1 if i < n_uniform % n_domains else 0) for i in range(n_domains)]
    nn = [n_near // n_domains + (1 if i < n_near % n_domains else 0) for i in range(n_domains)]
    idx = range(n_domains) if domain_subset is None else domain_subset
    for d in idx:
        rng = rng_for(seed_index, salt=d + 1)
        nl = int(rng.integers(loops[0], loops[1] + 1))
        lps = []
        for _ in range(nl):
            ns = int(rng.integers(segs[0], segs[1] + 1))
            degs = rng.integers(1, 6, ns)
            ctr = rng.uniform(0.2, 0.8, 2)
            rad = rng.uniform(0.05, 0.3)
            lps.append(star_loop(rng, ctr, rad, ns, degs, noise=1e-4, ccw=True,
                                 bend=0.2, gap_lo=1e-4, gap_hi=1e-2, radial_noise=0.2))
        dom = make_domain(lps, eps=1e-9)
        qrng = rng_for(seed_index, salt=100000 + d)
        q = np.concatenate([qrng.uniform(0.0, 1.0, (nu[d], 2)),
                            _near_points(qrng, dom, nn[d], 1e-7, 1e-3)], axis=0)
        doms.append(dom)
        qs.append(np.ascontiguousarray(q))
    return doms, qs


# --------------------------------------------------------------------------
# workload 6: rational segments (the rational case of App. A.1)
# --------------------------------------------------------------------------
def config6(n_domains=64, n_uniform=10_000_000, n_near=1_000_000, seed_index=6,
            loops=(4, 12), segs=(32, 512), domain_subset=None):
    """Workload 2's open/noisy star loops with every control point weighted
    (log-uniform in [0.8, 1.25], the range of conic-section weights), plus two
    holes per face that are exact circles
    of rational quadratic arcs of unequal angles; queries as in workload 2.
    Returns (list of domains, list of per-domain query arrays)."""
    doms, qs = [], []
    nu = [n_uniform // n_domains + (1 if i < n_uniform % n_domains else 0) for i in range(n_domains)]
    nn = [n_near // n_domains + (1 if i < n_near % n_domains else 0) for i in range(n_domains)]
    idx = range(n_domains) if domain_subset is None else domain_subset
    for d in idx:
        rng = rng_for(seed_index, salt=d + 1)
        nl = int(rng.integers(loops[0], loops[1] + 1))
        lps = []
        for _ in range(nl):
            ns = int(rng.integers(segs[0], segs[1] + 1))
            degs = rng.integers(1, 6, ns)
            ctr = rng.uniform(0.2, 0.8, 2)
            rad = rng.uniform(0.05, 0.3)
            star = star_loop(rng, ctr, rad, ns, degs, noise=1e-4, ccw=True,
                             bend=0.2, gap_lo=1e-4, gap_hi=1e-2, radial_noise=0.2)
            lps.append([(s, np.exp(rng.uniform(-math.log(1.25), math.log(1.25), s.shape[0]))) for s in star])
        for _ in range(2):
            k = int(rng.integers(3, 7))
            cuts = np.sort(rng.uniform(0.0, 1.0, k - 1))
            ang = np.diff(np.concatenate([[0.0], cuts, [1.0]])) * TWO_PI
            while np.any(ang >= 3.0) or np.any(ang <= 0.05):
                cuts = np.sort(rng.uniform(0.0, 1.0, k - 1))
                ang = np.diff(np.concatenate([[0.0], cuts, [1.0]])) * TWO_PI
            lps.append(rational_circle_loop(rng.uniform(0.2, 0.8, 2), rng.uniform(0.02, 0.1), ang, ccw=False))
        dom = make_domain(lps, eps=1e-9)
        qrng = rng_for(seed_index, salt=100000 + d)
        q = np.concatenate([qrng.uniform(0.0, 1.0, (nu[d], 2)),
                            _near_points(qrng, dom, nn[d], 1e-7, 1e-3)], axis=0)
        doms.append(dom)
        qs.append(np.ascontiguousarray(q))
    return doms, qs


# --------------------------------------------------------------------------
# periodic helpers
# --------------------------------------------------------------------------
def _wrap_segments(segs, pu, pv):
    """Store every segment translated by a lattice vector so that its start
    lies in [0,pu) x [0,pv) (axes with period 0 are left alone)."""
    out = []
    for s in segs:
        s = s.copy()
        if pu > 0:
            s[:, 0] -= pu * math.floor(s[0, 0] / pu)
        if pv > 0:
            s[:, 1] -= pv * math.floor(s[0, 1] / pv)
        out.append(s)
    return out


def _hermite_cubics(f, df, m, t0=0.0, t1=1.0):
    """Cubic Hermite segments through f(t) on m equal steps of [t0,t1]."""
    ts = np.linspace(t0, t1, m + 1)
    P = [np.asarray(f(t)) for t in ts]
    D = [np.asarray(df(t)) for t in ts]
    h = (t1 - t0) / m
    segs = []
    for i in range(m):
        segs.append(np.array([P[i], P[i] + D[i] * h / 3, P[i + 1] - D[i + 1] * h / 3, P[i + 1]]))
    return segs


def wavy_line(o, v, nrm, amp, k, m):
    """o + t v + amp sin(2 pi k t) nrm, t in [0,1], as m cubic segments; the
    end is exactly o + v."""
    o, v, nrm = (np.asarray(x, dtype=np.float64) for x in (o, v, nrm))
    f = lambda t: o + t * v + amp * math.sin(TWO_PI * k * t) * nrm
    df = lambda t: v + amp * TWO_PI * k * math.cos(TWO_PI * k * t) * nrm
    segs = _hermite_cubics(f, df, m)
    segs[-1][-1] = o + v
    segs[0][0] = o.copy()
    return segs


def reverse_loop(segs):
    return [s[::-1].copy() for s in segs[::-1]]


def sphere_cap_face(rng, v0=0.35, amp=0.15, k=3, m=24, hole=True):
    """A trimmed sphere, parameterized by longitude u in [0, 2 pi) (periodic)
    and latitude v in [-pi/2, pi/2], with the two poles (singular points of
    the parameterization) removed, so that the domain is a cylinder (Sec. 4.3):
    the face is the cap north of the wavy latitude curve
    v = v0 + amp sin(k u) (one loop with homology (1, 0), traversed in +u so
    the cap lies on its left) up to the punctured north pole, whose line
    v = pi/2 is the cap's second boundary loop (traversed in -u; B-Rep models
    store a degenerate edge there), less an optional small hole crossing the
    seam.  Returns (loops wrapped per segment, hole centre, hole radius)."""
    segs = wavy_line((0.0, v0), (TWO_PI, 0.0), (0.0, 1.0), amp, k, m)
    pole = reverse_loop(wavy_line((0.0, 0.5 * math.pi), (TWO_PI, 0.0), (0.0, 1.0), 0.0, 1, 4))
    loops = [segs, pole]
    hc, hr = (0.05, v0 + 0.6), 0.12
    if hole:
        loops.append(circle_loop(hc, hr, 16, ccw=False))
    return [_wrap_segments(lp, TWO_PI, 0.0) for lp in loops], hc, hr


def sphere_points(rng, n):
    """Points uniform on the unit sphere as (longitude in [0, 2 pi), latitude)."""
    z = rng.uniform(-1.0, 1.0, n)
    lon = rng.uniform(0.0, TWO_PI, n)
    return np.stack([lon, np.arcsin(z)], axis=1)


def cone_face(t0=0.3, t1=0.8, amp=0.05, k=2, m=16):
    """A trimmed cone, parameterized by the angle u in [0, 2 pi) (periodic) and
    the distance t from the apex, the apex (t = 0, a singular point) removed:
    the face is the apex region 0 < t < t0 + amp sin(k u) (a loop traversed
    in -u, the apex side on its left, and the punctured apex's line t = 0 in
    +u) and the band t1 < t < 1 (a loop in +u at t1 and one in -u at 1)."""
    apex = wavy_line((0.0, 0.0), (TWO_PI, 0.0), (0.0, 1.0), 0.0, 1, 4)
    a = reverse_loop(wavy_line((0.0, t0), (TWO_PI, 0.0), (0.0, 1.0), amp, k, m))
    b = wavy_line((0.0, t1), (TWO_PI, 0.0), (0.0, 1.0), 0.0, 1, 8)
    c = reverse_loop(wavy_line((0.0, 1.0), (TWO_PI, 0.0), (0.0, 1.0), 0.0, 1, 8))
    return [_wrap_segments(lp, TWO_PI, 0.0) for lp in (apex, a, b, c)]


def swap_axes_loops(loops):
    """The same loops with u and v exchanged and each loop reversed: a face
    periodic in u becomes a face periodic in v with the same inside (the
    mirror alone would flip every orientation)."""
    return [reverse_loop([s[:, ::-1].copy() for s in lp]) for lp in loops]


HOMOLOGIES = [(1, 0), (0, 1), (1, 1), (1, 2), (2, 1), (2, 3), (3, 2)]


def biperiodic_face(rng, n_loops, seg_range, P=TWO_PI, open_frac=0.1, nc_frac=0.3):
    """One bi-periodic face with period P on both axes: pairs of
    non-contractible wavy loops with homology +-(p,q) (each pair bounds a
    band), plus contractible star loops placed in the free strips between
    the curves.  Loops are stored per-segment wrapped."""
    n_pairs = int(math.floor(nc_frac * n_loops / 2.0 + rng.uniform(0, 1)))
    n_pairs = min(n_pairs, n_loops // 2)
    n_con = n_loops - 2 * n_pairs
    loops = []
    if n_pairs > 0:
        p, q = HOMOLOGIES[int(rng.integers(0, len(HOMOLOGIES)))]
        v = np.array([p * P, q * P])
        L = math.hypot(*v)
        nh = np.array([-v[1], v[0]]) / L
        spacing = P * P / L                        # distance between families
        slot = spacing / n_pairs                   # one pair per slot
        amp = 0.12 * slot
        base = rng.uniform(0, P, 2)
        free = []
        for j in range(n_pairs):
            k = int(rng.integers(1, 4))
            m = int(rng.integers(seg_range[0], seg_range[1] + 1))
            oa = base + nh * (j * slot)
            ob = oa + nh * (0.5 * slot)
            alpha = wavy_line(oa, v, nh, amp, k, m)
            beta = reverse_loop(wavy_line(ob, v, nh, amp, k, m))
            loops += [alpha, beta]
            free.append((j * slot + 0.25 * slot, 0.5 * slot - 2 * amp))
            free.append((j * slot + 0.75 * slot, 0.5 * slot - 2 * amp))
        for _ in range(n_con):
            c_n, width = free[int(rng.integers(0, len(free)))]
            rad = 0.4 * 0.5 * width
            along = rng.uniform(0, L)
            ctr = base + nh * c_n + (v / L) * along
            m = int(rng.integers(seg_range[0], seg_range[1] + 1))
            loops.append(star_loop(rng, ctr, rad, m, 3, ccw=bool(rng.integers(0, 2)),
                                   bend=0.1, radial_noise=0.15))
    else:
        for _ in range(n_con):
            ctr = rng.uniform(0, P, 2)
            rad = rng.uniform(0.05, 0.3) * P / 2
            m = int(rng.integers(seg_range[0], seg_range[1] + 1))
            loops.append(star_loop(rng, ctr, rad, m, 3, ccw=True, bend=0.1,
                                   radial_noise=0.15))
    out = []
    for lp in loops:
        if rng.uniform() < open_frac:
            if len(lp) > 3 and rng.uniform() < 0.5:
                drop = int(rng.integers(0, len(lp)))
                lp = lp[:drop] + lp[drop + 1:]
            else:
                lp = [s + np.where(np.arange(s.shape[0])[:, None] == 0,
                                   rng.normal(0, 1e-3, 2), 0.0) for s in lp]
        out.append(_wrap_segments(lp, P, P))
    return out


def uniperiodic_face(rng, n_loops, seg_range, P=1.0, degrees=(3, 3)):
    """Cylinder-like face, period P in u only: pairs of separation loops
    (homology +-1) with contractible star loops between them."""
    n_pairs = max(1, n_loops // 3)
    n_con = max(0, n_loops - 2 * n_pairs)
    loops = []
    slot = 1.0 / n_pairs
    amp = 0.1 * slot
    free = []
    for j in range(n_pairs):
        y0 = j * slot + 0.1 * slot
        y1 = y0 + 0.5 * slot
        k = int(rng.integers(1, 4))
        m = int(rng.integers(seg_range[0], seg_range[1] + 1))
        x0 = rng.uniform(0, P)
        a = wavy_line((x0, y0), (P, 0.0), (0.0, 1.0), amp, k, m)
        b = reverse_loop(wavy_line((x0, y1), (P, 0.0), (0.0, 1.0), amp, k, m))
        loops += [a, b]
        free.append((y0 + 0.25 * slot, 0.5 * slot - 2 * amp))
    for _ in range(n_con):
        yc, width = free[int(rng.integers(0, len(free)))]
        rad = 0.4 * 0.5 * width
        m = int(rng.integers(seg_range[0], seg_range[1] + 1))
        ctr = (rng.uniform(0, P), yc)
        loops.append(star_loop(rng, ctr, rad, m, int(rng.integers(degrees[0], degrees[1] + 1)),
                               ccw=False, bend=0.1, radial_noise=0.15))
    return [_wrap_segments(lp, P, 0.0) for lp in loops]


# --------------------------------------------------------------------------
# workload 3: bi-periodic torus-like faces
# --------------------------------------------------------------------------
def config3(n_faces=256, n_queries=20_000_000, seed_index=3, seg_range=(16, 256),
            loops=(2, 8), face_subset=None):
    doms, qs = [], []
    nq = [n_queries // n_faces + (1 if i < n_queries % n_faces else 0) for i in range(n_faces)]
    idx = range(n_faces) if face_subset is None else face_subset
    for f in idx:
        rng = rng_for(seed_index, salt=f + 1)
        nl = int(rng.integers(loops[0], loops[1] + 1))
        lps = biperiodic_face(rng, nl, seg_range)
        doms.append(make_domain(lps, TWO_PI, TWO_PI, eps=TWO_PI * 1e-9))
        qrng = rng_for(seed_index, salt=100000 + f)
        qs.append(np.ascontiguousarray(qrng.uniform(0.0, TWO_PI, (nq[f], 2))))
    return doms, qs


# --------------------------------------------------------------------------
# workload 4: batched B-Rep-shaped faces
# --------------------------------------------------------------------------
def _planar_closed_face(rng, n_loops, n_segs, degrees_per_seg):
    """Outer CCW star loop plus CW star holes placed inside it, disjoint,
    with C0 joins; ``n_segs`` split over the loops."""
    n_loops = max(1, n_loops)
    share = np.maximum(4, np.round(n_segs * rng.dirichlet(np.ones(n_loops) * 2.0)).astype(int))
    c = np.array([0.5, 0.5])
    loops = []
    pos = 0
    loops.append(star_loop(rng, c, 0.4, int(share[0]), degrees_per_seg[pos:pos + share[0]],
                           ccw=True, bend=0.1, radial_noise=0.1))
    pos += share[0]
    placed = []
    for j in range(1, n_loops):
        for _ in range(50):
            r = rng.uniform(0.02, 0.07)
            ctr = c + rng.uniform(-0.22, 0.22, 2)
            if all(np.hypot(*(ctr - q)) > r + rq + 0.02 for q, rq in placed):
                placed.append((ctr, r))
                break
        else:
            continue
        cnt = int(share[j])
        dg = degrees_per_seg[pos:pos + cnt] if pos + cnt <= len(degrees_per_seg) else 3
        pos += cnt
        loops.append(star_loop(rng, ctr, r, cnt, dg, ccw=False, bend=0.1, radial_noise=0.1))
    return loops


def config4_sizes(n_faces=10_000, total_queries=200_000_000, seed_index=4):
    rng = rng_for(seed_index)
    S = np.clip(np.round(np.exp(rng.normal(math.log(40), 1.0, n_faces))), 4, 4000).astype(int)
    Q = np.clip(np.exp(rng.normal(math.log(4096), 1.794, n_faces)), 16, 1_048_576)
    Q = Q * (total_queries / Q.sum())
    Q = np.clip(np.round(Q), 16, 1_048_576).astype(np.int64)
    kind = rng.uniform(0, 1, n_faces)
    return S, Q, kind


def config4(n_faces=10_000, total_queries=200_000_000, seed_index=4, face_subset=None,
            query_scale=1.0):
    S, Q, kind = config4_sizes(n_faces, total_queries, seed_index)
    doms, qs = [], []
    idx = range(n_faces) if face_subset is None else face_subset
    for f in idx:
        rng = rng_for(seed_index, salt=f + 1)
        nl = int(rng.integers(1, 9))
        s = int(S[f])
        nq = max(1, int(round(Q[f] * query_scale)))
        if kind[f] < 0.1:            # uni-periodic in u, period 1
            lps = uniperiodic_face(rng, max(2, nl), (max(4, s // max(2, nl)),) * 2, P=1.0,
                                   degrees=(1, 5))
            dom = make_domain(lps, 1.0, 0.0, eps=1e-9)
            q = np.stack([rng.uniform(0, 1, nq), rng.uniform(0, 1, nq)], axis=1)
        elif kind[f] < 0.2:          # bi-periodic, period 2 pi
            per = max(4, s // max(2, nl))
            lps = biperiodic_face(rng, max(2, nl), (per, per), open_frac=0.0)
            dom = make_domain(lps, TWO_PI, TWO_PI, eps=TWO_PI * 1e-9)
            q = rng.uniform(0, TWO_PI, (nq, 2))
        else:                        # planar closed
            degs = rng.integers(1, 6, s + 64)
            lps = _planar_closed_face(rng, nl, s, degs)
            dom = make_domain(lps, eps=1e-9)
            q = rng.uniform(0, 1, (nq, 2))
        doms.append(dom)
        qs.append(np.ascontiguousarray(q))
    return doms, qs


# --------------------------------------------------------------------------
# workload 5: tessellation-shaped dense grids
# --------------------------------------------------------------------------
def fractal_outer(rng, n_base=5, levels=14, radius=0.4, amp0=0.05, rough=0.6):
    """Closed polygon from recursive midpoint displacement of a circle,
    turned into C0 cubics (inner points at 1/3, 2/3 of each edge with a
    small normal bend)."""
    ang = TWO_PI * np.arange(n_base) / n_base
    P = 0.5 + radius * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    amp = amp0
    for _ in range(levels):
        Q = np.roll(P, -1, axis=0)
        mid = 0.5 * (P + Q)
        d = Q - P
        L = np.hypot(d[:, 0], d[:, 1])[:, None]
        nrm = np.stack([-d[:, 1], d[:, 0]], axis=1) / np.maximum(L, 1e-300)
        mid = mid + nrm * (rng.uniform(-1, 1, (P.shape[0], 1)) * amp * L / (L.mean() + 1e-300) * 0.5)
        out = np.empty((2 * P.shape[0], 2))
        out[0::2] = P
        out[1::2] = mid
        P = out
        amp *= rough
    Q = np.roll(P, -1, axis=0)
    d = Q - P
    L = np.hypot(d[:, 0], d[:, 1])[:, None]
    nrm = np.stack([-d[:, 1], d[:, 0]], axis=1) / np.maximum(L, 1e-300)
    b1 = rng.uniform(-0.05, 0.05, (P.shape[0], 1)) * L
    b2 = rng.uniform(-0.05, 0.05, (P.shape[0], 1)) * L
    cps = np.stack([P, P + d / 3 + nrm * b1, P + 2 * d / 3 + nrm * b2, Q], axis=1)
    return [cps[i] for i in range(cps.shape[0])]


def config5_face(face, seed_index=5, n_holes=200, levels=14, hole_segs=100):
    rng = rng_for(seed_index, salt=face + 1)
    outer = fractal_outer(rng, levels=levels)
    holes, placed = [], []
    tries = 0
    while len(holes) < n_holes and tries < 100 * n_holes:
        tries += 1
        r = rng.uniform(0.002, 0.01)
        ctr = 0.5 + rng.uniform(-0.2, 0.2, 2)
        if np.hypot(*(ctr - 0.5)) > 0.22:
            continue
        if any(np.hypot(*(ctr - q)) <= r + rq + 0.002 for q, rq in placed):
            continue
        placed.append((ctr, r))
        holes.append(star_loop(rng, ctr, r, hole_segs, 3, ccw=False, bend=0.1,
                               radial_noise=0.15))
    return make_domain([outer] + holes, eps=1e-9)


def grid_points(nu, nv):
    """Cell centres ((i+1/2)/nu, (j+1/2)/nv), row-major with i fastest."""
    u = (np.arange(nu) + 0.5) / nu
    v = (np.arange(nv) + 0.5) / nv
    U, V = np.meshgrid(u, v)
    return np.ascontiguousarray(np.stack([U.ravel(), V.ravel()], axis=1))
