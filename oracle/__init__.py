"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It builds
``wn_oracle.c`` with gcc and calls it through ctypes.  It shares no code with
the CUDA library in ``paper_2510_25159_gb300``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libwn_oracle.so")
_lock = threading.Lock()
_lib = None

OUTSIDE, INSIDE, BOUNDARY = 0, 1, 2


def build(force: bool = False, extra_flags=()) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_PATH if not extra_flags else os.path.join(
        _BUILD, "libwn_oracle_" + "_".join(f.strip("-").replace("=", "") for f in extra_flags) + ".so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", "-pthread", *extra_flags,
               _SRC, "-o", out + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)
    return out


def _bind(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.or_query.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int64, P, P, P, P, ctypes.c_int32, P]
    lib.or_query.restype = ctypes.c_int
    lib.or_segment_wn.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, P, P]
    lib.or_segment_wn.restype = ctypes.c_int
    lib.or_hull_segment_wn.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, P, P]
    lib.or_hull_segment_wn.restype = ctypes.c_int
    lib.or_eval.argtypes = [ctypes.c_int, P, ctypes.c_double, P]
    lib.or_eval.restype = ctypes.c_int
    lib.or_bound.argtypes = [ctypes.c_int, P]
    lib.or_bound.restype = ctypes.c_double
    lib.or_domain_info.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, P, P, P, P, P]
    lib.or_domain_info.restype = ctypes.c_int
    lib.or_extended_wn.argtypes = [ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, P]
    lib.or_extended_wn.restype = ctypes.c_int
    lib.or_query_w.argtypes = [ctypes.c_int32, P, P, P, P, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_int64, P, P, P, P, ctypes.c_int32, P]
    lib.or_query_w.restype = ctypes.c_int
    lib.or_segment_wn_w.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, P, P]
    lib.or_segment_wn_w.restype = ctypes.c_int
    lib.or_eval_w.argtypes = [ctypes.c_int, P, P, ctypes.c_double, P]
    lib.or_eval_w.restype = ctypes.c_int
    lib.or_bound_w.argtypes = [ctypes.c_int, P, P]
    lib.or_bound_w.restype = ctypes.c_double
    return lib


def lib(path=None):
    global _lib
    if path is not None:
        return _bind(path)
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _dom_arrays(dom):
    lo = np.ascontiguousarray(dom["loop_offsets"], dtype=np.int32)
    dg = np.ascontiguousarray(dom["degrees"], dtype=np.int32)
    cp = np.ascontiguousarray(dom["cps"], dtype=np.float64).reshape(-1)
    return lo, dg, cp


def _weights(w):
    return None if w is None else np.ascontiguousarray(w, dtype=np.float64).reshape(-1)


def query(dom, pts, threads=None, margins=False, stats=False, eps=None, L=None):
    """omega (NaN for BOUNDARY), state (u8) [, margin] [, stats dict].
    A domain with "weights" (one per control point) is rational."""
    L = L or lib()
    lo, dg, cp = _dom_arrays(dom)
    wt = _weights(dom.get("weights"))
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    n = pts.shape[0]
    w = np.empty(n)
    st = np.empty(n, dtype=np.uint8)
    mg = np.empty(n) if margins else None
    s5 = np.zeros(5, dtype=np.int64)
    th = threads or os.cpu_count() or 1
    e = dom["eps"] if eps is None else eps
    if wt is None:
        rc = L.or_query(len(lo) - 1, _p(lo), _p(dg), _p(cp), dom["period_u"], dom["period_v"], e,
                        n, _p(pts), _p(w), _p(st), _p(mg), th, _p(s5))
    else:
        rc = L.or_query_w(len(lo) - 1, _p(lo), _p(dg), _p(cp), _p(wt), dom["period_u"], dom["period_v"], e,
                          n, _p(pts), _p(w), _p(st), _p(mg), th, _p(s5))
    if rc != 0:
        raise OracleError(rc)
    out = [w, st]
    if margins:
        out.append(mg)
    if stats:
        out.append(dict(zip(["evals", "nodes", "chords", "max_depth", "depth_cap"], s5.tolist())))
    return tuple(out)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


def segment_wn(cps, p, eps=1e-12, L=None, weights=None):
    """Algorithm 1 on one segment (rational with weights): (angle_radians,
    boundary, stats dict)."""
    L = L or lib()
    cps = np.ascontiguousarray(cps, dtype=np.float64).reshape(-1)
    a = np.zeros(1)
    s5 = np.zeros(5, dtype=np.int64)
    wt = _weights(weights)
    if wt is None:
        b = L.or_segment_wn(cps.size // 2 - 1, _p(cps), float(p[0]), float(p[1]), eps, _p(a), _p(s5))
    else:
        b = L.or_segment_wn_w(cps.size // 2 - 1, _p(cps), _p(wt), float(p[0]), float(p[1]), eps, _p(a),
                              _p(s5))
    return float(a[0]), bool(b), dict(zip(["evals", "nodes", "chords", "max_depth", "depth_cap"], s5.tolist()))


def hull_segment_wn(cps, p, eps=1e-12, L=None):
    L = L or lib()
    cps = np.ascontiguousarray(cps, dtype=np.float64).reshape(-1)
    a = np.zeros(1)
    e = np.zeros(1, dtype=np.int64)
    b = L.or_hull_segment_wn(cps.size // 2 - 1, _p(cps), float(p[0]), float(p[1]), eps, _p(a), _p(e))
    return float(a[0]), bool(b), int(e[0])


def eval_point(cps, t, L=None, weights=None):
    L = L or lib()
    cps = np.ascontiguousarray(cps, dtype=np.float64).reshape(-1)
    o = np.zeros(2)
    wt = _weights(weights)
    if wt is None:
        L.or_eval(cps.size // 2 - 1, _p(cps), float(t), _p(o))
    else:
        L.or_eval_w(cps.size // 2 - 1, _p(cps), _p(wt), float(t), _p(o))
    return o


def bound(cps, L=None, weights=None):
    L = L or lib()
    cps = np.ascontiguousarray(cps, dtype=np.float64).reshape(-1)
    wt = _weights(weights)
    if wt is None:
        return float(L.or_bound(cps.size // 2 - 1, _p(cps)))
    return float(L.or_bound_w(cps.size // 2 - 1, _p(cps), _p(wt)))


def domain_info(dom, L=None):
    """Lifted control points, homology (n_loops,2), pairs (n,4), eps."""
    L = L or lib()
    lo, dg, cp = _dom_arrays(dom)
    nl = len(lo) - 1
    lifted = np.empty_like(cp)
    hom = np.zeros(2 * max(nl, 1), dtype=np.int32)
    pairs = np.zeros(4 * max(nl, 1), dtype=np.int64)
    npairs = np.zeros(1, dtype=np.int32)
    eps = np.zeros(1)
    rc = L.or_domain_info(nl, _p(lo), _p(dg), _p(cp), dom["period_u"], dom["period_v"],
                          dom["eps"], _p(lifted), _p(hom), _p(pairs), _p(npairs), _p(eps))
    if rc != 0:
        raise OracleError(rc)
    k = int(npairs[0])
    return lifted.reshape(-1, 2), hom[:2 * nl].reshape(nl, 2), pairs[:4 * k].reshape(k, 4), float(eps[0])


def extended_wn(segs, Pu, Pv, hp, hq, p, eps=1e-12, L=None):
    """Eq. 9 for a single lifted curve (list of (n+1,2) arrays)."""
    L = L or lib()
    dg = np.asarray([s.shape[0] - 1 for s in segs], dtype=np.int32)
    cp = np.ascontiguousarray(np.concatenate(segs, axis=0), dtype=np.float64).reshape(-1)
    w = np.zeros(1)
    rc = L.or_extended_wn(len(segs), _p(dg), _p(cp), Pu, Pv, hp, hq, eps, float(p[0]),
                          float(p[1]), _p(w))
    if rc < 0:
        raise OracleError(-rc)
    return float(w[0]), bool(rc)
