"""Containment queries on trimmed surfaces for GB300 (sm_103a).

Thin ctypes binding of the C ABI in ``include/wn.h`` (``_build/libwn.so``):
argument marshalling only.  Every step of the query runs in the library's
CUDA kernels; there is no CPU fallback, and importing a function that needs
the library raises when ``libwn.so`` has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).

Device buffers are torch CUDA tensors (``data_ptr()``) ordered on the current
torch stream; host buffers are numpy arrays (the library stages the copies).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OUTSIDE, INSIDE, BOUNDARY = 0, 1, 2
PLAIN_FP64, MIXED = 0, 1
MAX_DEGREE = 7

_STATUS = {0: "WN_OK", 1: "WN_ERR_ARG", 2: "WN_ERR_TOPOLOGY", 3: "WN_ERR_CUDA", 4: "WN_ERR_OOM",
           5: "WN_ERR_LIMIT"}
_lib = None


class WnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class WnStats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
                ("fp64_pairs", ctypes.c_int64), ("fp64_queries", ctypes.c_int64),
                ("overflow", ctypes.c_int64), ("depth_cap", ctypes.c_int64),
                ("kernels", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.wn_create_domain.argtypes = [P, I32, P, P, D, D, D, ctypes.POINTER(ctypes.c_void_p)]
        L.wn_create_domain_rational.argtypes = [P, I32, P, P, P, D, D, D, ctypes.POINTER(ctypes.c_void_p)]
        L.wn_grid_triangles.argtypes = [P, I32, I32, I32, I32, P, I64, P, P]
        L.wn_grid_triangles.restype = ctypes.c_int
        L.wn_query_surfaces.argtypes = [P, P, I32, P, P, P, ctypes.c_int, P]
        L.wn_query_surfaces.restype = ctypes.c_int
        L.wn_query_midpoints.argtypes = [P, P, I64, P, ctypes.c_int, P]
        L.wn_query_midpoints.restype = ctypes.c_int
        L.wn_destroy_domain.argtypes = [P]
        L.wn_destroy_domain.restype = None
        L.wn_query.argtypes = [P, P, I64, P, P, ctypes.c_int, P]
        L.wn_query_batched.argtypes = [P, I32, P, P, P, P, ctypes.c_int, P]
        L.wn_query_grid_bitmask.argtypes = [P, I32, I32, P, P, ctypes.c_int, P]
        L.wn_set_tuning.argtypes = [I32, I32, I32, I32, I32, I32]
        L.wn_get_stats.argtypes = [ctypes.POINTER(WnStats)]
        L.wn_last_error.restype = ctypes.c_char_p
        L.wn_version.restype = ctypes.c_char_p
        L.wn_query_noalloc.argtypes = [P, P, I64, P, P, P]
        L.wn_query_noalloc.restype = ctypes.c_int
        L.wn_autotune.argtypes = [P, I32, P, P, I32, P, P]
        L.wn_get_tuning.argtypes = [P, I32]
        L.wn_set_near_tuning.argtypes = [I32, I32, I32]
        L.wn_set_queue_limits.argtypes = [I64, I64]
        L.wn_set_flat_records.argtypes = [I32]
        L.wn_set_grid_tile.argtypes = [I32]
        L.wn_near_work.argtypes = [P]
        L.wn_last_escalated.argtypes = [P, I64, P]
        L.wn_eval_gap_angle.argtypes = [P, P, P, I64, P]
        L.wn_rational_bounds.argtypes = [P, P, I32, P]
        L.wn_set_profiling.argtypes = [I32]
        L.wn_kernel_times.argtypes = [P, P]
        L.wn_set_work_counting.argtypes = [I32]
        L.wn_sweep_work.argtypes = [P, I32]
        for f in ("wn_create_domain", "wn_create_domain_rational", "wn_query", "wn_query_batched", "wn_query_grid_bitmask",
                  "wn_set_tuning", "wn_get_stats", "wn_set_profiling", "wn_kernel_times", "wn_autotune",
                  "wn_get_tuning", "wn_set_work_counting", "wn_sweep_work", "wn_set_near_tuning",
                  "wn_set_queue_limits", "wn_near_work", "wn_last_escalated",
                  "wn_eval_gap_angle", "wn_set_flat_records", "wn_set_grid_tile", "wn_rational_bounds"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise WnError(rc, lib().wn_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


class Domain:
    """One face's trimming loops (``wn_create_domain``; with ``weights``, one
    per control point, ``wn_create_domain_rational``)."""

    def __init__(self, loop_offsets, degrees, control_points, period_u=0.0, period_v=0.0, eps=0.0,
                 weights=None):
        lo = np.ascontiguousarray(loop_offsets, dtype=np.int32)
        dg = np.ascontiguousarray(degrees, dtype=np.int32)
        cp = np.ascontiguousarray(control_points, dtype=np.float64).reshape(-1)
        h = ctypes.c_void_p()
        self._h = None
        if weights is None:
            _check(lib().wn_create_domain(_ptr(lo), len(lo) - 1, _ptr(dg), _ptr(cp), float(period_u),
                                          float(period_v), float(eps), ctypes.byref(h)))
        else:
            wt = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
            if wt.size * 2 != cp.size:
                raise ValueError("one weight per control point")
            _check(lib().wn_create_domain_rational(_ptr(lo), len(lo) - 1, _ptr(dg), _ptr(cp), _ptr(wt),
                                                   float(period_u), float(period_v), float(eps),
                                                   ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_dict(cls, d, eps=None):
        return cls(d["loop_offsets"], d["degrees"], d["cps"], d["period_u"], d["period_v"],
                   d["eps"] if eps is None else eps, weights=d.get("weights"))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and _lib is not None:
            _lib.wn_destroy_domain(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def query(domain, points, precision=MIXED, out_winding=None, out_inside=None, stream=None):
    """Winding numbers and states of ``points`` ((n,2) float64, torch CUDA or
    numpy host).  Returns (winding, inside) in the same kind of memory."""
    n = int(points.shape[0])
    if out_winding is None or out_inside is None:
        if isinstance(points, np.ndarray):
            out_winding = np.empty(n) if out_winding is None else out_winding
            out_inside = np.empty(n, dtype=np.uint8) if out_inside is None else out_inside
        else:
            import torch
            out_winding = torch.empty(n, dtype=torch.float64, device=points.device) if out_winding is None else out_winding
            out_inside = torch.empty(n, dtype=torch.uint8, device=points.device) if out_inside is None else out_inside
    _check(lib().wn_query(domain.handle, _ptr(points), n, _ptr(out_winding), _ptr(out_inside),
                          int(precision), _stream(stream)))
    return out_winding, out_inside


NOALLOC_MAX_QUERIES = 65536


def query_noalloc(domain, points, out_winding, out_inside, stream=None):
    """``wn_query_noalloc``: the mixed query of one domain with no memory
    allocation by the library (device tensors only, at most
    NOALLOC_MAX_QUERIES points).  Returns the status code."""
    return int(lib().wn_query_noalloc(domain.handle, _ptr(points), int(points.shape[0]),
                                      _ptr(out_winding), _ptr(out_inside), _stream(stream)))


def query_batched(domains, points, offsets, precision=MIXED, out_winding=None, out_inside=None,
                  stream=None):
    """Many domains in one call: domain d owns points[offsets[d]:offsets[d+1]]."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    n = int(off[-1])
    arr = (ctypes.c_void_p * len(domains))(*[d.handle.value for d in domains])
    if out_winding is None or out_inside is None:
        if isinstance(points, np.ndarray):
            out_winding = np.empty(n) if out_winding is None else out_winding
            out_inside = np.empty(n, dtype=np.uint8) if out_inside is None else out_inside
        else:
            import torch
            out_winding = torch.empty(n, dtype=torch.float64, device=points.device) if out_winding is None else out_winding
            out_inside = torch.empty(n, dtype=torch.uint8, device=points.device) if out_inside is None else out_inside
    _check(lib().wn_query_batched(ctypes.cast(arr, ctypes.c_void_p), len(domains), _ptr(off),
                                  _ptr(points), _ptr(out_winding), _ptr(out_inside),
                                  int(precision), _stream(stream)))
    return out_winding, out_inside


def query_grid_bitmask(domain, nu, nv, precision=MIXED, stream=None, out_bits=None, out_boundary=None):
    """Inside/boundary bitmask of the nu x nv cell-centre grid (device);
    returns (bits, boundary count), into the given buffers when passed."""
    import torch
    words = (nu * nv + 31) // 32
    bits = torch.empty(words, dtype=torch.int32, device="cuda") if out_bits is None else out_bits
    nb = torch.zeros(1, dtype=torch.int64, device="cuda") if out_boundary is None else out_boundary
    _check(lib().wn_query_grid_bitmask(domain.handle, int(nu), int(nv), _ptr(bits), _ptr(nb),
                                       int(precision), _stream(stream)))
    return bits, nb


def grid_triangles(bits, nu, nv, wrap_u=False, wrap_v=False, capacity=None, stream=None):
    """Kept triangles of a classified cell-centre grid (``bits`` from
    query_grid_bitmask): (T, 3) int32 device tensor of vertex indices."""
    import torch
    if capacity is None:
        qu = nu if wrap_u else nu - 1
        qv = nv if wrap_v else nv - 1
        capacity = 2 * max(qu, 0) * max(qv, 0)
    tris = torch.empty((max(capacity, 1), 3), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check(lib().wn_grid_triangles(_ptr(bits), int(nu), int(nv), 1 if wrap_u else 0, 1 if wrap_v else 0,
                                   _ptr(tris), int(capacity), _ptr(cnt), _stream(stream)))
    n = int(cnt.item())
    if n > capacity:
        raise RuntimeError(f"{n} triangles, capacity {capacity}")
    return tris[:n]


def query_surfaces(faces_by_surface, points, point_offsets, precision=MIXED, stream=None):
    """Inside flags (u8 device tensor) of points sampled on several surfaces,
    each tested against every face of its surface (OR)."""
    import torch
    faces = [f for group in faces_by_surface for f in group]
    sf = np.concatenate([[0], np.cumsum([len(g) for g in faces_by_surface])]).astype(np.int32)
    off = np.ascontiguousarray(point_offsets, dtype=np.int64)
    arr = (ctypes.c_void_p * max(len(faces), 1))(*[f.handle.value for f in faces])
    out = torch.empty(int(off[-1]), dtype=torch.uint8, device="cuda")
    _check(lib().wn_query_surfaces(ctypes.cast(arr, ctypes.c_void_p), _ptr(sf), len(faces_by_surface), _ptr(off),
                                   _ptr(points), _ptr(out), int(precision), _stream(stream)))
    return out


def query_midpoints(domain, pieces, precision=MIXED, stream=None):
    """States (u8 device tensor) of the midpoints of pieces ((n, 4) float64
    device tensor: ax, ay, bx, by)."""
    import torch
    out = torch.empty(int(pieces.shape[0]), dtype=torch.uint8, device="cuda")
    _check(lib().wn_query_midpoints(domain.handle, _ptr(pieces), int(pieces.shape[0]), _ptr(out), int(precision),
                                    _stream(stream)))
    return out


def autotune(domains, points, offsets, iterations=3, stream=None):
    """Time candidate launch shapes on this batch (device points) and keep
    the fastest; returns (best ms per call, tuning dict)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    arr = (ctypes.c_void_p * len(domains))(*[d.handle.value for d in domains])
    ms = np.zeros(1)
    _check(lib().wn_autotune(ctypes.cast(arr, ctypes.c_void_p), len(domains), _ptr(off), _ptr(points),
                             int(iterations), _ptr(ms), _stream(stream)))
    return float(ms[0]), get_tuning()


TUNING = ("qpt", "sweep_ctas_per_sm", "near_ctas_per_sm", "use_graph", "tree", "cell_q", "bucket",
          "near_depth", "near_chunk", "near_refill", "flat_max", "grid_tile_w")


def get_tuning():
    t = np.zeros(len(TUNING), dtype=np.int32)
    _check(lib().wn_get_tuning(_ptr(t), len(TUNING)))
    return dict(zip(TUNING, t.tolist()))


def set_near_tuning(depth_cap=0, chunk=0, refill=0):
    """FP32 near-walk depth cap (12..30), pairs drawn per atomic (multiple of
    32 in 32..1024) and refill threshold (1..32); 0 keeps a value."""
    _check(lib().wn_set_near_tuning(int(depth_cap), int(chunk), int(refill)))


def set_flat_records(max_records):
    """Planar domains with at most max_records records take the flat sweep
    (0: none)."""
    _check(lib().wn_set_flat_records(int(max_records)))


def set_grid_tile(width):
    """Grid queries: tiles of 64 cells, `width` (8, 16, 32, 64) wide."""
    _check(lib().wn_set_grid_tile(int(width)))


def set_queue_limits(near_pairs=0, fp64_pairs=0):
    """Test hook: cap the near-pair and FP64-pair queues (0 = no cap)."""
    _check(lib().wn_set_queue_limits(int(near_pairs), int(fp64_pairs)))


def set_tuning(qpt=0, sweep_ctas_per_sm=0, near_ctas_per_sm=0, use_graph=-1, tree=-1, bucket=-1):
    _check(lib().wn_set_tuning(int(qpt), int(sweep_ctas_per_sm), int(near_ctas_per_sm), int(use_graph),
                               int(tree), int(bucket)))


def eval_gap_angle(y, x, stream=None):
    """The mixed path's FP32 gap angle of (x, y) (device float32 tensors)."""
    import torch
    out = torch.empty_like(x)
    _check(lib().wn_eval_gap_angle(_ptr(y), _ptr(x), _ptr(out), int(x.numel()), _stream(stream)))
    return out


def rational_bounds(control_points, weights):
    """App. A.1's bounds of |gamma'| the walks use for one rational segment
    (host only): numpy [B, B_0, ..., B_7], B over the whole segment and B_j
    over its eighth [j/8, (j+1)/8]."""
    cp = np.ascontiguousarray(control_points, dtype=np.float64).reshape(-1, 2)
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    if len(w) != len(cp):
        raise ValueError("one weight per control point")
    out = np.zeros(9)
    _check(lib().wn_rational_bounds(_ptr(cp), _ptr(w), len(cp) - 1, _ptr(out)))
    return out


def last_escalated(capacity=1 << 22):
    """Query indices the last mixed call recomputed in FP64 (numpy int64)."""
    out = np.zeros(max(int(capacity), 1), dtype=np.int64)
    n = np.zeros(1, dtype=np.int64)
    _check(lib().wn_last_escalated(_ptr(out), int(capacity), _ptr(n)))
    return out[:min(int(n[0]), int(capacity))]


def stats():
    s = WnStats()
    _check(lib().wn_get_stats(ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in WnStats._fields_}


KERNELS = ("bucket", "sweep", "near_fp32", "pairs_fp64", "finalize", "queries_fp64")


def set_profiling(on=True):
    _check(lib().wn_set_profiling(1 if on else 0))


def kernel_times():
    """Summed device milliseconds per mixed-path kernel since the last read,
    and the number of calls they cover."""
    ms = np.zeros(len(KERNELS))
    n = np.zeros(1, dtype=np.int64)
    _check(lib().wn_kernel_times(_ptr(ms), _ptr(n)))
    return dict(zip(KERNELS, ms.tolist())), int(n[0])


WORK = ("node_tests", "telescoped_nodes", "expansions", "expansion_terms", "record_tests_near",
        "record_tests_far", "record_tests_cross", "exact_fp64", "ellipse_tests",
        "box_tests", "warp_node_visits", "warp_record_iterations")


def set_work_counting(on=True):
    """Run the counting build of the tree sweep in the following mixed calls."""
    _check(lib().wn_set_work_counting(1 if on else 0))


def sweep_work():
    """Work tallies of the tree sweep since the last read (see WORK)."""
    c = np.zeros(len(WORK), dtype=np.int64)
    _check(lib().wn_sweep_work(_ptr(c), len(WORK)))
    return dict(zip(WORK, c.tolist()))


NEAR_WORK = ("near_nodes", "near_far", "near_evals", "near_eval_degrees")


def near_work():
    """Work tallies of the FP32 near walk since the last read (see NEAR_WORK)."""
    c = np.zeros(len(NEAR_WORK), dtype=np.int64)
    _check(lib().wn_near_work(_ptr(c)))
    return dict(zip(NEAR_WORK, c.tolist()))


def version():
    return lib().wn_version().decode()
