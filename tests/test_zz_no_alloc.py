"""wn_query_noalloc through the C ABI.

This entry point exists for callers that cannot let the library allocate
device memory while they run (code inside an allocator or memory-pool
callback, real-time loops that forbid allocation after start-up, processes
with a fixed device-memory budget): its scratch lives in one fixed device
array of the library image.  Its states must equal wn_query's (mixed
precision) on the same inputs and its windings agree within the mixed
tolerance, on two calls in a row, since the second call finds the first
call's leftovers in the shared array; after the start-up call, a call must
not change the device's free memory.

The file name sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import ctypes

import numpy as np
import pytest

import wn_synth as ws
from tests.gpu_util import TOL_MIXED

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


def _call(wn, h, pts, n, w, s):
    import torch
    return wn.lib().wn_query_noalloc(h.handle, ctypes.c_void_p(pts.data_ptr()), n, ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(s.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _run_noalloc(wn, h, pts):
    import torch
    n = pts.shape[0]
    w = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
    s = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
    rc = _call(wn, h, pts, n, w, s)
    torch.cuda.synchronize()
    return rc, w.cpu().numpy(), s.cpu().numpy()


def test_noalloc_matches_wn_query_twice(wn):
    import torch
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 60000, n_near=64 * 6000, domain_subset=[3, 4])
    sizes = [wn.NOALLOC_MAX_QUERIES, 30001]        # the maximum, then a ragged smaller call
    for dom, q, n in zip(doms, qs, sizes):
        h = wn.Domain.from_dict(dom)
        pts = torch.from_numpy(np.ascontiguousarray(q[:n])).cuda()
        w_ref, s_ref = wn.query(h, pts, precision=wn.MIXED)
        torch.cuda.synchronize()
        w_ref, s_ref = w_ref.cpu().numpy(), s_ref.cpu().numpy()
        rc, w, s = _run_noalloc(wn, h, pts)
        assert rc == 0
        assert np.array_equal(s, s_ref)
        ok = s_ref != wn.BOUNDARY
        assert np.max(np.abs(w[ok] - w_ref[ok])) <= TOL_MIXED
        assert np.all(np.isnan(w[~ok]))
        # each query's arithmetic is its own, whatever queries share a warp:
        # the windings are in fact identical
        assert np.array_equal(w, w_ref, equal_nan=True)
        h.close()


def test_noalloc_allocates_nothing_after_startup(wn):
    """A start-up call (n = 0) places the array and the kernels on the
    device; later calls leave the device's free memory unchanged (read with
    cudaMemGetInfo, which sees every allocation, the library's included)."""
    import torch
    doms, qs = ws.config2(n_domains=64, n_uniform=64 * 20000, n_near=64 * 2000, domain_subset=[5])
    h = wn.Domain.from_dict(doms[0])
    n = 20000
    pts = torch.from_numpy(np.ascontiguousarray(qs[0][:n])).cuda()
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.empty(n, dtype=torch.uint8, device="cuda")
    assert _call(wn, h, pts, 0, w, s) == 0            # start-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(wn, h, pts, n, w, s) == 0
        torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    h.close()


def test_noalloc_rejects_oversize(wn):
    import torch
    dom, q = ws.config1(n_uniform=1000, n_near=0)
    h = wn.Domain.from_dict(dom)
    big = torch.zeros((wn.NOALLOC_MAX_QUERIES + 1, 2), dtype=torch.float64, device="cuda")
    rc, _, _ = _run_noalloc(wn, h, big)
    assert rc == 5            # WN_ERR_LIMIT
    h.close()
