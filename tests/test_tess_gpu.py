"""The grid-triangle emitter (tessellation, Sec. 5.4.3) on the GPU against
the plain definition in oracle.tess, index for index: from the GPU's own
bitmask (pure index work) and from the oracle's states (end to end), on
ragged grids, wrapped (periodic) axes and a short output buffer."""
import numpy as np
import pytest

import wn_synth as ws
from oracle import query
from oracle.tess import grid_triangles

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


def bits_to_bool(bits, n):
    b = bits.cpu().numpy().view(np.uint32)
    k = np.arange(n)
    return ((b[k >> 5] >> (k & 31).astype(np.uint32)) & 1).astype(bool)


@pytest.mark.parametrize("nu,nv", [(1, 9), (2, 2), (8, 8), (203, 61), (200, 137), (4099, 3)])
def test_planar_grid_triangles(wn, nu, nv):
    dom = ws.config5_face(1, levels=8, n_holes=25, hole_segs=24)
    h = wn.Domain.from_dict(dom)
    bits, _ = wn.query_grid_bitmask(h, nu, nv, precision=1)
    tri = wn.grid_triangles(bits, nu, nv).cpu().numpy()
    ins = bits_to_bool(bits, nu * nv)
    assert np.array_equal(tri, grid_triangles(ins, nu, nv))
    if nu * nv <= 30000:
        _, st = query(dom, ws.grid_points(nu, nv))
        assert np.array_equal(tri, grid_triangles(st != 0, nu, nv))
    h.close()


@pytest.mark.parametrize("wu,wv", [(1, 0), (0, 1), (1, 1)])
def test_periodic_grid_triangles(wn, wu, wv):
    doms, _ = ws.config3(n_faces=256, n_queries=256 * 10, face_subset=[5])
    dom = doms[0]
    nu, nv = 96, 77
    h = wn.Domain.from_dict(dom)
    bits, _ = wn.query_grid_bitmask(h, nu, nv, precision=1)
    tri = wn.grid_triangles(bits, nu, nv, wrap_u=bool(wu), wrap_v=bool(wv)).cpu().numpy()
    _, st = query(dom, ws.grid_points(nu, nv) * ws.TWO_PI)
    assert np.array_equal(bits_to_bool(bits, nu * nv), st != 0)
    assert np.array_equal(tri, grid_triangles(st != 0, nu, nv, wrap_u=bool(wu), wrap_v=bool(wv)))
    h.close()


def test_short_buffer_reports_count(wn):
    import torch
    dom = ws.config5_face(2, levels=8, n_holes=25, hole_segs=24)
    nu, nv = 300, 200
    h = wn.Domain.from_dict(dom)
    bits, _ = wn.query_grid_bitmask(h, nu, nv, precision=1)
    full = grid_triangles(bits_to_bool(bits, nu * nv), nu, nv)
    cap = len(full) // 3
    out = torch.full((cap, 3), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    import ctypes
    L = wn.lib()
    rc = L.wn_grid_triangles(ctypes.c_void_p(bits.data_ptr()), nu, nv, 0, 0, ctypes.c_void_p(out.data_ptr()), cap,
                             ctypes.c_void_p(cnt.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == 0 and int(cnt.item()) == len(full)
    assert np.array_equal(out.cpu().numpy(), full[:cap])
    h.close()
