"""Triangles of a trimmed cell-centre grid (test infrastructure only).

The tessellation application of Sec. 5.4.3 samples a uniform grid in the
parameter domain, triangulates it and drops the triangles outside the
trimmed region.  This is the plain definition the GPU emitter must match
exactly: vertices are the cell centres, vertex (i, j) has index j*nu + i;
the quad with lower-left vertex (i, j) has corners a = (i, j),
b = (i+1, j), c = (i, j+1), d = (i+1, j+1) (indices taken modulo nu / nv on
a wrapped axis, whose seam quads then exist as well); its triangles are
(a, b, d) and then (a, d, c), counter-clockwise in (u, v); a triangle is kept
when its three vertices are inside (state INSIDE or BOUNDARY).  Quads are
visited row by row (j outer, i inner).
"""
from __future__ import annotations

import numpy as np


def grid_triangles(inside, nu, nv, wrap_u=False, wrap_v=False):
    """(T, 3) int32 vertex indices of the kept triangles, in emission order."""
    inside = np.asarray(inside).reshape(-1).astype(bool)
    assert inside.size == nu * nv
    qu = nu if wrap_u else nu - 1
    qv = nv if wrap_v else nv - 1
    out = []
    for j in range(max(qv, 0)):
        for i in range(max(qu, 0)):
            i1, j1 = (i + 1) % nu, (j + 1) % nv
            a, b, c, d = j * nu + i, j * nu + i1, j1 * nu + i, j1 * nu + i1
            if inside[a] and inside[b] and inside[d]:
                out.append((a, b, d))
            if inside[a] and inside[d] and inside[c]:
                out.append((a, d, c))
    return np.asarray(out, dtype=np.int32).reshape(-1, 3)
