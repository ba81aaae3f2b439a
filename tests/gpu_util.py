"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and
compare element by element with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle

# mixed path: |omega_gpu - omega_oracle| bound for points the oracle classifies
# (the FP32 sweep keeps only gap angles in floating point; see DESIGN notes)
TOL_MIXED = 1e-5
# plain FP64 path: same recursion and atan2 sums in double precision
TOL_PLAIN = 1e-9
TIE = 1e-12


def domain_scale(dom):
    cp = dom["cps"]
    ext = float(max(np.ptp(cp[:, 0]), np.ptp(cp[:, 1]))) if len(cp) else 0.0
    return max(1.0, dom["period_u"], dom["period_v"], ext)


def compare(dom, pts, w, st, tol, closed=False, threads=None):
    """Assert 0 state mismatches (apart from oracle ties: decision margin
    below 1e-12 * domain scale) and |omega error| <= tol.  Returns stats."""
    ow, osd, om = oracle.query(dom, pts, margins=True, threads=threads)
    S = domain_scale(dom)
    tie = om < TIE * S
    mism = (st != osd) & ~tie
    assert int(mism.sum()) == 0, (
        f"{int(mism.sum())} state mismatches; first: gpu={st[mism][:5]}, oracle={osd[mism][:5]}, "
        f"w_gpu={w[mism][:5]}, w_or={ow[mism][:5]}, margin={om[mism][:5]}, idx={np.nonzero(mism)[0][:5]}")
    ok = (st != 2) & (osd != 2)
    err = float(np.max(np.abs(w[ok] - ow[ok]))) if ok.any() else 0.0
    assert err <= tol, f"max |omega error| {err} > {tol}"
    if closed and ok.any():
        assert np.array_equal(np.round(w[ok]), np.round(ow[ok])), "rounded omega differs"
    return {"n": len(pts), "max_err": err, "ties": int((tie & (st != osd)).sum()),
            "boundary": int((osd == 2).sum())}


def run(wn, doms, qs, precision, host=False):
    """Batched query of the lists (domain dicts, query arrays) through the
    C ABI; returns per-domain (w, st) numpy arrays."""
    import torch
    handles = [wn.Domain.from_dict(d) for d in doms]
    pts = np.ascontiguousarray(np.concatenate(qs, axis=0))
    off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
    if host:
        w, s = wn.query_batched(handles, pts, off, precision=precision)
    else:
        w, s = wn.query_batched(handles, torch.from_numpy(pts).cuda(), off, precision=precision)
        torch.cuda.synchronize()
        w, s = w.cpu().numpy(), s.cpu().numpy()
    for h in handles:
        h.close()
    return [(w[a:b], s[a:b]) for a, b in zip(off[:-1], off[1:])]
