"""Host logic of bench.py (CPU only): the oracle samples cover what they
claim, the parity count separates mismatches from oracle ties and leaves
boundary points out of the winding error, and the kernel-code hash that
keeps a DRAM-traffic capture valid ignores comments but not code."""
import os
import shutil

import numpy as np

import bench


def test_proportional_sample():
    rng = np.random.default_rng(1)
    qs = [np.zeros((n, 2)) for n in (5, 0, 1000, 37, 20000)]
    picks = bench.proportional_sample(qs, 4000, rng)
    assert sum(len(p) for p in picks) == 4000
    for q, p in zip(qs, picks):
        assert np.all((p >= 0) & (p < len(q)))
        assert len(np.unique(p)) == len(p)
    # in proportion to the domains' sizes (binomial spread)
    assert abs(len(picks[4]) - 4000 * 20000 / 21042) < 6 * np.sqrt(4000 * 0.05)
    # a sample larger than the workload takes every query once
    allp = bench.proportional_sample(qs, 10 ** 9, rng)
    assert [len(p) for p in allp] == [len(q) for q in qs]


def test_stratified_sample():
    rng = np.random.default_rng(2)
    qs = [np.zeros((n, 2)) for n in (3, 50, 100000)]
    picks = bench.stratified_sample(qs, 20, rng)
    assert [len(p) for p in picks] == [3, 20, 20]
    for q, p in zip(qs, picks):
        assert np.all(np.diff(p) > 0) and p[-1] < len(q)


def test_grid_sample():
    rng = np.random.default_rng(3)
    G = 4096
    for cells in bench.grid_sample(4, G, rng, 1000):
        assert np.all((cells >= 0) & (cells < G * G))
        assert len(np.unique(cells)) == len(cells)
        rows = cells // G
        # one cell per block of rows: every eighth of the rows is visited
        assert len(np.unique(rows * 8 // G)) == 8


def test_parity_check_counts():
    doms = [{"cps": np.array([[0.0, 0.0], [1.0, 1.0]]), "period_u": 0.0, "period_v": 0.0}]
    idx = np.arange(6)
    ow = np.array([0.0, 1.0, 0.25, np.nan, 0.7, 0.2])
    osd = np.array([0, 1, 0, 2, 1, 0], dtype=np.uint8)
    om = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1e-14])          # the last query is an oracle tie
    w = ow.copy()
    s = osd.copy()
    w[2] += 3e-7                                              # a winding difference off the boundary
    s[4] = 0                                                  # a state mismatch
    s[5] = 1                                                  # a difference inside the tie margin
    w[3] = 12.0                                               # boundary on both sides: no winding check
    r = bench.parity_check(doms, {0: (idx, ow, osd, om)}, w, s, np.array([0, 6]))
    assert r["oracle_mismatches"] == 1 and r["ties"] == 1 and r["checked"] == 6
    assert abs(r["max_abs_domega"] - 3e-7) < 1e-15


def test_kernel_sha_ignores_comments(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2510_25159_gb300", "csrc")
    dst = tmp_path / "paper_2510_25159_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("wn_kernels.cu", "wn_dev.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_sha()
    k = dst / "wn_kernels.cu"
    text = k.read_text()
    k.write_text("// a comment line\n/* and a block\n   comment */\n" + text.replace("\n", "\n\n", 3))
    assert bench._kernel_sha() == h0
    k.write_text(text.replace("kChunk = 64", "kChunk = 32", 1))
    assert bench._kernel_sha() != h0
