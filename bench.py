#!/usr/bin/env python3
"""Containment-query benchmark (one JSON line on rank 0).

Default workload (4): a batched B-Rep-shaped job of 10,000 faces -- segments
per face log-normal (median 40, 4..4000), degrees 1-5, 20% periodic (half
cylinders, half tori), queries per face log-normal (median 4096, 16..1M),
about 2.0e8 queries -- classified in one batched call of the mixed FP32 +
FP64-fallback path, autotuned and replayed from a captured CUDA graph.  A
step is one such call over the whole batch with the queries already in HBM
(3.2 GB of points, far larger than L2; L2 is also flushed between steps
outside the timed events).

Also reported: e2e (the same call with host buffers, copies included); the
plain FP64 path on the same GPU (one launch per face); the mixed path with
the flat sweep instead of the record tree (so that "x plain" splits into the
precision pattern's gain and the path hierarchy's); per-kernel times from an
untimed profiling pass with direct launches; the roofline of the dominant
kernel (the sweep) on the algorithmic FP32 work of the method, counted per
unit as the recursion's own steps (far test 7, chord 27, evaluation 4n+4),
next to the implementation's own operation count; the FP64 oracle on the
host cores (all cores and one thread, a bounded sample, which doubles as a
parity check of the timed results); and the SM clocks seen during the timed
region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload 1..6] [--scale F]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import wn_synth as ws  # noqa: E402

METRIC = "containment queries/s, batched FP32+FP64-fallback vs plain, 0 oracle mismatches"
UNIT = "queries/s"
DEFAULT_WORKLOAD = 4
FP32_LANES_PER_SM = 128

# Algorithmic FP32 work of the method, counted by convention (add/sub/mul/
# compare 1, FMA 2, square root 1, atan2 20), per unit of the recursion:
#   far test of a (sub-)segment or sub-path against its ellipse (Eq. 5): 7
#   chord of a far (sub-)segment or sub-path (Eq. 3): 27
#   evaluation of gamma(m) of a degree-n segment: 4n + 4
FAR_TEST, CHORD = 7.0, 27.0
# The record tree's tallies mapped to those units (wn_sweep_work): a node
# test is a sub-path's far test; a telescoped node and an expansion sum are
# an accepted sub-path's chord; a leaf record test is a segment's far test
# and, unless it became a near pair, its chord.
S8D_PER_TALLY = {"node_tests": FAR_TEST, "telescoped_nodes": CHORD, "expansions": CHORD,
                 "record_tests_near": FAR_TEST + CHORD, "record_tests_far": FAR_TEST + CHORD,
                 "record_tests_cross": FAR_TEST + CHORD}
# The operations the sweep kernel itself performs per tally (a second,
# labelled figure, not the roofline's):
#   node test: near-box test 8, ray-extent test 6, expansion distance and
#     series-length choice 14, right-of-p test 2
#   telescoped node: two end signs and their bands 8
#   expansion sum: w = r_c/(z_c - p) 12, Horner step 8 per term, Im part 3,
#     compensated add 6
#   record test with the near check: circle test 6 + end signs and their
#     bands 8 + the gap: next-vertex sign and band 3, hi/lo gap ends 8,
#     choice of the shorter cross-product operand 6, cross and dot products
#     6, gap angle by the odd series 18 (6 FMA + divide), accumulation 5
#     = 60 (the chord crossings, taken only on a sign change, not counted)
#   record test with crossings and gap angle: the same without the circle
#     test, 54; with crossings only: 20
#   ellipse test inside a record's circle 16; control-point box test 21
IMPL_FLOPS = {"node_tests": 30.0, "telescoped_nodes": 8.0, "expansions": 21.0, "expansion_terms": 8.0,
              "record_tests_near": 60.0, "record_tests_far": 54.0, "record_tests_cross": 20.0,
              "exact_fp64": 0.0, "ellipse_tests": 16.0, "box_tests": 21.0}

SHARD_SEED_STRIDE = 1000


def workload(k, scale=1.0, shard=0):
    """Faces and queries of workload k.  Shard r (one per rank) draws its own
    faces and queries (seed offset r * SHARD_SEED_STRIDE; the tessellation
    workload takes faces 64r..64r+63): the ranks' problems are independent,
    as the faces of a B-Rep are."""
    off = SHARD_SEED_STRIDE * shard
    tag = f" (shard {shard})" if shard else ""
    at = f" at {scale:g} of its queries" if scale != 1.0 else ""
    if k == 1:
        d, q = ws.config1(seed_index=1 + off)
        return [d], [q], ("one planar [0,1]^2 domain: 64-cubic CCW star (C0) + two 16-cubic CW holes; "
                          "100k uniform + 10k near (1e-6) queries" + tag)
    if k == 2:
        d, q = ws.config2(n_uniform=int(10_000_000 * scale), n_near=int(1_000_000 * scale), seed_index=2 + off)
        return d, q, ("64 planar domains, 4-12 loops x 32-512 segments of degree 1-5, every join opened by a "
                      "1e-4..1e-2 gap, control-point noise 1e-4; 10M uniform + 1M near-curve (1e-7..1e-3) queries"
                      + at + tag)
    if k == 3:
        d, q = ws.config3(seed_index=3 + off, n_queries=int(20_000_000 * scale))
        return d, q, ("256 bi-periodic faces (2pi x 2pi), 2-8 loops of 16-256 cubics, 30% non-contractible pairs, "
                      "10% open; 20M uniform queries" + at + tag)
    if k == 4:
        d, q = ws.config4(seed_index=4 + off, query_scale=scale)
        return d, q, ("10k faces (B-Rep-shaped batch): segments log-normal median 40 in [4, 4000], degree 1-5, "
                      "1-8 loops, 10% cylinders + 10% tori + 80% planar closed; queries log-normal median 4096 "
                      "in [16, 1M], ~2.0e8 total; one batched call, autotuned, CUDA-graph replay" + at + tag)
    if k == 6:
        d, q = ws.config6(seed_index=6 + off, n_uniform=int(10_000_000 * scale), n_near=int(1_000_000 * scale))
        return d, q, ("64 planar domains of rational segments (weights log-uniform in [0.8, 1.25]): workload 2's "
                      "open/noisy star loops plus two exact rational-arc circles per face; 10M uniform + 1M "
                      "near-curve queries" + at + tag)
    if k == 5:
        d = [ws.config5_face(64 * shard + f) for f in range(64)]
        return d, None, ("64 planar faces of ~100k cubics (fractal outer loop + 200 holes), 4096x4096 "
                         "cell-centre grids, inside/boundary bitmask" + tag)
    raise SystemExit(f"unknown workload {k}")


def reduce_over_ranks(dist, ms, n_q, device):
    """(slowest rank's milliseconds, all ranks' queries): the whole-job
    figures of a weak-scaling run, each rank on its own shard."""
    if dist is None:
        return ms, n_q
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q = torch.tensor([n_q], dtype=torch.int64, device=device)
    dist.all_reduce(q, op=dist.ReduceOp.SUM)
    return float(t.item()), int(q.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (the samples go
    to a temporary file that is removed after reading)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        fd, self.path = tempfile.mkstemp(prefix="wn_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        rows = []
        if self.p is not None:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def proportional_sample(qs, n_total, rng):
    """Indices per domain of n_total queries drawn uniformly from all of a
    workload's queries (so each domain appears in proportion to its query
    count)."""
    counts = np.array([len(q) for q in qs], dtype=np.int64)
    tot = int(counts.sum())
    pick = np.sort(rng.choice(tot, size=min(n_total, tot), replace=False))
    starts = np.concatenate([[0], np.cumsum(counts)])
    out = []
    for d in range(len(qs)):
        a, b = np.searchsorted(pick, [starts[d], starts[d + 1]])
        out.append(pick[a:b] - starts[d])
    return out


def stratified_sample(qs, per_domain, rng):
    """Indices per domain: per_domain queries of every domain (all of a
    smaller one), so every face -- the largest ones included -- is checked."""
    return [np.sort(rng.choice(len(q), min(per_domain, len(q)), replace=False)) for q in qs]


def oracle_run(doms, qs, picks, threads, budget_s=None):
    """The FP64 oracle on the picked queries of each domain, on `threads`
    host threads: a domain with many picked queries splits them over the
    oracle's own threads, the others run one domain per thread (larger
    samples first).  Stops taking new domains after budget_s seconds when
    given.  Returns ({domain: (idx, w, state, margin)}, queries done,
    seconds)."""
    import concurrent.futures as cf

    import oracle
    res = {}
    order = sorted((d for d in range(len(doms)) if len(picks[d])), key=lambda d: -len(picks[d]))
    big = [d for d in order if len(picks[d]) >= 256 * threads] if threads > 1 else []
    small = [d for d in order if d not in set(big)]
    t0 = time.perf_counter()

    def one(d, th):
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            return
        w, s, mg = oracle.query(doms[d], qs[d][picks[d]], threads=th, margins=True)
        res[d] = (picks[d], w, s, mg)

    for d in big:
        one(d, threads)
    if threads > 1:
        with cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda d: one(d, 1), small))
    else:
        for d in small:
            one(d, 1)
    dt = time.perf_counter() - t0
    return res, sum(len(v[0]) for v in res.values()), dt


def calibrate_oracle(doms, qs, threads, rng, budget_s):
    """Size of a proportional sample that takes about budget_s seconds."""
    picks = proportional_sample(qs, 2000, rng)
    _, n, dt = oracle_run(doms, qs, picks, threads)
    return int(np.clip(budget_s * n / max(dt, 1e-3), 1000, 5_000_000))


def parity_check(doms, res, w_all, s_all, off):
    """States must match the oracle's except its ties (decision margin below
    1e-12 of the domain scale); the largest |omega difference| over the
    points neither side puts on the boundary."""
    mism, ties, maxerr, n = 0, 0, 0.0, 0
    for d, (i, ow, osd, om) in res.items():
        w = w_all[off[d] + i]
        s = s_all[off[d] + i]
        cp = doms[d]["cps"]
        S = max(1.0, doms[d]["period_u"], doms[d]["period_v"], float(np.ptp(cp[:, 0])), float(np.ptp(cp[:, 1])))
        tie = om < 1e-12 * S
        mism += int(((s != osd) & ~tie).sum())
        ties += int(((s != osd) & tie).sum())
        ok = (s != 2) & (osd != 2)
        if ok.any():
            maxerr = max(maxerr, float(np.max(np.abs(w[ok] - ow[ok]))))
        n += len(i)
    return {"oracle_mismatches": mism, "ties": ties, "max_abs_domega": maxerr, "checked": n,
            "domains_checked": len(res)}


def grid_sample(n_faces, G, rng, n_per_face):
    """Seeded cell indices of a G x G grid per face (a stratified sample:
    one uniform cell in each of n_per_face equal blocks of rows)."""
    out = []
    for _ in range(n_faces):
        rows = (np.arange(n_per_face) * G) // n_per_face + rng.integers(0, max(1, G // n_per_face), n_per_face)
        rows = np.minimum(rows, G - 1)
        cols = rng.integers(0, G, n_per_face)
        out.append(np.unique(rows.astype(np.int64) * G + cols))
    return out


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, each step a bounded proportional
    sample of the same workload (the reference arm of this benchmark)."""
    if rank != 0:
        return
    import oracle
    doms, qs, desc = workload(args.workload, args.scale)
    if qs is None:
        G = 4096
        qs = [ws.grid_points(G, G)[i] for i in grid_sample(len(doms), G, np.random.default_rng(5), 4096)]
    threads = os.cpu_count() or 1
    oracle.build()
    rng = np.random.default_rng(12345)
    per_step = min(10.0, 150.0 / max(1, args.steps + args.warmup))
    m = calibrate_oracle(doms, qs, threads, rng, per_step)
    tn, tt = 0, 0.0
    for s in range(args.warmup + args.steps):
        _, n, dt = oracle_run(doms, qs, proportional_sample(qs, m, rng), threads)
        if s >= args.warmup:
            tn += n
            tt += dt
    value = tn / tt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": desc},
           "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": threads,
                            "cpu_model": cpu_model(),
                            "sample": f"{tn // max(1, args.steps)} queries per step drawn uniformly from all "
                                      f"of the workload's queries"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _kernel_sha():
    """Hash of the kernels' code (wn_kernels.cu, wn_dev.cuh) with comments
    and whitespace removed: a capture of the kernels' counters stays valid
    until their code changes."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in ("wn_kernels.cu", "wn_dev.cuh"):
        src = open(os.path.join(ROOT, "paper_2510_25159_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=DEFAULT_WORKLOAD)
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the queries (profiling cases)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of all-core oracle work")
    ap.add_argument("--grid-sample", type=int, default=1 << 14,
                    help="workload 5: stratified cells checked by the oracle (all faces together)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-flat", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--qpt", type=int, default=0, help="queries per sweep thread (profiling cases; 0: tuned)")
    ap.add_argument("--ctas", type=int, default=0, help="sweep CTAs per SM (profiling cases; 0: tuned)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2510_25159_gb300 as wn
    from paper_2510_25159_gb300 import build as wb

    wb.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    doms, qs, desc = workload(args.workload, args.scale, shard=rank)
    handles = [wn.Domain.from_dict(d) for d in doms]
    dev = torch.device("cuda", local)
    grid = qs is None
    G = 4096
    if not grid:
        pts_h = np.ascontiguousarray(np.concatenate(qs, axis=0))
        off = np.concatenate([[0], np.cumsum([len(x) for x in qs])]).astype(np.int64)
        n_q = int(off[-1])
        pts = torch.from_numpy(pts_h).to(dev)
        out_w = torch.empty(n_q, dtype=torch.float64, device=dev)
        out_s = torch.empty(n_q, dtype=torch.uint8, device=dev)
        seg = np.array([ws.n_segments(d) for d in doms], dtype=np.float64)
        pairs = float(np.sum(seg * np.diff(off)))
    else:
        n_q = len(doms) * G * G
        pairs = float(sum(ws.n_segments(d) for d in doms)) * G * G
        bits = [torch.empty((G * G + 31) // 32, dtype=torch.int32, device=dev) for _ in doms]
        nbnd = torch.zeros(len(doms), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)          # a non-default stream, so calls can replay a graph
    torch.cuda.set_stream(stream)
    if not grid and not args.no_autotune:
        wn.autotune(handles, pts, off, iterations=2, stream=stream)
    if args.qpt or args.ctas:
        wn.set_tuning(qpt=args.qpt, sweep_ctas_per_sm=args.ctas)

    def step(prec=wn.MIXED):
        if grid:
            for f, h in enumerate(handles):
                wn.query_grid_bitmask(h, G, G, precision=prec, out_bits=bits[f], out_boundary=nbnd[f:f + 1])
        else:
            wn.query_batched(handles, pts, off, precision=prec, out_winding=out_w, out_inside=out_s)

    # the timed region replays the captured CUDA graph of the batched call
    wn.set_tuning(use_graph=0 if args.no_graph else 1)
    tuning = wn.get_tuning()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    st = wn.stats()
    clocks = clk.summary()
    ms, n_all = reduce_over_ranks(dist, ms, n_q, dev)
    value = n_all / (ms / 1e3)
    launches_per_step = int(st["kernels"]) * (len(handles) if grid else 1)
    escalated = None
    if grid:
        # the cells each face's last (timed) call recomputed in FP64
        escalated = []
        for f, h in enumerate(handles):
            wn.query_grid_bitmask(h, G, G, out_bits=bits[f], out_boundary=nbnd[f:f + 1])
            escalated.append(wn.last_escalated())

    # per-kernel times: an untimed pass with direct launches and CUDA events
    # around each kernel on the launching stream
    wn.set_tuning(use_graph=0)
    wn.set_profiling(True)
    n_prof = max(2, min(args.steps, 5))
    for _ in range(n_prof):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ktimes, ncalls = wn.kernel_times()
    wn.set_profiling(False)
    kernel_ms = {k: v / max(1, ncalls) for k, v in ktimes.items()}        # per call
    calls_per_step = ncalls / n_prof

    # algorithmic work: one more step with the counting builds of the sweep
    # and the near walk (same decisions, so the same work as each timed step)
    wn.set_work_counting(True)
    near_pairs = 0
    if grid:
        for f, h in enumerate(handles):
            wn.query_grid_bitmask(h, G, G, out_bits=bits[f], out_boundary=nbnd[f:f + 1])
            torch.cuda.synchronize()
            near_pairs += wn.stats()["near_pairs"]
    else:
        step()
        torch.cuda.synchronize()
        near_pairs = wn.stats()["near_pairs"]
    work = wn.sweep_work()
    nwork = wn.near_work()
    wn.set_work_counting(False)

    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * f_max * 1e6 / 1e12
    f_run = clocks.get("sm_mhz") or f_max
    peak_run = n_sm * FP32_LANES_PER_SM * 2 * f_run * 1e6 / 1e12
    sweep_ms = kernel_ms["sweep"] * calls_per_step            # per step
    near_ms = kernel_ms["near_fp32"] * calls_per_step
    # a record that became a near pair takes no chord in the sweep (its
    # chords are the near walk's)
    s8d_sweep = sum(S8D_PER_TALLY.get(k, 0.0) * v for k, v in work.items()) - CHORD * near_pairs
    s8d_near = (FAR_TEST * nwork["near_nodes"] + CHORD * nwork["near_far"] +
                4.0 * nwork["near_eval_degrees"] + 4.0 * nwork["near_evals"])
    impl_sweep = sum(IMPL_FLOPS.get(k, 0.0) * v for k, v in work.items())
    # SIMT efficiency of the tree walk: query-slot tests over the slots the
    # warps' visits and record iterations offer (32 x queries per thread)
    slots = 32 * int(tuning.get("qpt", 1))
    simt = {"nodes": work["node_tests"] / max(1, slots * work.get("warp_node_visits", 0)),
            "records": (work["record_tests_near"] + work["record_tests_far"] + work["record_tests_cross"]) /
                       max(1, slots * work.get("warp_record_iterations", 0))}
    achieved = s8d_sweep / (sweep_ms / 1e3) / 1e12 if sweep_ms > 0 else None
    traffic = None
    tf = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if os.path.exists(tf):
        try:
            t = json.load(open(tf))
            if t.get("workload") == args.workload and t.get("kernel_source_sha") == _kernel_sha():
                traffic = t.get("bytes_per_launch")
        except Exception:
            traffic = None
    roof = {"bound": "alu", "kernel": "k_sweep_tree", "achieved": achieved, "peak": peak_tflops,
            "unit": "TFLOP/s", "frac": (achieved / peak_tflops) if achieved else None, "traffic": traffic,
            "peak_basis": f"derived FP32 peak: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {f_max:.0f} MHz "
                          f"(sm_max_mhz of MEASURED_PEAKS.json; no measured FP32 figure there)",
            "frac_at_run_clock": (achieved / peak_run) if achieved else None,
            "work_basis": "far test 7 per node or record, chord 27 per accepted node (telescoped or expanded) "
                          "and per record that is not a near pair, 4n+4 per near evaluation",
            "algorithmic_flops_per_step": s8d_sweep, "work_per_step": work,
            "near_kernel": {"algorithmic_flops_per_step": s8d_near, "ms_per_step": near_ms,
                            "tflops": s8d_near / (near_ms / 1e3) / 1e12 if near_ms > 0 else None,
                            "work_per_step": nwork},
            "whole_step_tflops": (s8d_sweep + s8d_near) / (ms / 1e3) / 1e12,
            "implementation_ops": {"flops_per_step": impl_sweep, "per_tally": IMPL_FLOPS,
                                   "tflops": impl_sweep / (sweep_ms / 1e3) / 1e12 if sweep_ms > 0 else None},
            "simt_efficiency": simt,
            "brute_force_pairs_per_step": pairs,
            "kernel_ms_per_step": {k: v * calls_per_step for k, v in kernel_ms.items()}}

    extra = {}
    if grid:
        # tessellation consumer (Sec. 5.4.3): each face's bitmask -> kept
        # triangles of its 4096 x 4096 cell-centre grid, outside the timed
        # region of the metric; CUDA events around the triangle kernels
        import ctypes
        cap = 2 * (G - 1) * (G - 1)
        tri_buf = torch.empty((cap, 3), dtype=torch.int32, device=dev)
        cnt = torch.zeros(len(handles), dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        L = wn.lib()
        tms = []
        for rep in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for f, bt in enumerate(bits):
                rc = L.wn_grid_triangles(ctypes.c_void_p(bt.data_ptr()), G, G, 0, 0,
                                         ctypes.c_void_p(tri_buf.data_ptr()), cap,
                                         ctypes.c_void_p(cnt.data_ptr() + 8 * f), ctypes.c_void_p(stream.cuda_stream))
                assert rc == 0
            b.record(stream)
            torch.cuda.synchronize()
            tms.append(a.elapsed_time(b))
        n_tri = int(cnt.sum().item())
        t_ms = tms[-1]
        tbytes = n_tri * 12 + len(bits) * (G * G // 8)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        extra["tessellation"] = {
            "what": "kept triangles of each face's 4096x4096 cell-centre grid (wn_grid_triangles), all 64 faces",
            "ms": t_ms, "triangles": n_tri, "kernels": 3 * len(bits),
            "roofline": {"bound": "hbm", "achieved": tbytes / (t_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": tbytes / (t_ms / 1e3) / 1e9 / hbm, "algorithmic_bytes": tbytes}}
        del tri_buf

    # the mixed path with the flat sweep (no record tree): the precision
    # pattern alone, against the plain FP64 path
    if not grid and not args.no_flat:
        wn.set_tuning(tree=0)
        step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        fms, _ = reduce_over_ranks(dist, a.elapsed_time(b), n_q, dev)
        wn.set_tuning(tree=1)
        extra["mixed_flat"] = {"value": n_all / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
                               "what": "same mixed FP32 + FP64-fallback path with the flat sweep (every "
                                       "(query, segment) pair, no record tree, no bucketing)"}

    # plain FP64 path on the same GPU (one launch per face); on grids, a
    # seeded sample of one row of cells per face through wn_query
    if not args.no_plain:
        if grid:
            rng_p = np.random.default_rng(99)
            rows = rng_p.integers(0, G, len(handles))
            gp = ws.grid_points(G, G)
            rp = [torch.from_numpy(np.ascontiguousarray(gp[r * G:(r + 1) * G])).to(dev) for r in rows]
            pw = torch.empty(G, dtype=torch.float64, device=dev)
            ps = torch.empty(G, dtype=torch.uint8, device=dev)

            def plain_step():
                for h, p in zip(handles, rp):
                    wn.query(h, p, precision=wn.PLAIN_FP64, out_winding=pw, out_inside=ps)
            n_plain = G * len(handles)
        else:
            def plain_step():
                step(wn.PLAIN_FP64)
            n_plain = n_q
        plain_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        plain_step()
        b.record(stream)
        torch.cuda.synchronize()
        pms, n_plain_all = reduce_over_ranks(dist, a.elapsed_time(b), n_plain, dev)
        prate = n_plain_all / (pms / 1e3)
        extra["plain_fp64"] = {"value": prate, "unit": UNIT, "ms_per_step": pms, "queries": n_plain_all,
                               "launches_per_step": len(handles),
                               "what": ("one seeded row of 4096 cells per face through wn_query, plain FP64"
                                        if grid else "the whole batch, one plain FP64 launch per face")}
        extra["speedup_vs_plain"] = value / prate
        if "mixed_flat" in extra:
            extra["speedup_split"] = {"precision_pattern": extra["mixed_flat"]["value"] / prate,
                                      "path_hierarchy": value / extra["mixed_flat"]["value"]}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not grid and not args.no_e2e:
        hp = torch.from_numpy(pts_h).pin_memory()
        hw = torch.empty(n_q, dtype=torch.float64).pin_memory()
        hs = torch.empty(n_q, dtype=torch.uint8).pin_memory()
        hpn, hwn, hsn = hp.numpy(), hw.numpy(), hs.numpy()
        wn.query_batched(handles, hpn, off, out_winding=hwn, out_inside=hsn)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            wn.query_batched(handles, hpn, off, out_winding=hwn, out_inside=hsn)
        torch.cuda.synchronize()
        et_ms, _ = reduce_over_ranks(dist, (time.perf_counter() - t0) / args.steps * 1e3, n_q, dev)
        e2e = {"value": n_all / (et_ms / 1e3), "unit": UNIT, "ms_per_step": et_ms,
               "h2d_bytes_per_step": int(pts_h.nbytes), "d2h_bytes_per_step": int(n_q * 9)}
    elif grid and not args.no_e2e:
        # host result: every face's bitmask copied to pinned host memory
        hb = [torch.empty(bt.shape, dtype=torch.int32).pin_memory() for bt in bits]
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
            for bt, h in zip(bits, hb):
                h.copy_(bt, non_blocking=True)
        torch.cuda.synchronize()
        et_ms, _ = reduce_over_ranks(dist, (time.perf_counter() - t0) / args.steps * 1e3, n_q, dev)
        e2e = {"value": n_all / (et_ms / 1e3), "unit": UNIT, "ms_per_step": et_ms, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": int(sum(bt.numel() * 4 for bt in bits)),
               "note": "grid points are made on the device from the cell index (no input copy)"}

    # the FP64 oracle on the host cores: bounded samples, which double as a
    # parity check of the timed results (outputs of the last call)
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        rng = np.random.default_rng(12345)
        if not grid:
            w_all = out_w.cpu().numpy()
            s_all = out_s.cpu().numpy()
            m = calibrate_oracle(doms, qs, threads, rng, args.cpu_budget)
            res_p, n_p, dt_p = oracle_run(doms, qs, proportional_sample(qs, m, rng), threads)
            per_dom = int(np.clip(m // max(1, len(doms)), 8, 20000))
            res_s, n_s, dt_s = oracle_run(doms, qs, stratified_sample(qs, per_dom, rng), threads)
            res_1, n_1, dt_1 = oracle_run(doms, qs, proportional_sample(qs, max(1000, m // threads), rng), 1,
                                          budget_s=args.cpu_budget / 2)
            par_p = parity_check(doms, res_p, w_all, s_all, off)
            par_s = parity_check(doms, res_s, w_all, s_all, off)
            big = [d for d in range(len(doms)) if seg[d] >= 1000 or len(qs[d]) >= (1 << 18)]
            parity = {"oracle_mismatches": par_p["oracle_mismatches"] + par_s["oracle_mismatches"],
                      "ties": par_p["ties"] + par_s["ties"],
                      "max_abs_domega": max(par_p["max_abs_domega"], par_s["max_abs_domega"]),
                      "checked": par_p["checked"] + par_s["checked"],
                      "samples": f"{n_p} queries drawn uniformly from all queries + {per_dom} per domain from "
                                 f"every one of the {len(doms)} domains",
                      "large_domains_checked": f"{sum(1 for d in big if d in res_s)} of {len(big)} "
                                               f"(segments >= 1000 or queries >= 2^18)"}
            cpu = {"kind": "oracle", "value": n_p / dt_p, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(),
                   "sample": f"{n_p} queries drawn uniformly from all of the workload's queries, {dt_p:.1f} s",
                   "one_thread": {"value": n_1 / dt_1, "unit": UNIT, "cores": 1,
                                  "sample": f"{n_1} queries drawn uniformly, {dt_1:.1f} s"}}
        else:
            n_face = len(doms)
            per_face = max(1, args.grid_sample // n_face)
            strat = grid_sample(n_face, G, rng, per_face)
            # the cells nearest the curves: next to a change of state in the
            # bitmask (where a wrong decision would show), 1/16 as many
            near_cells = []
            for f in range(n_face):
                b = bits[f].cpu().numpy().view(np.uint32)
                k = np.arange(G * G, dtype=np.int64)
                v = ((b[k >> 5] >> (k & 31).astype(np.uint32)) & 1).reshape(G, G)
                edge = np.zeros_like(v, dtype=bool)
                edge[:, :-1] |= v[:, 1:] != v[:, :-1]
                edge[:-1, :] |= v[1:, :] != v[:-1, :]
                cand = np.flatnonzero(edge)
                near_cells.append(rng.choice(cand, min(len(cand), max(1, per_face // 16)), replace=False)
                                  if len(cand) else cand)
            gp = ws.grid_points(G, G)
            picks = [np.unique(np.concatenate([strat[f], near_cells[f], escalated[f]])) for f in range(n_face)]
            cells = [gp[p] for p in picks]
            res, n_c, dt_c = oracle_run(doms, cells, [np.arange(len(p)) for p in picks], threads)
            mism, ties = 0, 0
            for f, (i, ow, osd, om) in res.items():
                b = bits[f].cpu().numpy().view(np.uint32)
                k = picks[f]
                got = (b[k >> 5] >> (k & 31).astype(np.uint32)) & 1
                tie = om < 1e-12
                bad = got != (osd != 0).astype(np.uint32)
                mism += int((bad & ~tie).sum())
                ties += int((bad & tie).sum())
            n_esc = int(sum(len(e) for e in escalated))
            parity = {"oracle_mismatches": mism, "ties": ties, "checked": n_c,
                      "samples": f"{sum(len(s) for s in strat)} stratified cells + {n_esc} cells the GPU "
                                 f"recomputed in FP64 + {sum(len(c) for c in near_cells)} cells next to a state "
                                 f"change of the bitmask, over all {n_face} faces",
                      "boundary_cells": int(nbnd.sum().item())}
            cpu = {"kind": "oracle", "value": n_c / dt_c, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(),
                   "sample": f"{n_c} sampled cells of the 64 grids, {dt_c:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": desc, "domains": len(doms), "queries": n_q,
                           "segments": int(sum(ws.n_segments(d) for d in doms)),
                           "l2": ("inputs larger than L2 (16 B per query point)" if not grid else
                                  "outputs 2 MiB per face; points made on the device") +
                                 "; 256 MB L2 flush between timed steps outside the events",
                           "timed": "CUDA-graph replay of the batched call" if not args.no_graph else
                                    "direct launches",
                           "queries_all_ranks": n_all,
                           "parallelism": f"independent shards x{world} (no collective on the data path)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "clocks": clocks, "parity": parity, "tuning": tuning,
                "escalation": {"near_pairs": st["near_pairs"], "fp64_pairs": st["fp64_pairs"],
                               "fp64_queries": st["fp64_queries"], "overflow": st["overflow"],
                               "depth_cap": st["depth_cap"], "note": "last call" + (" (last face)" if grid else "")}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    for h in handles:
        h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
