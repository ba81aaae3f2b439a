#!/usr/bin/env python3
"""Containment-query benchmark (one JSON line on rank 0).

Default workload: 64 planar domains with open, noisy loops (4-12 loops of
32-512 segments of degree 1-5, gaps 1e-4..1e-2, control-point noise 1e-4),
10M uniform + 1M near-curve queries, classified in one batched call of the
mixed FP32 + FP64-fallback path.  A step is one such call over the whole
batch with the queries already in HBM (176 MB of points, larger than L2; L2
is also flushed between steps outside the timed events).

Also reported: e2e (the same call with host buffers, copies included), the
plain FP64 path on the same GPU (one launch per domain), the sweep kernel's
achieved FP32 rate against the ALU peak, the FP64 oracle on the host cores
(a bounded sample, which doubles as a parity check of the timed results),
and the SM clocks seen during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload 1..6]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import wn_synth as ws  # noqa: E402

METRIC = "containment queries/s, batched FP32+FP64-fallback vs plain, 0 oracle mismatches"
UNIT = "queries/s"
# Algorithmic FP32 work, counted by convention (add/sub/mul/compare 1, FMA 2,
# atan2 20).  A brute-force (query, segment) test: ellipse far test ~7 flops +
# chord angle ~27 flops.
FLOPS_PER_PAIR = 34.0
# Per unit of the tree sweep's work tallies (wn_sweep_work):
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
#     test, 54
#   record test with crossings only: 20
#   ellipse test inside a record's circle: two distances 8 (with the two
#     square roots), focal sum, band and square 4, comparisons 3, chord
#     difference 1 = 16
#   control-point box test inside a record's ellipse: chord vector 2, the two
#     projections 6, band 5, widened bounds 4, comparisons 4 = 21
WORK_FLOPS = {"node_tests": 30.0, "telescoped_nodes": 8.0, "expansions": 21.0, "expansion_terms": 8.0,
              "record_tests_near": 60.0, "record_tests_far": 54.0, "record_tests_cross": 20.0,
              "exact_fp64": 0.0, "ellipse_tests": 16.0, "box_tests": 21.0}
FP32_LANES_PER_SM = 128


SHARD_SEED_STRIDE = 1000


def workload(k, scale=1.0, shard=0):
    """Faces and queries of workload k.  Shard r (one per rank) draws its own
    faces and queries (seed offset r * SHARD_SEED_STRIDE; the tessellation
    workload takes faces 64r..64r+63): the ranks' problems are independent,
    as the faces of a B-Rep are."""
    off = SHARD_SEED_STRIDE * shard
    tag = f" (shard {shard})" if shard else ""
    if k == 2 and scale != 1.0:
        d, q = ws.config2(n_uniform=int(10_000_000 * scale), n_near=int(1_000_000 * scale), seed_index=2 + off)
        return d, q, (f"workload 2 at {scale:g} of its queries (profiling case): 64 planar open/noisy domains, "
                      f"{int(11_000_000 * scale)} queries" + tag)
    if k == 1:
        d, q = ws.config1(seed_index=1 + off)
        return [d], [q], ("one planar [0,1]^2 domain: 64-cubic CCW star (C0) + two 16-cubic CW holes; "
                          "100k uniform + 10k near (1e-6) queries" + tag)
    if k == 2:
        d, q = ws.config2(seed_index=2 + off)
        return d, q, ("64 planar domains, 4-12 loops x 32-512 segments of degree 1-5, every join opened by a "
                      "1e-4..1e-2 gap, control-point noise 1e-4; 10M uniform + 1M near-curve (1e-7..1e-3) queries"
                      + tag)
    if k == 3:
        d, q = ws.config3(seed_index=3 + off, n_queries=int(20_000_000 * scale))
        return d, q, ("256 bi-periodic faces (2pi x 2pi), 2-8 loops of 16-256 cubics, 30% non-contractible pairs, "
                      "10% open; 20M uniform queries" + (f" at {scale:g} of its queries" if scale != 1.0 else "")
                      + tag)
    if k == 4:
        d, q = ws.config4(seed_index=4 + off)
        return d, q, ("10k faces, log-normal segments (median 40) and queries (median 4096, ~2e8 total), "
                      "20% periodic" + tag)
    if k == 6:
        d, q = ws.config6(seed_index=6 + off, n_uniform=int(10_000_000 * scale), n_near=int(1_000_000 * scale))
        return d, q, ("64 planar domains of rational segments (weights log-uniform in [0.8, 1.25]): workload 2's "
                      "open/noisy star loops plus two exact rational-arc circles per face; 10M uniform + 1M "
                      "near-curve queries" + (f" at {scale:g} of its queries" if scale != 1.0 else "") + tag)
    if k == 5:
        d = [ws.config5_face(64 * shard + f) for f in range(64)]
        return d, None, ("64 planar faces of ~100k cubics (fractal outer loop + 200 holes), 4096x4096 "
                         "cell-centre grids" + tag)
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
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def oracle_sample(doms, qs, budget_s, threads):
    """FP64 oracle on a stratified sample of every domain's queries, sized to
    take about budget_s seconds.  Returns (indices per domain, results, rate)."""
    import oracle
    rng = np.random.default_rng(12345)
    # calibrate on 4 queries per domain
    t0 = time.perf_counter()
    for d, q in zip(doms, qs):
        oracle.query(d, q[:4], threads=threads)
    per_q = max((time.perf_counter() - t0) / (4 * len(doms)), 1e-7)
    m = int(np.clip(budget_s * threads / per_q / len(doms), 8, 20000))
    idx, res = [], []
    t0 = time.perf_counter()
    tot = 0
    for d, q in zip(doms, qs):
        i = np.sort(rng.choice(len(q), min(m, len(q)), replace=False))
        w, s, mg = oracle.query(d, q[i], threads=threads, margins=True)
        idx.append(i)
        res.append((w, s, mg))
        tot += len(i)
    dt = time.perf_counter() - t0
    return idx, res, tot / dt, tot, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    doms, qs, desc = workload(args.workload)
    if qs is None:
        qs = [ws.grid_points(4096, 4096)[::4099] for _ in doms]
    threads = os.cpu_count() or 1
    oracle.build()
    times, nq = [], 0
    for _ in range(args.warmup + args.steps):
        _, _, rate, n, dt = oracle_sample(doms, qs, budget_s=min(10.0, 120.0 / max(1, args.steps + args.warmup)),
                                          threads=threads)
        times.append((n, dt))
    tn = sum(n for n, _ in times[args.warmup:])
    tt = sum(dt for _, dt in times[args.warmup:])
    value = tn / tt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": desc},
           "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": threads,
                            "sample": f"{tn // max(1, args.steps)} stratified queries per step over all domains"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--qpt", type=int, default=0)
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the queries (profiling cases)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
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
    if args.qpt:
        wn.set_tuning(qpt=args.qpt)

    doms, qs, desc = workload(args.workload, args.scale, shard=rank)
    handles = [wn.Domain.from_dict(d) for d in doms]
    dev = torch.device("cuda", local)
    grid = qs is None
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
        n_q = 64 * 4096 * 4096
        pairs = float(sum(ws.n_segments(d) for d in doms)) * 4096 * 4096
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)          # a non-default stream, so calls can replay a graph
    torch.cuda.set_stream(stream)
    tuning = None
    if not grid and not args.no_autotune:
        tune_ms, tuning = wn.autotune(handles, pts, off, iterations=2, stream=stream)
    # per-kernel CUDA events in the timed region need direct launches (no graph replay)
    wn.set_tuning(use_graph=0)
    tuning = wn.get_tuning()

    def step(prec=wn.MIXED):
        if grid:
            for h in handles:
                wn.query_grid_bitmask(h, 4096, 4096, precision=prec)
        else:
            wn.query_batched(handles, pts, off, precision=prec, out_winding=out_w, out_inside=out_s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    wn.set_profiling(True)
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
    ktimes, ncalls = wn.kernel_times()
    wn.set_profiling(False)
    st = wn.stats()
    clocks = clk.summary()
    ms, n_all = reduce_over_ranks(dist, ms, n_q, dev)
    value = n_all / (ms / 1e3)
    launches_per_step = int(st["kernels"]) * (len(handles) if grid else 1)

    # roofline of the dominant kernel (the sweep): algorithmic FP32 flops / its event time
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * f_max * 1e6 / 1e12
    sweep_ms = ktimes["sweep"] / max(1, ncalls)               # per sweep launch
    launches_sweep = ncalls / max(1, args.steps)                # sweep launches per step
    # one more step with the counting build of the sweep (outside the timed
    # region; same decisions, so the same work as each timed step)
    wn.set_work_counting(True)
    step()
    torch.cuda.synchronize()
    work = wn.sweep_work()
    wn.set_work_counting(False)
    flops_launch = sum(WORK_FLOPS[k] * v for k, v in work.items()) / max(1.0, launches_sweep)
    achieved = flops_launch / (sweep_ms / 1e3) / 1e12 if sweep_ms > 0 and flops_launch > 0 else None
    brute = pairs / max(1.0, launches_sweep) * FLOPS_PER_PAIR / (sweep_ms / 1e3) / 1e12 if sweep_ms > 0 else None
    traffic = None
    tf = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if os.path.exists(tf):
        try:
            t = json.load(open(tf))
            if t.get("workload") == args.workload and t.get("kernel_source_sha") == _kernel_sha():
                traffic = t.get("bytes_per_launch")
        except Exception:
            traffic = None
    roof = {"bound": "alu", "kernel": "k_sweep_tree", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": (achieved / peak_tflops) if achieved else None, "traffic": traffic,
            "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {f_max:.0f} MHz (sm_max_mhz)",
            "algorithmic_flops_per_launch": flops_launch, "work_per_step": work, "flops_per_unit": WORK_FLOPS,
            "brute_force_equiv": {"tflops": brute, "flops_per_pair": FLOPS_PER_PAIR,
                                  "pairs_per_step": pairs},
            "kernel_ms": {k: v / max(1, ncalls) for k, v in ktimes.items()}}

    extra = {}
    if grid:
        # tessellation consumer (Sec. 5.4.3): each face's bitmask -> kept
        # triangles of its 4096 x 4096 cell-centre grid, outside the timed
        # region of the metric; CUDA events around the triangle kernels
        import ctypes
        G = 4096
        cap = 2 * (G - 1) * (G - 1)
        tri_buf = torch.empty((cap, 3), dtype=torch.int32, device=dev)
        cnt = torch.zeros(len(handles), dtype=torch.int64, device=dev)
        masks = [wn.query_grid_bitmask(h, G, G)[0] for h in handles]
        torch.cuda.synchronize()
        L = wn.lib()
        tms = []
        for rep in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for f, bits in enumerate(masks):
                rc = L.wn_grid_triangles(ctypes.c_void_p(bits.data_ptr()), G, G, 0, 0,
                                         ctypes.c_void_p(tri_buf.data_ptr()), cap,
                                         ctypes.c_void_p(cnt.data_ptr() + 8 * f), ctypes.c_void_p(stream.cuda_stream))
                assert rc == 0
            b.record(stream)
            torch.cuda.synchronize()
            tms.append(a.elapsed_time(b))
        n_tri = int(cnt.sum().item())
        t_ms = tms[-1]
        tbytes = n_tri * 12 + len(masks) * (G * G // 8)
        extra["tessellation"] = {
            "what": "kept triangles of each face's 4096x4096 cell-centre grid (wn_grid_triangles), all 64 faces",
            "ms": t_ms, "triangles": n_tri, "kernels": 3 * len(masks),
            "roofline": {"bound": "hbm", "achieved": tbytes / (t_ms / 1e3) / 1e9,
                         "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                         "frac": tbytes / (t_ms / 1e3) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
                         "algorithmic_bytes": tbytes}}
        del tri_buf, masks
    # plain FP64 path on the same GPU (one launch per domain)
    if not args.no_plain and not grid:
        step(wn.PLAIN_FP64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        step(wn.PLAIN_FP64)
        b.record(stream)
        torch.cuda.synchronize()
        pms, _ = reduce_over_ranks(dist, a.elapsed_time(b), n_q, dev)
        extra["plain_fp64"] = {"value": n_all / (pms / 1e3), "unit": UNIT, "ms_per_step": pms,
                               "launches_per_step": len(handles)}
        extra["speedup_vs_plain"] = pms / ms
        step()
        torch.cuda.synchronize()

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

    # oracle on the host cores: bounded sample, also a parity check of the timed results
    cpu = None
    parity = None
    if rank == 0 and world == 1 and not grid and not args.no_cpu:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        idx, res, rate, tot, dt = oracle_sample(doms, qs, args.cpu_budget, threads)
        w_all = out_w.cpu().numpy()
        s_all = out_s.cpu().numpy()
        mism, ties, maxerr = 0, 0, 0.0
        for d, i, (ow, osd, om), a0 in zip(doms, idx, res, off[:-1]):
            w = w_all[a0 + i]
            s = s_all[a0 + i]
            cp = d["cps"]
            S = max(1.0, d["period_u"], d["period_v"], float(np.ptp(cp[:, 0])), float(np.ptp(cp[:, 1])))
            tie = om < 1e-12 * S
            mism += int(((s != osd) & ~tie).sum())
            ties += int(((s != osd) & tie).sum())
            ok = (s != 2) & (osd != 2)
            if ok.any():
                maxerr = max(maxerr, float(np.max(np.abs(w[ok] - ow[ok]))))
        cpu = {"kind": "oracle", "value": rate, "unit": UNIT, "cores": threads,
               "sample": f"{tot} stratified queries ({tot // len(doms)} per domain) of the same workload, {dt:.1f} s"}
        parity = {"oracle_mismatches": mism, "ties": ties, "max_abs_domega": maxerr, "checked": tot}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": desc, "domains": len(doms), "queries": n_q,
                           "segments": int(sum(ws.n_segments(d) for d in doms)),
                           "l2": "inputs (16 B/query) larger than L2; 256 MB L2 flush between steps outside the events",
                           "queries_all_ranks": n_all,
                           "parallelism": f"independent shards x{world} (no collective on the data path)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "clocks": clocks, "parity": parity, "tuning": tuning,
                "escalation": {"near_pairs": st["near_pairs"], "fp64_pairs": st["fp64_pairs"],
                               "fp64_queries": st["fp64_queries"], "overflow": st["overflow"]}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    for h in handles:
        h.close()
    if dist:
        dist.destroy_process_group()


def _kernel_sha():
    import hashlib
    h = hashlib.sha1()
    for f in ("wn_kernels.cu", "wn_dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2510_25159_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    main()
