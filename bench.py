#!/usr/bin/env python3
"""Benchmark of the CCD hot path: one step = boxes + broad phase + earliest-TOI
narrow phase (Algorithm 1) over the folded-cloth self-contact scene, 512 x 512
vertices (262,144 V, 784,385 E, 522,242 F, 1,568,771 boxes), delta = 1e-6,
min_sep = 0, max_iter = 1e6, synthetic seeded input.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is CCD queries per second of the
whole job: narrow-phase candidate pairs of every rank / max-over-ranks step
time.  The reference arm times the CPU oracle (C, OpenMP) on the same scene.
Multi-GPU: independent replicas, one per rank, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CCD queries/s and ms/step (broad+narrow) vs plain FP64 GPU form; % HBM/FP64 peak"
UNIT = "queries/s"
HBM_FALLBACK_GBS = 6800.0

# Per-launch DRAM traffic from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel with the hash of the source file it
# was taken on; ignored once the source changes.
NCU_TRAFFIC = {}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=512, help="cloth grid size")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload_name(n):
    return (f"folded cloth {n}x{n} vertices, fold gap 1e-3, 8-sinusoid push (amplitude 0.01), "
            f"delta=1e-6, min_sep=0, max_iter=1e6, earliest-TOI step")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(ms, e2e_ms, queries, device="cpu"):
    """Whole-job numbers over the ranks of the default process group: step
    times are the max over ranks, queries the sum.  Works on any backend
    (tensors on `device`)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    q = torch.tensor([float(queries)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(q, op=dist.ReduceOp.SUM)
    ms, e2e_ms = t.tolist()
    total = q.item()
    return {"ms": ms, "e2e_ms": e2e_ms, "queries": total,
            "value": total / (ms * 1e-3), "e2e_value": total / (e2e_ms * 1e-3)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path)), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def src_hash(name):
    p = os.path.join(ROOT, "paper_2112_06300_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


# ---------------------------------------------------------------------------
# Algorithmic work per stage (the roofline numerators).
# ---------------------------------------------------------------------------

# FP64 operations per evaluated interval: 18 DFMA for w, e1, e2 at the two
# time ends, 24 DFMA for the corner hull (2 corners x 2 time ends x 3 axes x
# 2 terms), 3 DADD for the width test; a DFMA counts 2 flops.
FLOPS_PER_INTERVAL = 2 * 42 + 3
# Per-unit set-up: 27 DSUB (c0, c1, dc), 3 DMUL + 3 DADD (error box),
# 6 DADD (time-derivative bound), 6 DADD (edge vectors at t = 1).
FLOPS_PER_UNIT = 27 + 3 + 3 + 6 + 6


def stage_algorithmic(st, nV, nE, nF):
    nB = nV + nE + nF
    pairs = st["n_vf"] + st["n_ee"]
    return {
        # V0, V1 (48 B per vertex), topology (8 B per edge, 12 B per face);
        # out: float box (24 B), ordered FP64 extents (48 B), ids (16 B)
        "boxes": ("hbm", 48 * nV + 8 * nE + 12 * nF + 88 * nB),
        # 4 passes of key + value in and out, plus the gather to sorted order
        "sort": ("hbm", 4 * 16 * nB + 8 * nB + 44 * nB + 40 * nB),
        # sorted boxes once (40 B), FP64 extents of box i (48 B) and of every
        # single-precision survivor (48 B), 8 B per pair written
        "sweep": ("hbm", 40 * nB + 48 * nB + 48 * st["n_superset"] + 8 * pairs),
        "narrow": ("alu", FLOPS_PER_INTERVAL * st["n_intervals"]
                   + FLOPS_PER_UNIT * (pairs + st["n_exported"])),
    }


def run_ours(args):
    import torch
    rank, local_rank, world = dist_info()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2112_06300_gb300 import build, ccd, scenes
    build.build()
    s = scenes.folded_cloth(args.n, seed=1)
    nV, nE, nF = len(s.V0), len(s.E), len(s.F)
    dev = f"cuda:{local_rank}"
    V0, V1, E, F = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F, dev)
    c = ccd.CCD(local_rank, profile_stages=1)
    stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float64, device=dev)
    t_ref = c.step(V0, V1, E, F)                    # sizes the pair buffers (synchronous)
    for _ in range(args.warmup):
        ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
    torch.cuda.synchronize()
    rc, st = c.status()
    assert rc == 0, ccd.ccd_status_str(rc)
    queries = st["n_vf"] + st["n_ee"]
    launches0 = st["n_launches"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stage_ms = {k: [] for k in ccd.STAGES}
    stats = []
    sampler = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        ccd.ccd_step(c.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
        ev[k][1].record(stream)
        for name, v in c.stage_times().items():      # synchronizes
            stage_ms[name].append(v)
        stats.append(c.status()[1])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    t_dev = float(out.item())
    assert t_dev == t_ref, (t_dev, t_ref)
    launches = stats[-1]["n_launches"] - launches0

    # end to end: host inputs copied in and the result read back every step
    hV0 = V0.cpu().pin_memory(); hV1 = V1.cpu().pin_memory()
    hE = E.cpu().pin_memory(); hF = F.cpu().pin_memory()
    dV0, dV1, dE, dF = (torch.empty_like(x) for x in (V0, V1, E, F))
    h2d = sum(x.numel() * x.element_size() for x in (hV0, hV1, hE, hF))
    res = np.empty(1, np.float64)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, h in ((dV0, hV0), (dV1, hV1), (dE, hE), (dF, hF)):
            d.copy_(h, non_blocking=True)
        ccd.ccd_step(c.ctx, dV0, dV1, dE, dF, 1e-6, 0.0, 10 ** 6, res)   # host output: synchronous
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    assert res[0] == t_ref

    agg = aggregate(ms, float(np.mean(e2e_ms)), queries, dev)
    ms, e2e_mean = agg["ms"], agg["e2e_ms"]

    # roofline of the dominant stage
    mean_stage = {k: float(np.mean(v)) for k, v in stage_ms.items()}
    algo = stage_algorithmic(stats[-1], nV, nE, nF)
    peaks, peak_src = measured_peaks()
    fp64 = ccd.ccd_measure_fp64_peak(local_rank)            # GFLOP/s, DFMA chains
    dom = max(mean_stage, key=mean_stage.get)
    kind, work = algo[dom]
    kernel = {"boxes": "k_build_boxes", "sort": "k_radix_scatter", "sweep": "k_sweep",
              "narrow": "k_narrow"}[dom]
    traffic = None
    tr = NCU_TRAFFIC.get(kernel)
    srcfile = "ccd_narrow.cu" if dom == "narrow" else "ccd_broad.cu"
    if tr and tr[1] == src_hash(srcfile):
        traffic = tr[0]
    if kind == "alu":
        achieved = work / (mean_stage[dom] * 1e-3) / 1e12
        peak = fp64 / 1e3
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "peak_source": "FP64 DFMA throughput measured live by ccd_measure_fp64_peak",
                "work_per_launch": work}
    else:
        achieved = work / (mean_stage[dom] * 1e-3) / 1e9
        peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "peak_source": peak_src, "work_per_launch": work}
    stage_frac = {}
    for k, (kk, w) in algo.items():
        if mean_stage[k] <= 0:
            continue
        if kk == "alu":
            stage_frac[k] = {"ms": mean_stage[k], "TFLOP/s": w / (mean_stage[k] * 1e-3) / 1e12,
                             "frac_fp64": w / (mean_stage[k] * 1e-3) / (fp64 * 1e9)}
        else:
            g = w / (mean_stage[k] * 1e-3) / 1e9
            stage_frac[k] = {"ms": mean_stage[k], "GB/s": g,
                             "frac_hbm": g / float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))}

    line = {
        "metric": METRIC, "value": agg["value"], "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded folded cloth; the paper's scenes are not available)",
        "config": {"workload": workload_name(args.n), "boxes": nV + nE + nF,
                   "queries_per_step": queries, "n_vf": st["n_vf"], "n_ee": st["n_ee"],
                   "superset_fp32": st["n_superset"], "intervals_per_step": stats[-1]["n_intervals"],
                   "toi": t_ref, "l2": "flushed (256 MiB write) before every timed step",
                   "precision": "broad FP32 outward-rounded + exact FP64 filter; narrow FP64",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": agg["e2e_value"], "unit": UNIT, "ms_per_step": e2e_mean,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8},
        "gpu_launches": launches,
        "stages_ms": mean_stage,
        "stage_roofline": stage_frac,
        "fp64_peak_gflops": fp64,
        "roofline": roof,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _oracle_step(s):
    from oracle import oracle as O
    t0 = time.perf_counter()
    vf, ee = O.broad(s.V0, s.V1, s.E, s.F)
    t1 = time.perf_counter()
    tmin = O.narrow(vf, ee, s.V0, s.V1, s.E, s.F, 1e-6, 0.0, 10 ** 6, 1)[4]
    t2 = time.perf_counter()
    return len(vf) + len(ee), tmin, t1 - t0, t2 - t1


def cpu_baseline(s):
    from oracle import oracle as O
    q, tmin, tb, tn = _oracle_step(s)
    return {"value": q / (tb + tn), "unit": UNIT, "cores": O.openmp_threads() or 1, "kind": "oracle",
            "sample": "one full oracle step on the same scene (serial sweep, OpenMP narrow phase)",
            "broad_s": tb, "narrow_s": tn, "toi": tmin}


def run_reference(args):
    rank, local_rank, world = dist_info()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2112_06300_gb300 import scenes
    s = scenes.folded_cloth(args.n, seed=1)
    for _ in range(args.warmup):
        _oracle_step(s)
    times, q, tmin = [], 0, None
    for _ in range(args.steps):
        q, tmin, tb, tn = _oracle_step(s)
        times.append(tb + tn)
    sec = float(np.mean(times))
    v = q / sec
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded folded cloth)",
            "config": {"workload": workload_name(args.n), "queries_per_step": q, "toi": tmin},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.openmp_threads() or 1, "kind": "oracle",
                             "sample": "full oracle step per timed step on the same scene"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
