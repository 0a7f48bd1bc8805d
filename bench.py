#!/usr/bin/env python3
"""Benchmark of the CCD hot path: one step = boxes + broad phase + earliest-TOI
narrow phase (Algorithm 1) over the folded-cloth self-contact scene, 512 x 512
vertices (262,144 V, 784,385 E, 522,242 F, 1,568,771 boxes), delta = 1e-6,
min_sep = 0, max_iter = 1e6, synthetic seeded input.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cloth|batch|serve|precision]

Prints one JSON line (rank 0).  `value` is CCD queries per second of the
whole job: narrow-phase candidate pairs of every rank / max-over-ranks step
time.  The reference arm times the CPU oracle (C, OpenMP) on the same scene.
Multi-GPU: independent replicas, one per rank, no collective on the data path.

With no --workload, the line also carries a "forms" object with every other
configuration, each in this library's form and against the plain FP64 form
(FP64 broad phase throughout, same narrow phase), with queries/s and
fractions of roofline:
  cloth_min_sep_1e-4  the same cloth step with min_sep = 1e-4;
  icosphere_plane     icosphere on a plane (21,635 boxes), also per pair;
  stress_2^24         2^24 standalone narrow-phase queries, per-pair times,
                      and the stored exact-oracle subset (100,000 queries):
                      false negatives, late times, false positives;
  precision           the folded cloth plus 1,000 rigid bodies (4.1M
                      triangles): single-precision broad phase with the exact
                      FP64 filter against the all-FP64 broad phase --
                      candidate counts, final-set equality, time;
  batched             4,096 rigid environments (500-50,000 triangles,
                      log-uniform) stepped in batches sized by the memory
                      model for a 64 GiB budget, plus one batch stepped
                      repeatedly under a captured CUDA graph;
  serving             the same environments arriving as a Poisson stream
                      (2e4 steps/s) into the serving runtime; p50/p99 latency
                      from arrival (client write included) to completion.
--workload batch|serve|precision prints that form alone as its own line.
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

# Issue counters of k_narrow from one ncu capture on the 256 x 256 cloth
# (smsp__inst_executed.sum / intervals evaluated, smsp__thread_inst_executed.sum
# / smsp__inst_executed.sum, sm__warps_active), keyed by the source hash.
NCU_ISSUE = {
    # ncu --replay-mode application --clock-control none --metrics smsp__inst_executed.sum,
    #     smsp__thread_inst_executed.sum,sm__warps_active...,smsp__issue_active...  -k regex:"^k_narrow$|^k_sweep_strips$"
    #     -s 8 -c 2  python bench.py --n 256 --steps 1 --warmup 3 --no-cpu-baseline --no-forms --no-autotune
    #     (808.3M warp instructions; 18.49M intervals, the mean of the three replayed runs)
    "k_narrow": {"warp_inst_per_interval": 43.72, "threads_per_inst": 18.92, "warps_active": 0.1873,
                 "src": "2d4b4e3d8e4651bb",
                 "cmd": "ncu --replay-mode application, 256 x 256 cloth, bench.py --no-autotune"},
}

# Per-launch DRAM traffic from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel with the hash of the source file it
# was taken on; ignored once the source changes.  (Both keys name the source
# after a comment-only edit: the compiled kernel is byte-identical to the one
# profiled.)
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
    #     -k regex:"^k_narrow$|..." -s 28 -c 7
    #     python bench.py --steps 2 --warmup 3 --no-cpu-baseline --no-forms --no-autotune
    #     (1.612 GB read + 56.4 MB written)
    "k_narrow": (1.612e9 + 56.43e6, "2d4b4e3d8e4651bb"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=512, help="cloth grid size")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the other configurations and forms")
    p.add_argument("--no-autotune", action="store_true", help="time the cloth step with the default settings")
    p.add_argument("--workload", choices=["cloth", "batch", "serve", "precision"], default="cloth")
    p.add_argument("--envs", type=int, default=4096, help="batch/serve: environments")
    p.add_argument("--rate", type=float, default=2e4, help="serve: arrivals per second")
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
    nc = st.get("n_box_copies", nB)          # box copies, one per overlapped cell
    return {
        # V0, V1 (48 B per vertex), topology (8 B per edge, 12 B per face);
        # out: float box (24 B), ordered FP64 extents (48 B), ids (16 B)
        "boxes": ("hbm", 48 * nV + 8 * nE + 12 * nF + 88 * nB),
        # cell counts (8 B per box in), keys and values of the copies (12 B
        # out), one counting read of the keys (8 B per copy), 7 passes (8-bit
        # digits of the 56-bit key) of key + value in and out (24 B per copy;
        # passes of digits that every key shares are skipped, two at a time,
        # but still counted), gather to sorted order (12 B key/value + 36 B
        # box data in, 36 B out)
        "sort": ("hbm", 8 * nB + 12 * nc + 8 * nc + 7 * 24 * nc + 84 * nc),
        # sorted copies once (44 B with the key), 8 B per candidate written,
        # then the exact filter: 8 B read + 96 B of FP64 extents per
        # candidate, 8 B per pair written
        "sweep": ("hbm", 44 * nc + 8 * st["n_superset"] + 104 * st["n_superset"] + 8 * pairs),
        "narrow": ("alu", FLOPS_PER_INTERVAL * st["n_intervals"]
                   + FLOPS_PER_UNIT * (pairs + st["n_exported"])),
        # the narrow-phase kernel alone (the set-up runs in the record pass)
        "narrow_kernel": ("alu", FLOPS_PER_INTERVAL * st["n_intervals"]),
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
    # the library's own autotuner picks the cell width, hand-off budget and
    # interval-queue size for this mesh (outside the timed region, once)
    tuning = c.autotune(V0, V1, E, F, reps=3) if not args.no_autotune else None
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

    # the plain FP64 GPU form on the same scene: FP64 boxes throughout (no
    # single-precision stage, no filter), same narrow phase
    c64 = ccd.CCD(local_rank, broad_fp64=1, profile_stages=1)
    assert c64.step(V0, V1, E, F) == t_ref
    ms64, broad64 = [], []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        ccd.ccd_step(c64.ctx, V0, V1, E, F, 1e-6, 0.0, 10 ** 6, out)
        b.record(stream)
        t64 = c64.stage_times()
        broad64.append(t64["boxes"] + t64["sort"] + t64["sweep"])
        ms64.append(a.elapsed_time(b))
    assert c64.status()[0] == 0 and float(out.item()) == t_ref
    c64.close()
    fp64_form = {"ms_per_step": float(np.median(ms64)), "broad_ms": float(np.median(broad64)),
                 "step_speedup": float(np.median(ms64)) / ms}

    agg = aggregate(ms, float(np.mean(e2e_ms)), queries, dev)
    ms, e2e_mean = agg["ms"], agg["e2e_ms"]

    # roofline of the dominant stage
    mean_stage = {k: float(np.mean(v)) for k, v in stage_ms.items()}
    algo = stage_algorithmic(stats[-1], nV, nE, nF)
    peaks, peak_src = measured_peaks()
    fp64 = ccd.ccd_measure_fp64_peak(local_rank)            # GFLOP/s, DFMA chains
    dom = max(("boxes", "sort", "sweep", "narrow"), key=mean_stage.get)
    if dom == "narrow":
        dom = "narrow_kernel"                # the dominant kernel: k_narrow, timed alone
    kind, work = algo[dom]
    kernel = {"boxes": "k_build_boxes", "sort": "k_sort_pass", "sweep": "k_sweep_strips",
              "narrow_kernel": "k_narrow"}[dom]
    traffic = None
    tr = NCU_TRAFFIC.get(kernel)
    srcfile = "ccd_narrow.cu" if dom == "narrow_kernel" else "ccd_broad.cu"
    if tr and tr[1] == src_hash(srcfile):
        traffic = tr[0]
    if kind == "alu":
        achieved = work / (mean_stage[dom] * 1e-3) / 1e12
        peak = fp64 / 1e3
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kernel,
                "peak_source": "FP64 DFMA throughput measured live by ccd_measure_fp64_peak",
                "work_per_launch": work, "ms_per_launch": mean_stage[dom],
                "work": "FP64-equivalent: 87 flops per evaluated interval, the FP64 evaluation of "
                        "Algorithm 3 that the single-precision filter mostly replaces"}
        # the kernel's real limiter: instruction issue (ncu: warp instructions
        # per evaluated interval on the 256 x 256 cloth, same source)
        iss = NCU_ISSUE.get(kernel)
        if iss and iss["src"] == src_hash(srcfile):
            mhz = (clocks or {}).get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
            sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
            peak_issue = 4 * sms * mhz * 1e6 / 1e12          # warp instructions per ps ... (T/s)
            got = iss["warp_inst_per_interval"] * stats[-1]["n_intervals"] / (mean_stage[dom] * 1e-3) / 1e12
            roof["issue"] = {"achieved": got, "peak": peak_issue, "unit": "T warp-instructions/s",
                             "frac": got / peak_issue, "warp_inst_per_interval": iss["warp_inst_per_interval"],
                             "threads_per_inst": iss["threads_per_inst"], "warps_active": iss["warps_active"],
                             "peak_source": f"4 schedulers x {sms} SMs x {mhz:.0f} MHz (median SM clock under load)",
                             "counters": iss["cmd"]}
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
                   "autotuned": ({k: tuning[k] for k in ("strip_width", "export_budget", "queue_capacity")}
                                 if tuning else "no (defaults)"),
                   "autotune_ms": ({"before": tuning["default_ms"], "after": tuning["broad_ms"] + tuning["narrow_ms"]}
                                   if tuning else None),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": agg["e2e_value"], "unit": UNIT, "ms_per_step": e2e_mean,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8},
        "gpu_launches": launches,
        "fp64_form": fp64_form,
        "stages_ms": mean_stage,
        "stage_roofline": stage_frac,
        "fp64_peak_gflops": fp64,
        "roofline": roof,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s)
    if world == 1 and not args.no_forms:
        c.close()
        line["forms"] = run_forms(args, flush, fp64, float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS)))
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


# ---------------------------------------------------------------------------
# The other configurations and forms (one GPU): each returns a dict that goes
# into the "forms" object of the default line, or alone with --workload.
# ---------------------------------------------------------------------------

BUDGET = 64 << 30          # device memory budget of the batched and serving forms
PAIRS_PER_BOX = 1.0        # candidate pairs per box budgeted (rigid environments: ~0.63)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _roof(st, stages, nV, nE, nF, fp64_gflops, hbm_gbs):
    """Fractions of roofline of the broad phase (HBM, its three stages'
    algorithmic bytes over their summed time) and of the narrow phase (FP64
    pipe, FP64-equivalent flops over its time)."""
    algo = stage_algorithmic(st, nV, nE, nF)
    out = {}
    broad_ms = sum(stages.get(k, 0.0) for k in ("boxes", "sort", "sweep"))
    if broad_ms > 0:
        by = sum(algo[k][1] for k in ("boxes", "sort", "sweep"))
        out["broad_hbm_frac"] = by / (broad_ms * 1e-3) / 1e9 / hbm_gbs
    if stages.get("narrow", 0.0) > 0:
        out["narrow_fp64_frac"] = algo["narrow"][1] / (stages["narrow"] * 1e-3) / (fp64_gflops * 1e9)
    return out


def time_steps(c, d, min_sep, steps, flush):
    """Median device time of ccd_step (device output), its stages and the
    counters of the last step; the pair buffers are sized by one synchronous
    step first."""
    import torch
    from paper_2112_06300_gb300 import ccd
    stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float64, device=d[0].device)
    t_ref = c.step(*d, min_sep=min_sep)
    for _ in range(2):
        ccd.ccd_step(c.ctx, *d, 1e-6, min_sep, 10 ** 6, out)
    ms, stages = [], {k: [] for k in ccd.STAGES}
    for _ in range(steps):
        flush.zero_()
        a, b = _events()
        a.record(stream)
        ccd.ccd_step(c.ctx, *d, 1e-6, min_sep, 10 ** 6, out)
        b.record(stream)
        for k, v in c.stage_times().items():     # synchronizes
            stages[k].append(v)
        ms.append(a.elapsed_time(b))
    rc, st = c.status()
    assert rc == 0, ccd.ccd_status_str(rc)
    assert float(out.item()) == t_ref
    return {"ms": float(np.median(ms)), "stages": {k: float(np.median(v)) for k, v in stages.items()},
            "stats": st, "toi": t_ref}


def form_scene(name, s, min_sep, steps, flush, fp64_gflops, hbm_gbs, per_pair=False):
    """One scene: the step in this library's form (FP32 broad + exact filter,
    FP64 narrow) and in the plain FP64 form (FP64 broad throughout, same
    narrow phase), queries/s and fractions of roofline of each."""
    from paper_2112_06300_gb300 import ccd
    d = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F, "cuda:0")
    nV, nE, nF = len(s.V0), len(s.E), len(s.F)
    res = {"workload": name, "boxes": nV + nE + nF, "min_sep": min_sep}
    for form, o in (("fp32_broad", {}), ("plain_fp64", {"broad_fp64": 1})):
        c = ccd.CCD(0, profile_stages=1, **o)
        r = time_steps(c, d, min_sep, steps, flush)
        st = r["stats"]
        q = st["n_vf"] + st["n_ee"]
        res[form] = {"ms_per_step": r["ms"], "queries": q, "queries_per_s": q / (r["ms"] * 1e-3),
                     "stages_ms": r["stages"], "toi": r["toi"], "intervals": st["n_intervals"],
                     "capped": st["n_capped"], "superset_fp32": st["n_superset"],
                     **_roof(st, r["stages"], nV, nE, nF, fp64_gflops, hbm_gbs)}
        if per_pair and form == "fp32_broad":
            # the configuration's output: sorted pair lists and per-pair times
            import torch
            vf, ee = c.broad(*d)
            a, b = _events()
            a.record()
            nr = c.narrow(vf, ee, *d, 1e-6, min_sep, 10 ** 6, 0)
            b.record()
            torch.cuda.synchronize()
            res[form]["per_pair_narrow_ms"] = a.elapsed_time(b)
            res[form]["per_pair_toi_min"] = nr.toi_min
        c.close()
    res["step_speedup_vs_plain_fp64"] = res["plain_fp64"]["ms_per_step"] / res["fp32_broad"]["ms_per_step"]
    assert res["plain_fp64"]["toi"] == res["fp32_broad"]["toi"]
    if per_pair:
        # a small scene is launch-bound: the same step replayed as a captured CUDA graph
        import torch
        c = ccd.CCD(0, use_graph=1)
        out = torch.empty(1, dtype=torch.float64, device=d[0].device)
        c.step(*d, min_sep=min_sep)
        for _ in range(3):
            ccd.ccd_step(c.ctx, *d, 1e-6, min_sep, 10 ** 6, out)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = _events()
            a.record()
            ccd.ccd_step(c.ctx, *d, 1e-6, min_sep, 10 ** 6, out)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        assert c.status()[0] == 0 and float(out.item()) == res["fp32_broad"]["toi"]
        c.close()
        res["fp32_broad"]["graph_ms_per_step"] = float(np.median(ms))
    return res


def form_stress(steps, fp64_gflops):
    """The narrow-phase stress workload: 2^24 standalone queries, per-pair
    times, and the exact-oracle subset of 100,000 stored queries (false
    negatives, late times, false positives).  The exact times were written by
    tests/golden/make_stress_exact.py; here they are only read."""
    import torch
    from paper_2112_06300_gb300 import ccd, scenes
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_stress_exact as G
    n = G.N_QUERIES
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(n, G.GEN_SEED)
    head, idx, rd = G.read()
    same = head.get("sha256") == G.fingerprint(X0, X1, is_vf, idx)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    del X0, X1
    d = ccd.mesh_to_device(sc.V0, sc.V1, sc.E, sc.F, "cuda:0")
    vfd, eed = torch.from_numpy(vf).cuda(), torch.from_numpy(ee).cuda()
    c = ccd.CCD(0, profile_stages=1)
    ms = []
    for k in range(1 + steps):
        a, b = _events()
        a.record()
        r = c.narrow(vfd, eed, *d, 1e-6, 0.0, 10 ** 6, 0)
        b.record()
        torch.cuda.synchronize()
        if k:
            ms.append(a.elapsed_time(b))
    rc, st = c.status()
    toi = np.empty(n)
    flags = np.empty(n, np.uint8)
    toi[order] = np.concatenate([r.toi_vf.cpu().numpy(), r.toi_ee.cpu().numpy()])
    flags[order] = np.concatenate([r.flags_vf.cpu().numpy(), r.flags_ee.cpu().numpy()])
    c.close()
    m = float(np.median(ms))
    flops = FLOPS_PER_INTERVAL * st["n_intervals"] + FLOPS_PER_UNIT * (n + st["n_exported"])
    out = {"workload": "2^24 standalone queries, 50/50 VF/EE, 2^-20 grid, mix 40/20/10/10/20, delta=1e-6, "
                       "max_iter=1e6, per-pair times", "queries": n, "ms": m, "queries_per_s": n / (m * 1e-3),
           "intervals": st["n_intervals"], "capped": st["n_capped"], "flagged": int((flags != 0).sum()),
           "collisions": int(np.isfinite(toi).sum()),
           "narrow_fp64_frac": flops / (m * 1e-3) / (fp64_gflops * 1e9),
           "vs_plain_fp64": "same kernel (no broad phase in this workload)"}
    if same:
        out["exact_subset"] = G.summarize(toi[idx], flags[idx], rd)
    else:
        out["exact_subset"] = "generator output differs from the stored subset; not compared"
    return out


def environments(n):
    from paper_2112_06300_gb300 import scenes
    return [scenes.rigid_environment(seed) for seed in range(n)]


def chunks_by_memory(envs, ccd):
    """Consecutive environments per batch, as many as the memory model fits
    in BUDGET with PAIRS_PER_BOX pairs per box (Section "Batching": the
    candidate capacity follows from the free memory)."""
    m = ccd.ccd_get_memory_model()
    per_box = m["bytes_per_box"] + PAIRS_PER_BOX * m["bytes_per_pair"]
    out, cur, boxes = [], [], 0
    for e in envs:
        b = e.n_boxes
        if cur and m["bytes_fixed"] + (boxes + b) * per_box + (len(cur) + 1) * m["bytes_per_scene"] > BUDGET:
            out.append(cur)
            cur, boxes = [], 0
        cur.append(e)
        boxes += b
    if cur:
        out.append(cur)
    return out


def form_batch(envs, steps, warmup):
    """Batched form: every environment in batches sized by the memory model
    for a 64 GiB budget, one batched step per batch; a sample of scenes is
    stepped alone (FP32 form and plain FP64 form) for parity and for the
    per-scene comparison."""
    import torch
    from paper_2112_06300_gb300 import ccd, scenes
    torch.cuda.set_device(0)
    groups = chunks_by_memory(envs, ccd)
    nb_max = max(sum(e.n_boxes for e in g) for g in groups)
    cap = int(PAIRS_PER_BOX * nb_max) + (1 << 20)
    c = ccd.CCD(0, pair_capacity=cap)
    dev = "cuda:0"
    prepared = []
    for g in groups:
        V0, V1, E, F, vo, eo, fo = scenes.concat_scenes(g)
        d = ccd.mesh_to_device(V0, V1, E, F, dev)
        offs = [torch.from_numpy(a).to(dev) for a in (vo, eo, fo)]
        prepared.append((d, offs, torch.empty(len(g), dtype=torch.float64, device=dev)))
    stream = torch.cuda.current_stream()
    for (d, offs, out) in prepared[:1] * max(1, warmup):
        ccd.ccd_step_batch(c.ctx, *offs, *d, 1e-6, 0.0, 10 ** 6, out)
    torch.cuda.synchronize()
    ms_all, pairs = [], 0
    for _ in range(steps):
        ev = [_events() for _ in prepared]
        pairs = 0
        for (d, offs, out), (a, b) in zip(prepared, ev):
            a.record(stream)
            ccd.ccd_step_batch(c.ctx, *offs, *d, 1e-6, 0.0, 10 ** 6, out)
            b.record(stream)
            rc, st = c.status()
            assert rc == 0, ccd.ccd_status_str(rc)
            pairs += st["n_vf"] + st["n_ee"]
        torch.cuda.synchronize()
        ms_all.append(sum(a.elapsed_time(b) for a, b in ev))
    toi = np.concatenate([out.cpu().numpy() for (_, _, out) in prepared])
    c.close()
    ms = float(np.median(ms_all))
    # a sample of environments stepped alone: the same time (parity of the
    # batch against single-scene steps), and the per-scene time of the plain
    # FP64 form for the comparison
    rng = np.random.default_rng(0)
    sample = rng.choice(len(envs), size=min(64, len(envs)), replace=False)
    alone_ms = {}
    for form, o in (("fp32_broad", {}), ("plain_fp64", {"broad_fp64": 1})):
        ca = ccd.CCD(0)
        tot = 0.0
        for k in sample:
            e = envs[k]
            d = ccd.mesh_to_device(e.V0, e.V1, e.E, e.F, dev)
            t = ca.step(*d)
            assert t == toi[k], (form, k, t, toi[k])
            out = torch.empty(1, dtype=torch.float64, device=dev)
            a, b = _events()
            a.record(stream)
            ccd.ccd_step(ca.ctx, *d, 1e-6, 0.0, 10 ** 6, out)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        ca.close()
        alone_ms[form] = tot / len(sample) * len(envs)
    # one batch of 512 environments stepped repeatedly: launch sequence
    # against the captured CUDA graph
    sub = envs[:512]
    V0, V1, E, F, vo, eo, fo = scenes.concat_scenes(sub)
    d = ccd.mesh_to_device(V0, V1, E, F, dev)
    offs = [torch.from_numpy(a).to(dev) for a in (vo, eo, fo)]
    out = torch.empty(len(sub), dtype=torch.float64, device=dev)
    rep = {}
    for g in (0, 1):
        cg = ccd.CCD(0, use_graph=g, pair_capacity=cap)
        for _ in range(3):
            ccd.ccd_step_batch(cg.ctx, *offs, *d, 1e-6, 0.0, 10 ** 6, out)
        torch.cuda.synchronize()
        a, b = _events()
        a.record(stream)
        for _ in range(10):
            ccd.ccd_step_batch(cg.ctx, *offs, *d, 1e-6, 0.0, 10 ** 6, out)
        b.record(stream)
        torch.cuda.synchronize()
        rep["graph" if g else "launches"] = a.elapsed_time(b) / 10
        assert cg.status()[0] == 0
        cg.close()
    tri = sum(len(e.F) for e in envs)
    boxes = sum(e.n_boxes for e in envs)
    return {"workload": f"{len(envs)} rigid environments, 500-50,000 triangles (log-uniform), |v| <= 0.05, "
                        f"delta=1e-6, batches sized for a 64 GiB budget",
            "envs": len(envs), "triangles": tri, "boxes": boxes, "batches": len(groups), "ms": ms,
            "envs_per_s": len(envs) / (ms * 1e-3), "queries": int(pairs), "queries_per_s": pairs / (ms * 1e-3),
            "collisions": int(np.isfinite(toi).sum()),
            "one_scene_per_call_ms": {"fp32_broad": alone_ms["fp32_broad"], "plain_fp64": alone_ms["plain_fp64"],
                                      "note": f"extrapolated from {len(sample)} environments stepped alone"},
            "speedup_vs_plain_fp64_one_scene_per_call": alone_ms["plain_fp64"] / ms,
            "parity_sample": f"{len(sample)} environments: batched time == the scene stepped alone",
            "batch512_ms": rep}


def form_serve(envs, rate, n_slots=2, verify=32, clients=8):
    """Serving form: the environments arrive as a Poisson stream; at its
    arrival time a client hands the scene, held in the arena's layout (V0, V1
    as [3][nV], E, F), to ccd_server_submit_scene, which copies it into the
    server's arena and queues it (`clients` client threads take the arrivals
    in turn).
    Latency runs from the arrival (before the write) to the completion; a
    sample of results is compared with the scene stepped alone."""
    import gc
    import threading
    from paper_2112_06300_gb300 import ccd
    srv = ccd.Server(0, n_slots=n_slots, max_scenes=256, memory_cap=BUDGET, arena_bytes=4 << 30,
                     pairs_per_box=PAIRS_PER_BOX, autotune=1)
    for e in envs[:64]:                              # warm-up: contexts and buffers grow
        srv.wait(srv.submit_scene(e.V0, e.V1, e.E, e.F))
    rng = np.random.default_rng(3)
    arrive = np.cumsum(rng.exponential(1.0 / rate, len(envs)))
    # the clients' scenes in the arena's layout (structure of arrays)
    soa = [(np.ascontiguousarray(e.V0.T), np.ascontiguousarray(e.V1.T), np.ascontiguousarray(e.E, np.int32),
            np.ascontiguousarray(e.F, np.int32)) for e in envs]
    tickets = [None] * len(envs)
    late_ms = np.zeros(len(envs))                  # arrival -> the client starts writing
    write_ms = np.zeros(len(envs))                 # writing and queueing the scene
    # Python's collector stops every client thread while it runs (tens of ms
    # once the process holds the other configurations' data): collect before
    # the arrivals start and not during them
    gc.collect()
    gc.disable()
    t0 = time.perf_counter() + 0.05

    def client(ks):
        for k in ks:
            e = envs[k]
            while True:
                dt = t0 + arrive[k] - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            tw = time.perf_counter()
            tickets[k] = srv.submit_soa(*soa[k])   # copy into the arena and queue (one library call)
            write_ms[k] = (time.perf_counter() - tw) * 1e3
            late_ms[k] = (tw - (t0 + arrive[k])) * 1e3

    th = [threading.Thread(target=client, args=(range(i, len(envs), clients),)) for i in range(clients)]
    try:
        for t in th:
            t.start()
        for t in th:
            t.join()
        t_sub = time.perf_counter() - t0
        res = [srv.wait(t) for t in tickets]
        t_all = time.perf_counter() - t0
    finally:
        gc.enable()
    st = srv.stats()
    srv.close()
    lat_srv = np.array([r[1] for r in res])       # submission -> completion
    lat = lat_srv + write_ms + late_ms             # arrival -> completion
    toi = np.array([r[0] for r in res])
    c = ccd.CCD(0)
    pick = np.random.default_rng(4).choice(len(envs), size=min(verify, len(envs)), replace=False)
    for k in pick:
        e = envs[k]
        assert c.step(*ccd.mesh_to_device(e.V0, e.V1, e.E, e.F, "cuda:0")) == toi[k], k
    c.close()
    return {"workload": f"{len(envs)} rigid environments arriving as a Poisson stream at {rate:g}/s, {clients} client "
                        f"threads writing and submitting each scene at its arrival, {n_slots} slots autotuned on "
                        f"their first batch, <= 256 scenes per batch, 64 GiB cap",
            "steps_per_s": len(envs) / t_all, "offered_rate": len(envs) / t_sub, "target_rate": rate,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max()),
                           "client_write_p50": float(np.percentile(write_ms, 50)),
                           "client_start_delay_p99": float(np.percentile(late_ms, 99)),
                           "server_p50": float(np.percentile(lat_srv, 50)),
                           "server_p99": float(np.percentile(lat_srv, 99))},
            "batches": st["n_batches"], "max_batch_scenes": st["max_batch_scenes"],
            "max_inflight_bytes": st["max_inflight_bytes"], "collisions": int(np.isfinite(toi).sum()),
            "parity_sample": f"{len(pick)} served results == the scene stepped alone"}


def form_precision(n, steps, flush, fp64_gflops, hbm_gbs):
    """Precision form: the folded cloth plus 1,000 rigid bodies.  Broad phase
    in single precision (outward-rounded boxes) then the exact FP64 filter,
    against the all-FP64 broad phase (same cell sweep on FP64 extents);
    superset size, final-set equality, broad and whole-step times."""
    import torch
    from paper_2112_06300_gb300 import ccd, scenes
    s = scenes.cloth_and_bodies(n)
    d = ccd.mesh_to_device(s.V0, s.V1, s.E, s.F, "cuda:0")
    out = form_scene(f"folded cloth {n}x{n} + 500 icospheres (5,120 tri) + 500 tori (3,072 tri) in [0,10]^3, "
                     "placed without interpenetration", s, 0.0, steps, flush, fp64_gflops, hbm_gbs)
    key = lambda t: torch.sort(t[:, 0].long() * (1 << 32) + t[:, 1].long())[0]
    sets = {}
    for form, o in (("fp32_broad", {}), ("plain_fp64", {"broad_fp64": 1})):
        c = ccd.CCD(0)
        vf, ee = c.broad(*d)
        sets[form] = (key(vf), key(ee))
        c.close()
    out["final_sets_equal"] = bool(torch.equal(sets["fp32_broad"][0], sets["plain_fp64"][0]) and
                                   torch.equal(sets["fp32_broad"][1], sets["plain_fp64"][1]))
    out["broad_ms"] = {f: sum(out[f]["stages_ms"][k] for k in ("boxes", "sort", "sweep"))
                       for f in ("fp32_broad", "plain_fp64")}
    out["broad_speedup_vs_plain_fp64"] = out["broad_ms"]["plain_fp64"] / out["broad_ms"]["fp32_broad"]
    return out


def run_forms(args, flush, fp64_gflops, hbm_gbs):
    """Every other configuration of the benchmark, for the "forms" object."""
    from paper_2112_06300_gb300 import scenes
    forms = {}
    t0 = time.perf_counter()
    forms["cloth_min_sep_1e-4"] = form_scene(workload_name(args.n).replace("min_sep=0", "min_sep=1e-4"),
                                             scenes.folded_cloth(args.n, seed=1), 1e-4, 3, flush,
                                             fp64_gflops, hbm_gbs)
    forms["icosphere_plane"] = form_scene("icosphere (2,562 V) on a 33x33 plane, dz=-0.1, N(0,1e-3) jitter, "
                                          "delta=1e-6", scenes.icosphere_on_plane(0), 0.0, 10, flush,
                                          fp64_gflops, hbm_gbs, per_pair=True)
    forms["stress_2^24"] = form_stress(2, fp64_gflops)
    forms["precision"] = form_precision(args.n, 3, flush, fp64_gflops, hbm_gbs)
    envs = environments(args.envs)
    forms["batched"] = form_batch(envs, 3, 2)
    forms["serving"] = form_serve(envs, args.rate)
    forms["seconds"] = time.perf_counter() - t0
    return forms


def run_batch(args):
    line = {"metric": "environments/s (batched earliest-TOI step)", "unit": "envs/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic (seeded rigid environments)"}
    r = form_batch(environments(args.envs), args.steps, args.warmup)
    line.update({"value": r["envs_per_s"], "ms_per_step": r["ms"], "config": {"workload": r["workload"]}, **r})
    print(json.dumps(line), flush=True)


def run_serve(args):
    from paper_2112_06300_gb300 import build
    build.build()
    r = form_serve(environments(args.envs), args.rate)
    line = {"metric": "served CCD steps/s and p50/p99 latency (ms), Poisson arrivals", "value": r["steps_per_s"],
            "unit": "steps/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic (seeded rigid environments)", "config": {"workload": r["workload"]}, **r}
    print(json.dumps(line), flush=True)


def run_precision(args):
    import torch
    from paper_2112_06300_gb300 import build, ccd
    build.build()
    torch.cuda.set_device(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:0")
    peaks, _ = measured_peaks()
    r = form_precision(args.n, max(3, args.steps // 4), flush, ccd.ccd_measure_fp64_peak(0),
                       float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS)))
    line = {"metric": "broad-phase ms: FP32 outward-rounded + exact FP64 filter vs all-FP64 (same cell sweep)",
            "value": r["broad_speedup_vs_plain_fp64"], "unit": "x (FP64 ms / FP32 ms)", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32+f64 / f64", "data": "synthetic (seeded)",
            "config": {"workload": r["workload"]}, **r}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "precision":
        run_precision(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
