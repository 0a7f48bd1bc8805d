"""Write the exact times of impact of a 100,000-query subset of the narrow-phase
stress workload (2^24 standalone queries, generator seed 2) to
stress_exact_1e5.txt.gz.

Calls only the exact rational oracle (oracle/exact.py: Sturm root isolation
and exact feasibility on the dyadic inputs); nothing here touches the CUDA
library.  The subset is the first 100,000 indices of a seeded permutation
(numpy default_rng(5)) of the 2^24 queries, stored sorted.

File format (text, gzip): '#' header lines -- the generator call, the subset
seed, and the SHA-256 of the subset's inputs (X0, X1 as little-endian float64
and is_vf as uint8, in index order) so that a reader can check that it
regenerated the same queries -- then one line per query:
    <index> <rd>
where <rd> is the largest double <= the exact time of impact (float.hex), or
'-' when the primitives never touch in [0, 1].  For a double t,
t <= t_exact exactly when t <= rd, so the line decides conservativeness
exactly.

    python tests/golden/make_stress_exact.py [--jobs N]
"""
from __future__ import annotations

import argparse
import gzip
import hashlib
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N_QUERIES = 1 << 24
GEN_SEED = 2
SUBSET_SEED = 5
SUBSET = 100_000
OUT = os.path.join(HERE, "stress_exact_1e5.txt.gz")


def subset_indices():
    return np.sort(np.random.default_rng(SUBSET_SEED).permutation(N_QUERIES)[:SUBSET])


def fingerprint(X0, X1, is_vf, idx):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(X0[idx], "<f8").tobytes())
    h.update(np.ascontiguousarray(X1[idx], "<f8").tobytes())
    h.update(np.ascontiguousarray(is_vf[idx], np.uint8).tobytes())
    return h.hexdigest()


def _round_down(x) -> float:
    """Largest double <= the exact number x."""
    from oracle import exact as X
    d = float(x)
    while not X.le_float(d, x):
        d = math.nextafter(d, -math.inf)
    while True:
        up = math.nextafter(d, math.inf)
        if X.le_float(up, x):
            d = up
        else:
            return d


def _one(job):
    from oracle import exact as X
    vf, x0, x1 = job
    r = X.toi(vf, x0, x1)
    return None if r is None else _round_down(r)


def read(path=OUT):
    """(header dict, indices int64, rd float64 with NaN for 'never touch')."""
    head, idx, rd = {}, [], []
    with gzip.open(path, "rt") as f:
        for line in f:
            if line.startswith("#"):
                k, _, v = line[1:].strip().partition("=")
                head[k.strip()] = v.strip()
                continue
            a, b = line.split()
            idx.append(int(a))
            rd.append(float("nan") if b == "-" else float.fromhex(b))
    return head, np.array(idx, np.int64), np.array(rd)


def summarize(toi, flags, rd):
    """Results t (float64, +inf for no collision) on the subset against the
    stored exact times: false negatives (an exact collision, none reported),
    late times (t > t_exact, decided exactly as t > rd), false positives (a
    collision reported where none exists), and t_exact - t on the queries
    where both find one (rd stands in for t_exact: within one ulp)."""
    hit = ~np.isnan(rd)
    fin = np.isfinite(toi)
    both = hit & fin
    err = rd[both] - toi[both]
    return {"n": int(len(rd)), "n_collide": int(hit.sum()), "fn": int((hit & ~fin).sum()),
            "late": int((toi[both] > rd[both]).sum()), "fp": int((~hit & fin).sum()),
            "fp_rate": float((~hit & fin).sum() / max(1, (~hit).sum())),
            "flagged": int((np.asarray(flags) != 0).sum()),
            "err_median": float(np.median(err)) if len(err) else 0.0,
            "err_mean": float(np.mean(err)) if len(err) else 0.0,
            "err_max": float(np.max(err)) if len(err) else 0.0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    args = ap.parse_args()
    from paper_2112_06300_gb300 import scenes
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(N_QUERIES, GEN_SEED)
    idx = subset_indices()
    fp = fingerprint(X0, X1, is_vf, idx)
    jobs = [(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist()) for q in idx]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        res = pool.map(_one, jobs, chunksize=64)
    dt = time.time() - t0
    with gzip.open(OUT, "wt", compresslevel=9) as f:
        f.write(f"# generator = scenes.narrow_stress_queries({N_QUERIES}, {GEN_SEED})\n")
        f.write(f"# subset = sorted(default_rng({SUBSET_SEED}).permutation({N_QUERIES})[:{SUBSET}])\n")
        f.write(f"# sha256 = {fp}\n")
        f.write("# columns = index, largest double <= exact time of impact (hex) or - for none\n")
        for q, r in zip(idx, res):
            f.write(f"{q} {'-' if r is None else float(r).hex()}\n")
    n_hit = sum(r is not None for r in res)
    print(f"{len(idx)} queries, {n_hit} collide, {dt:.0f} s on {args.jobs} processes -> {OUT}")


if __name__ == "__main__":
    main()
