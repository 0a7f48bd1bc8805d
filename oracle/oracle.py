"""Python wrapper of the C oracle (``ccd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The oracle shares no code with the
CUDA library and never imports it.

Layouts used here (the oracle's own, independent of the library's):
  V0, V1   float64 (nV, 3)
  E        int32 (nE, 2);  F int32 (nF, 3)
  pairs    int64 (n, 2): vertex-face (v, f), edge-edge (e_lo, e_hi), sorted
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libccd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available), without FMA
    contraction so that only the explicit fma() calls fuse."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _configure(L):
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    L.oracle_boxes.argtypes = [i64, P, P, i64, P, i64, P, P, P, P, P]
    L.oracle_boxes.restype = None
    for name in ("oracle_broad_brute", "oracle_broad_sweep"):
        fn = getattr(L, name)
        fn.argtypes = [i64, i64, P, i64, P, P, P, P, P, ctypes.c_int,
                       P, i64, P, P, i64, P]
        fn.restype = ctypes.c_int
    L.oracle_narrow.argtypes = [i64, P, P, P, P, ctypes.c_double,
                                ctypes.c_double, i64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, P, P, P, P]
    L.oracle_narrow.restype = None
    L.oracle_inclusion.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, P, P, P, P, P]
    L.oracle_inclusion.restype = None
    L.oracle_split_weights.argtypes = [ctypes.c_int, P, P, P, P]
    L.oracle_split_weights.restype = None
    L.oracle_has_openmp.argtypes = []
    L.oracle_has_openmp.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def load_variant(path: str):
    """Load another build of the oracle source (used by the tests that plant
    mistakes in a copy of it to show that the pins catch them)."""
    return _configure(ctypes.CDLL(path))


class using:
    """Context manager: route this module's calls to another loaded build."""

    def __init__(self, handle):
        self.handle = handle

    def __enter__(self):
        global _lib
        lib()
        self.saved, _lib = _lib, self.handle
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(V0, V1, E, F):
    V0 = np.ascontiguousarray(V0, dtype=np.float64).reshape(-1, 3)
    V1 = np.ascontiguousarray(V1, dtype=np.float64).reshape(-1, 3)
    E = np.ascontiguousarray(E, dtype=np.int32).reshape(-1, 2)
    F = np.ascontiguousarray(F, dtype=np.int32).reshape(-1, 3)
    assert V0.shape == V1.shape
    return V0, V1, E, F


def boxes(V0, V1, E, F):
    """FP64 extents and FP32 outward-rounded boxes of every vertex, edge and
    face (in that order).  Returns (lo64, hi64, lo32, hi32), each (nB, 3)."""
    V0, V1, E, F = _prep(V0, V1, E, F)
    nB = len(V0) + len(E) + len(F)
    lo64 = np.empty((nB, 3)); hi64 = np.empty((nB, 3))
    lo32 = np.empty((nB, 3), np.float32); hi32 = np.empty((nB, 3), np.float32)
    lib().oracle_boxes(len(V0), _p(V0), _p(V1), len(E), _p(E), len(F), _p(F),
                       _p(lo64), _p(hi64), _p(lo32), _p(hi32))
    return lo64, hi64, lo32, hi32


def broad(V0, V1, E, F, method: str = "sweep", fp32: bool = False):
    """Candidate pairs: vertex-face (v, f) and edge-edge (e_lo, e_hi) whose
    boxes overlap, no shared vertex.  method = "sweep" or "brute"; fp32 selects
    the outward-rounded single-precision boxes instead of the FP64 extents.
    Returns (vf, ee) as sorted int64 (n, 2) arrays."""
    V0, V1, E, F = _prep(V0, V1, E, F)
    lo64, hi64, lo32, hi32 = boxes(V0, V1, E, F)
    fn = lib().oracle_broad_sweep if method == "sweep" else lib().oracle_broad_brute
    nvf = np.zeros(1, np.int64); nee = np.zeros(1, np.int64)
    cap = 0
    dummy = np.zeros((1, 2), np.int64)
    rc = fn(len(V0), len(E), _p(E), len(F), _p(F), _p(lo64), _p(hi64), _p(lo32),
            _p(hi32), int(fp32), _p(dummy), cap, _p(nvf), _p(dummy), cap, _p(nee))
    if rc:
        raise MemoryError("oracle broad phase: allocation failed")
    vf = np.zeros((max(int(nvf[0]), 1), 2), np.int64)
    ee = np.zeros((max(int(nee[0]), 1), 2), np.int64)
    rc = fn(len(V0), len(E), _p(E), len(F), _p(F), _p(lo64), _p(hi64), _p(lo32),
            _p(hi32), int(fp32), _p(vf), len(vf), _p(nvf), _p(ee), len(ee), _p(nee))
    if rc:
        raise MemoryError("oracle broad phase: allocation failed")
    return vf[: int(nvf[0])], ee[: int(nee[0])]


def query_ids(vf, ee, E, F):
    """Stack vertex-face pairs then edge-edge pairs into (qtype, ids) with the
    four vertex ids of each query (VF: P, T0, T1, T2; EE: A0, A1, B0, B1)."""
    vf = np.asarray(vf, np.int64).reshape(-1, 2)
    ee = np.asarray(ee, np.int64).reshape(-1, 2)
    E = np.asarray(E, np.int64).reshape(-1, 2)
    F = np.asarray(F, np.int64).reshape(-1, 3)
    ids_vf = np.concatenate([vf[:, :1], F[vf[:, 1]]], axis=1) if len(vf) else np.zeros((0, 4), np.int64)
    ids_ee = np.concatenate([E[ee[:, 0]], E[ee[:, 1]]], axis=1) if len(ee) else np.zeros((0, 4), np.int64)
    qtype = np.concatenate([np.ones(len(vf), np.uint8), np.zeros(len(ee), np.uint8)])
    ids = np.ascontiguousarray(np.concatenate([ids_vf, ids_ee], axis=0), dtype=np.int64)
    return qtype, ids


def narrow_queries(qtype, ids, V0, V1, delta=1e-6, min_sep=0.0, max_iter=10**6,
                   mode=0, nthreads=0, no_zero=False):
    """Conservative interval bisection (Algorithm 3) on explicit queries.
    Returns (toi, flags, iters, toi_min); toi = +inf where no collision."""
    V0 = np.ascontiguousarray(V0, dtype=np.float64).reshape(-1, 3)
    V1 = np.ascontiguousarray(V1, dtype=np.float64).reshape(-1, 3)
    qtype = np.ascontiguousarray(qtype, dtype=np.uint8)
    ids = np.ascontiguousarray(ids, dtype=np.int64).reshape(-1, 4)
    n = len(qtype)
    toi = np.empty(n); flags = np.zeros(n, np.uint8); iters = np.zeros(n, np.int64)
    tmin = np.empty(1)
    lib().oracle_narrow(n, _p(qtype), _p(ids), _p(V0), _p(V1), float(delta),
                        float(min_sep), int(max_iter), int(mode), int(bool(no_zero)), int(nthreads),
                        _p(toi), _p(flags), _p(iters), _p(tmin))
    return toi, flags, iters, float(tmin[0])


def narrow(vf, ee, V0, V1, E, F, delta=1e-6, min_sep=0.0, max_iter=10**6, mode=0,
           nthreads=0, no_zero=False):
    """Narrow phase over pair lists; per-pair results are split back into the
    vertex-face and edge-edge parts: (toi_vf, toi_ee, flags_vf, flags_ee,
    toi_min)."""
    qtype, ids = query_ids(vf, ee, E, F)
    toi, flags, _, tmin = narrow_queries(qtype, ids, V0, V1, delta, min_sep,
                                         max_iter, mode, nthreads, no_zero)
    nvf = len(np.asarray(vf).reshape(-1, 2))
    return toi[:nvf], toi[nvf:], flags[:nvf], flags[nvf:], tmin


NO_ZERO_SCALE = 0.8


def step(V0, V1, E, F, delta=1e-6, min_sep=0.0, max_iter=10**6, nthreads=0, no_zero_toi=False):
    """Whole CCD (Algorithm 1): boxes, broad phase, earliest-TOI narrow phase.
    no_zero_toi (appendix "Zero time of impact and minimum separation"): when
    the earliest time is 0, run the narrow phase again with min_sep = 0 and
    the zero-TOI rule, and return that time scaled by 0.8."""
    vf, ee = broad(V0, V1, E, F, "sweep")
    t = narrow(vf, ee, V0, V1, E, F, delta, min_sep, max_iter, 1, nthreads)[4]
    if no_zero_toi and t == 0.0:
        t2 = narrow(vf, ee, V0, V1, E, F, delta, 0.0, max_iter, 1, nthreads, no_zero=True)[4]
        t = NO_ZERO_SCALE * t2
    return t


def inclusion(vf, x0, x1, n, l, min_sep=0.0):
    """B_F(I) and the error box for one query (4 points at t = 0 and t = 1)
    over the interval with dyadic ends n[k] / 2^l[k] .. (n[k] + 1) / 2^l[k]
    on (t, u, v).  Returns (bmin, bmax, ebox)."""
    V0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(4, 3)
    V1 = np.ascontiguousarray(x1, dtype=np.float64).reshape(4, 3)
    ids = np.arange(4, dtype=np.int64)
    nn = np.ascontiguousarray(n, dtype=np.uint64)
    ll = np.ascontiguousarray(l, dtype=np.int32)
    bmin = np.empty(3); bmax = np.empty(3); ebox = np.empty(3)
    lib().oracle_inclusion(int(vf), _p(ids), _p(V0), _p(V1), float(min_sep), _p(nn),
                           _p(ll), _p(bmin), _p(bmax), _p(ebox))
    return bmin, bmax, ebox


def split_weights(vf, x0, x1):
    """Split weights (L_t, L_u, L_v) of one query given by its 4 points at
    t = 0 and t = 1 (vertex-face: P, T0, T1, T2; edge-edge: A0, A1, B0, B1)."""
    V0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(4, 3)
    V1 = np.ascontiguousarray(x1, dtype=np.float64).reshape(4, 3)
    ids = np.arange(4, dtype=np.int64)
    L = np.empty(3)
    lib().oracle_split_weights(int(vf), _p(ids), _p(V0), _p(V1), _p(L))
    return L


def openmp_threads() -> int:
    return int(lib().oracle_has_openmp())
