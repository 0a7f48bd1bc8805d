"""Python binding of the C ABI in include/ccd.h (argument marshalling only).

Every function here forwards to libccd.so; device memory and streams come
from PyTorch tensors.  There is no CPU path: importing works anywhere, but
every call raises when the CUDA library or a CUDA device is missing.

Layouts (as in include/ccd.h):
  V0, V1   float64 CUDA tensors, shape (3, nV) (structure of arrays)
  E        int32 CUDA tensor (nE, 2);  F int32 CUDA tensor (nF, 3)
  pairs    int32 CUDA tensors (n, 2): vertex-face (v, f), edge-edge (e_lo, e_hi)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libccd.so")

CCD_OK, CCD_EINVAL, CCD_ENOMEM, CCD_ETRUNC, CCD_EQUEUE, CCD_ETIMEOUT, CCD_ECUDA, CCD_EDEVICE = range(8)
CCD_FLAG_ITER_CAP = 1
CCD_FLAG_LEVEL_CAP = 2


class ccd_opts(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("min_sep", ctypes.c_double),
                ("max_iter", ctypes.c_int64), ("broad_fp64", ctypes.c_int32),
                ("sweep_kernel", ctypes.c_int32), ("pair_capacity", ctypes.c_int64),
                ("queue_capacity", ctypes.c_int64), ("export_budget", ctypes.c_int32),
                ("profile_stages", ctypes.c_int32), ("no_zero_toi", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("strip_width", ctypes.c_double), ("memory_limit", ctypes.c_int64)]


class ccd_stats(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int64), ("sweep_axis", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("n_superset", ctypes.c_int64), ("n_vf", ctypes.c_int64), ("n_ee", ctypes.c_int64),
                ("n_intervals", ctypes.c_int64), ("n_exported", ctypes.c_int64),
                ("n_capped", ctypes.c_int64), ("queue_peak", ctypes.c_int64),
                ("device_status", ctypes.c_int32), ("pad1", ctypes.c_int32),
                ("n_launches", ctypes.c_int64), ("narrow_bulk_ns", ctypes.c_int64),
                ("narrow_tail_ns", ctypes.c_int64), ("n_donated", ctypes.c_int64),
                ("n_intervals_tail", ctypes.c_int64), ("n_intervals_fp64", ctypes.c_int64),
                ("n_box_copies", ctypes.c_int64), ("n_ranges", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


class ccd_memory_model(ctypes.Structure):
    _fields_ = [("bytes_per_box", ctypes.c_int64), ("bytes_per_pair", ctypes.c_int64),
                ("bytes_per_scene", ctypes.c_int64), ("bytes_fixed", ctypes.c_int64)]


class ccd_server_opts(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("max_scenes", ctypes.c_int32), ("max_boxes", ctypes.c_int64),
                ("memory_cap", ctypes.c_int64), ("arena_bytes", ctypes.c_int64), ("delta", ctypes.c_double),
                ("min_sep", ctypes.c_double), ("max_iter", ctypes.c_int64), ("pairs_per_box", ctypes.c_double),
                ("autotune", ctypes.c_int32), ("pad", ctypes.c_int32)]


class ccd_server_stats(ctypes.Structure):
    _fields_ = [("n_submitted", ctypes.c_int64), ("n_done", ctypes.c_int64), ("n_batches", ctypes.c_int64),
                ("max_batch_scenes", ctypes.c_int64), ("sum_latency_ms", ctypes.c_double),
                ("max_batch_bytes", ctypes.c_int64), ("max_inflight_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ccd_tuning(ctypes.Structure):
    _fields_ = [("sweep_kernel", ctypes.c_int32), ("export_budget", ctypes.c_int32),
                ("strip_width", ctypes.c_double), ("queue_capacity", ctypes.c_int64),
                ("broad_ms", ctypes.c_double), ("narrow_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("n_trials", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


class CCDError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {ccd_status_str(status)} (status {status})")


_lib = None


def lib():
    """Load libccd.so (built by paper_2112_06300_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2112_06300_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.ccd_default_opts.argtypes = [ctypes.POINTER(ccd_opts)]
    L.ccd_default_opts.restype = None
    L.ccd_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ccd_opts), ctypes.c_int]
    L.ccd_destroy.argtypes = [P]
    L.ccd_broad.argtypes = [P, P, P, i64, P, i64, P, i64, P, i64, ctypes.POINTER(i64), P, i64,
                            ctypes.POINTER(i64), P]
    L.ccd_broad_shard.argtypes = [P, P, P, i64, P, i64, P, i64, i32, i32, P, i64, ctypes.POINTER(i64), P, i64,
                                  ctypes.POINTER(i64), P]
    L.ccd_narrow.argtypes = [P, P, i64, P, i64, P, P, i64, P, i64, P, i64, d, d, i64, i32,
                             P, P, P, P, P, P]
    L.ccd_step.argtypes = [P, P, P, i64, P, i64, P, i64, d, d, i64, P, P]
    L.ccd_get_status.argtypes = [P, ctypes.POINTER(ccd_stats)]
    L.ccd_status_str.argtypes = [ctypes.c_int]
    L.ccd_status_str.restype = ctypes.c_char_p
    L.ccd_measure_fp64_peak.argtypes = [ctypes.c_int, ctypes.POINTER(d)]
    L.ccd_stage_times.argtypes = [P, ctypes.POINTER(d)]
    L.ccd_step_batch.argtypes = [P, i32, P, P, P, P, P, i64, P, i64, P, i64, d, d, i64, P, P]
    L.ccd_step_batch.restype = ctypes.c_int
    L.ccd_narrow_noalloc.argtypes = [P, i64, P, i64, P, P, i64, P, i64, P, i64, d, d, i64, i32,
                                     P, P, P, P, P, P, P]
    L.ccd_narrow_noalloc.restype = ctypes.c_int
    L.ccd_autotune.argtypes = [P, P, P, i64, P, i64, P, i64, i32, ctypes.POINTER(ccd_tuning), P]
    L.ccd_autotune.restype = ctypes.c_int
    L.ccd_autotune_batch.argtypes = [P, i32, P, P, P, P, P, i64, P, i64, P, i64, i32, ctypes.POINTER(ccd_tuning), P]
    L.ccd_autotune_batch.restype = ctypes.c_int
    L.ccd_status_async.argtypes = [P, P, P]
    L.ccd_status_async.restype = ctypes.c_int
    L.ccd_selftest_unfinished_work.argtypes = [P, ctypes.POINTER(ctypes.c_int32), P]
    L.ccd_selftest_unfinished_work.restype = ctypes.c_int
    L.ccd_selftest_radix_sort.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_int32), P]
    L.ccd_selftest_radix_sort.restype = ctypes.c_int
    L.ccd_get_memory_model.argtypes = [ctypes.POINTER(ccd_opts), ctypes.POINTER(ccd_memory_model)]
    L.ccd_get_memory_model.restype = ctypes.c_int
    L.ccd_pair_capacity_for.argtypes = [ctypes.POINTER(ccd_opts), i64, i64, i32]
    L.ccd_pair_capacity_for.restype = ctypes.c_int64
    L.ccd_server_default_opts.argtypes = [ctypes.POINTER(ccd_server_opts)]
    L.ccd_server_default_opts.restype = None
    L.ccd_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ccd_server_opts), ctypes.c_int]
    L.ccd_server_create.restype = ctypes.c_int
    L.ccd_server_destroy.argtypes = [P]
    L.ccd_server_destroy.restype = ctypes.c_int
    PD, PI = ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
    L.ccd_server_request.argtypes = [P, i64, i64, i64, PD, PD, PI, PI, ctypes.POINTER(ctypes.c_uint64)]
    L.ccd_server_request.restype = ctypes.c_int
    L.ccd_server_submit.argtypes = [P, ctypes.c_uint64]
    L.ccd_server_submit.restype = ctypes.c_int
    L.ccd_server_submit_scene.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P, P,
                                          ctypes.POINTER(ctypes.c_uint64)]
    L.ccd_server_submit_scene.restype = ctypes.c_int
    L.ccd_server_wait.argtypes = [P, ctypes.c_uint64, d, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    L.ccd_server_wait.restype = ctypes.c_int
    L.ccd_server_get_stats.argtypes = [P, ctypes.POINTER(ccd_server_stats)]
    L.ccd_server_get_stats.restype = ctypes.c_int
    for f in ("ccd_create", "ccd_destroy", "ccd_broad", "ccd_narrow", "ccd_step", "ccd_get_status",
              "ccd_measure_fp64_peak", "ccd_stage_times"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, where: str):
    if rc != CCD_OK:
        raise CCDError(rc, where)


def ccd_status_str(status: int) -> str:
    return lib().ccd_status_str(int(status)).decode()


def ccd_default_opts() -> ccd_opts:
    o = ccd_opts()
    lib().ccd_default_opts(ctypes.byref(o))
    return o


def ccd_create(opts: Optional[ccd_opts] = None, device: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().ccd_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None, device),
           "ccd_create")
    return h


def ccd_destroy(ctx) -> None:
    _check(lib().ccd_destroy(ctx), "ccd_destroy")


def _mesh(V0, V1, E, F):
    nV = V0.shape[1] if V0.numel() else 0
    assert V0.dtype == V1.dtype and V0.shape == V1.shape and V0.is_contiguous() and V1.is_contiguous()
    assert E.is_contiguous() and F.is_contiguous()
    return nV, E.shape[0], F.shape[0]


def ccd_broad(ctx, V0, V1, E, F, vf_out, ee_out, stream=None, check=True) -> Tuple[int, int, int]:
    """Broad phase into caller buffers; returns (status, n_vf, n_ee) totals."""
    nV, nE, nF = _mesh(V0, V1, E, F)
    nvf, nee = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().ccd_broad(ctx, _ptr(V0), _ptr(V1), nV, _ptr(E), nE, _ptr(F), nF,
                         _ptr(vf_out), vf_out.shape[0], ctypes.byref(nvf),
                         _ptr(ee_out), ee_out.shape[0], ctypes.byref(nee), _stream(stream))
    if check and rc not in (CCD_OK, CCD_ETRUNC):
        raise CCDError(rc, "ccd_broad")
    return rc, nvf.value, nee.value


def ccd_broad_shard(ctx, V0, V1, E, F, shard, n_shards, vf_out, ee_out, stream=None, check=True) -> Tuple[int, int, int]:
    """One shard of the broad phase into caller buffers; returns (status,
    n_vf, n_ee) totals of the shard."""
    nV, nE, nF = _mesh(V0, V1, E, F)
    nvf, nee = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().ccd_broad_shard(ctx, _ptr(V0), _ptr(V1), nV, _ptr(E), nE, _ptr(F), nF, int(shard), int(n_shards),
                               _ptr(vf_out), vf_out.shape[0], ctypes.byref(nvf),
                               _ptr(ee_out), ee_out.shape[0], ctypes.byref(nee), _stream(stream))
    if check and rc not in (CCD_OK, CCD_ETRUNC):
        raise CCDError(rc, "ccd_broad_shard")
    return rc, nvf.value, nee.value


def ccd_narrow(ctx, vf, ee, V0, V1, E, F, delta, min_sep, max_iter, mode,
               toi_vf, toi_ee, flags_vf, flags_ee, toi_min, stream=None) -> None:
    nV, nE, nF = _mesh(V0, V1, E, F)
    rc = lib().ccd_narrow(ctx, _ptr(vf), vf.shape[0], _ptr(ee), ee.shape[0], _ptr(V0), _ptr(V1), nV,
                          _ptr(E), nE, _ptr(F), nF, float(delta), float(min_sep), int(max_iter), int(mode),
                          _ptr(toi_vf), _ptr(toi_ee), _ptr(flags_vf), _ptr(flags_ee), _ptr(toi_min),
                          _stream(stream))
    _check(rc, "ccd_narrow")


def ccd_narrow_noalloc(vf, ee, V0, V1, E, F, delta, min_sep, max_iter, mode,
                       toi_vf, toi_ee, flags_vf, flags_ee, toi_min, status, stream=None) -> None:
    """Narrow phase with no device allocation (fixed scratch inside the
    library, at most 65536 pairs per call); `status` is a CUDA int32 tensor of
    one element that receives the device status."""
    nV, nE, nF = _mesh(V0, V1, E, F)
    rc = lib().ccd_narrow_noalloc(_ptr(vf), vf.shape[0], _ptr(ee), ee.shape[0], _ptr(V0), _ptr(V1), nV,
                                  _ptr(E), nE, _ptr(F), nF, float(delta), float(min_sep), int(max_iter),
                                  int(mode), _ptr(toi_vf), _ptr(toi_ee), _ptr(flags_vf), _ptr(flags_ee),
                                  _ptr(toi_min), _ptr(status), _stream(stream))
    _check(rc, "ccd_narrow_noalloc")


def ccd_step(ctx, V0, V1, E, F, delta, min_sep, max_iter, toi_min, stream=None) -> int:
    """toi_min: a CUDA float64 tensor of one element (asynchronous) or a numpy
    float64 array of one element (synchronous; returns the device status)."""
    nV, nE, nF = _mesh(V0, V1, E, F)
    if isinstance(toi_min, np.ndarray):
        assert toi_min.dtype == np.float64 and toi_min.size >= 1 and toi_min.flags.c_contiguous
        out = toi_min.ctypes.data_as(ctypes.c_void_p)
    else:
        out = _ptr(toi_min)
    rc = lib().ccd_step(ctx, _ptr(V0), _ptr(V1), nV, _ptr(E), nE, _ptr(F), nF, float(delta), float(min_sep),
                        int(max_iter), out, _stream(stream))
    if rc not in (CCD_OK,):
        raise CCDError(rc, "ccd_step")
    return rc


def ccd_step_batch(ctx, vert_off, edge_off, face_off, V0, V1, E, F, delta, min_sep, max_iter, toi_out,
                   stream=None) -> None:
    """Batched step; offsets are CUDA int64 tensors of n_scenes + 1 entries,
    toi_out a CUDA float64 tensor of n_scenes entries (asynchronous)."""
    nV, nE, nF = _mesh(V0, V1, E, F)
    n = toi_out.shape[0]
    assert vert_off.shape[0] == n + 1 and edge_off.shape[0] == n + 1 and face_off.shape[0] == n + 1
    rc = lib().ccd_step_batch(ctx, n, _ptr(vert_off), _ptr(edge_off), _ptr(face_off), _ptr(V0), _ptr(V1), nV,
                              _ptr(E), nE, _ptr(F), nF, float(delta), float(min_sep), int(max_iter), _ptr(toi_out),
                              _stream(stream))
    _check(rc, "ccd_step_batch")


def ccd_autotune(ctx, V0, V1, E, F, reps=3, stream=None) -> dict:
    """Run the autotuner on one mesh (synchronous); returns the chosen
    settings and the median times."""
    nV, nE, nF = _mesh(V0, V1, E, F)
    out = ccd_tuning()
    rc = lib().ccd_autotune(ctx, _ptr(V0), _ptr(V1), nV, _ptr(E), nE, _ptr(F), nF, int(reps), ctypes.byref(out),
                            _stream(stream))
    _check(rc, "ccd_autotune")
    return out.as_dict()


def ccd_get_status(ctx) -> Tuple[int, dict]:
    st = ccd_stats()
    rc = lib().ccd_get_status(ctx, ctypes.byref(st))
    return rc, st.as_dict()


def ccd_selftest_unfinished_work(ctx, stream=None) -> int:
    """Device status the narrow kernel leaves when one unit can never
    finish (CCD_ETIMEOUT when detection works); synchronous."""
    st = ctypes.c_int32()
    _check(lib().ccd_selftest_unfinished_work(ctx, ctypes.byref(st), _stream(stream)), "ccd_selftest_unfinished_work")
    return st.value


def ccd_selftest_radix_sort(ctx, keys, vals, key_bits=0, n_cap=None, skip_all=False, stream=None) -> int:
    """Sort device tensors keys (int32/uint32 or int64/uint64, n) and vals
    (int32/uint32, n) in place with the broad phase's radix sort, stably by
    the low key_bits bits (0: all); n_cap > n passes the count through
    device memory; skip_all skips every pass of a digit all keys share (the
    cell sort's mode).  Returns the device status; synchronous."""
    n = keys.numel()
    assert vals.numel() == n and keys.is_contiguous() and vals.is_contiguous() and vals.element_size() == 4
    st = ctypes.c_int32()
    _check(lib().ccd_selftest_radix_sort(ctx, keys.element_size(), key_bits, n, n if n_cap is None else n_cap,
                                         1 if skip_all else 0, _ptr(keys), _ptr(vals), ctypes.byref(st),
                                         _stream(stream)),
           "ccd_selftest_radix_sort")
    return st.value


STAGES = ("boxes", "sort", "sweep", "narrow", "narrow_kernel")


def ccd_stage_times(ctx) -> dict:
    ms = (ctypes.c_double * len(STAGES))()
    _check(lib().ccd_stage_times(ctx, ms), "ccd_stage_times")
    return dict(zip(STAGES, list(ms)))


def ccd_measure_fp64_peak(device: int = 0) -> float:
    g = ctypes.c_double()
    _check(lib().ccd_measure_fp64_peak(device, ctypes.byref(g)), "ccd_measure_fp64_peak")
    return g.value


# ----------------------------------------------------------------------------
# Convenience layer over the same calls.
# ----------------------------------------------------------------------------

def mesh_to_device(V0, V1, E, F, device="cuda"):
    """numpy (nV, 3) / (nE, 2) / (nF, 3) arrays -> device tensors in the
    library's layout (positions transposed to (3, nV))."""
    import torch
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
    V0d = t(np.asarray(V0, np.float64).T, torch.float64).contiguous()
    V1d = t(np.asarray(V1, np.float64).T, torch.float64).contiguous()
    Ed = t(np.asarray(E, np.int32).reshape(-1, 2), torch.int32)
    Fd = t(np.asarray(F, np.int32).reshape(-1, 3), torch.int32)
    return V0d, V1d, Ed, Fd


@dataclass
class NarrowResult:
    toi_vf: "object"
    toi_ee: "object"
    flags_vf: "object"
    flags_ee: "object"
    toi_min: float


class CCD:
    """A context on one GPU with the library's calls as methods."""

    def __init__(self, device: int = 0, **opts):
        o = ccd_default_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        self.opts = o
        self.device = device
        self.ctx = ccd_create(o, device)

    def close(self):
        if self.ctx:
            ccd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def broad(self, V0, V1, E, F, stream=None):
        """Candidate pairs as int32 CUDA tensors (vf (n, 2), ee (m, 2)),
        unordered; sized with one retry when the first guess is too small."""
        import torch
        dev = V0.device
        cap = max(1024, 4 * (V0.shape[1] + E.shape[0] + F.shape[0]))
        for _ in range(2):
            vf = torch.empty((cap, 2), dtype=torch.int32, device=dev)
            ee = torch.empty((cap, 2), dtype=torch.int32, device=dev)
            rc, nvf, nee = ccd_broad(self.ctx, V0, V1, E, F, vf, ee, stream)
            if rc == CCD_OK:
                return vf[:nvf], ee[:nee]
            cap = max(nvf, nee) + 1
        raise CCDError(CCD_ETRUNC, "CCD.broad")

    def broad_shard(self, V0, V1, E, F, shard, n_shards, stream=None):
        """Pairs of one shard of the broad phase (ccd_broad_shard) as int32
        CUDA tensors (vf, ee)."""
        import torch
        dev = V0.device
        cap = max(1024, 4 * (V0.shape[1] + E.shape[0] + F.shape[0]))
        for _ in range(2):
            vf = torch.empty((cap, 2), dtype=torch.int32, device=dev)
            ee = torch.empty((cap, 2), dtype=torch.int32, device=dev)
            rc, nvf, nee = ccd_broad_shard(self.ctx, V0, V1, E, F, shard, n_shards, vf, ee, stream)
            if rc == CCD_OK:
                return vf[:nvf], ee[:nee]
            cap = max(nvf, nee) + 1
        raise CCDError(CCD_ETRUNC, "CCD.broad_shard")

    def narrow(self, vf, ee, V0, V1, E, F, delta=None, min_sep=None, max_iter=None, mode=0, stream=None):
        import torch
        dev = V0.device
        delta = self.opts.delta if delta is None else delta
        min_sep = self.opts.min_sep if min_sep is None else min_sep
        max_iter = self.opts.max_iter if max_iter is None else max_iter
        tv = torch.empty(vf.shape[0], dtype=torch.float64, device=dev)
        te = torch.empty(ee.shape[0], dtype=torch.float64, device=dev)
        fv = torch.empty(vf.shape[0], dtype=torch.uint8, device=dev)
        fe = torch.empty(ee.shape[0], dtype=torch.uint8, device=dev)
        tm = torch.empty(1, dtype=torch.float64, device=dev)
        ccd_narrow(self.ctx, vf, ee, V0, V1, E, F, delta, min_sep, max_iter, mode, tv, te, fv, fe, tm, stream)
        rc, _ = ccd_get_status(self.ctx)
        _check(rc, "ccd_narrow (device)")
        return NarrowResult(tv, te, fv, fe, float(tm.item()))

    def step(self, V0, V1, E, F, delta=None, min_sep=None, max_iter=None, stream=None) -> float:
        out = np.empty(1, np.float64)
        ccd_step(self.ctx, V0, V1, E, F,
                 self.opts.delta if delta is None else delta,
                 self.opts.min_sep if min_sep is None else min_sep,
                 self.opts.max_iter if max_iter is None else max_iter, out, stream)
        return float(out[0])

    def step_batch(self, scenes_list, delta=None, min_sep=None, max_iter=None, stream=None):
        """Earliest time of every scene of a list (scenes.Scene), one batched
        step; returns a numpy array and checks the device status."""
        import torch
        from . import scenes as S
        V0, V1, E, F, vo, eo, fo = S.concat_scenes(scenes_list)
        dev = f"cuda:{self.device}"
        V0d, V1d, Ed, Fd = mesh_to_device(V0, V1, E, F, dev)
        t = lambda a: torch.from_numpy(a).to(dev)
        out = torch.empty(len(scenes_list), dtype=torch.float64, device=dev)
        ccd_step_batch(self.ctx, t(vo), t(eo), t(fo), V0d, V1d, Ed, Fd,
                       self.opts.delta if delta is None else delta,
                       self.opts.min_sep if min_sep is None else min_sep,
                       self.opts.max_iter if max_iter is None else max_iter, out, stream)
        rc, _ = ccd_get_status(self.ctx)
        _check(rc, "ccd_step_batch (device)")
        return out.cpu().numpy()

    def autotune(self, V0, V1, E, F, reps=3, stream=None):
        """Pick the sweep, cell width, hand-off budget and queue capacity for
        this mesh (kept in the context)."""
        return ccd_autotune(self.ctx, V0, V1, E, F, reps, stream)

    def status(self):
        return ccd_get_status(self.ctx)

    def stage_times(self):
        return ccd_stage_times(self.ctx)


def ccd_get_memory_model(opts: Optional[ccd_opts] = None) -> dict:
    m = ccd_memory_model()
    _check(lib().ccd_get_memory_model(ctypes.byref(opts) if opts is not None else None, ctypes.byref(m)),
           "ccd_get_memory_model")
    return {k: getattr(m, k) for k, _ in m._fields_}


def ccd_pair_capacity_for(mem_bytes: int, n_boxes: int, n_scenes: int = 0, opts: Optional[ccd_opts] = None) -> int:
    return int(lib().ccd_pair_capacity_for(ctypes.byref(opts) if opts is not None else None, int(mem_bytes),
                                           int(n_boxes), int(n_scenes)))


class Server:
    """Serving runtime (ccd_server_*): scenes are written into the server's
    pinned arena, queued, batched by its scheduler thread and completed
    asynchronously."""

    def __init__(self, device: int = 0, **opts):
        o = ccd_server_opts()
        lib().ccd_server_default_opts(ctypes.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown server option {k}")
            setattr(o, k, v)
        self.opts = o
        self.handle = ctypes.c_void_p()
        _check(lib().ccd_server_create(ctypes.byref(self.handle), ctypes.byref(o), device), "ccd_server_create")

    def request(self, nV: int, nE: int, nF: int):
        """Arena space for one scene: returns (ticket, V0 (3, nV), V1 (3, nV),
        E (nE, 2), F (nF, 3)) as numpy views to fill."""
        pv0, pv1 = ctypes.POINTER(ctypes.c_double)(), ctypes.POINTER(ctypes.c_double)()
        pe, pf = ctypes.POINTER(ctypes.c_int32)(), ctypes.POINTER(ctypes.c_int32)()
        t = ctypes.c_uint64()
        _check(lib().ccd_server_request(self.handle, nV, nE, nF, ctypes.byref(pv0), ctypes.byref(pv1),
                                        ctypes.byref(pe), ctypes.byref(pf), ctypes.byref(t)), "ccd_server_request")
        view = lambda p, shape: np.ctypeslib.as_array(p, shape=shape) if shape[0] * shape[1] else \
            np.zeros(shape, np.float64 if p._type_ is ctypes.c_double else np.int32)
        return (t.value, view(pv0, (3, nV)), view(pv1, (3, nV)), view(pe, (nE, 2)), view(pf, (nF, 3)))

    def submit_scene(self, V0, V1, E, F) -> int:
        """Copy one scene ((nV, 3) positions, local (nE, 2) / (nF, 3) ids) into
        the arena and queue it; returns its ticket."""
        t, v0, v1, e, f = self.request(len(V0), len(E), len(F))
        if len(V0):
            v0[...] = np.asarray(V0, np.float64).T
            v1[...] = np.asarray(V1, np.float64).T
        if len(E):
            e[...] = E
        if len(F):
            f[...] = F
        _check(lib().ccd_server_submit(self.handle, t), "ccd_server_submit")
        return t

    def submit_soa(self, V0T, V1T, E, F) -> int:
        """Queue one scene given in the arena's layout (V0T, V1T float64 (3, nV)
        C-contiguous, E int32 (nE, 2), F int32 (nF, 3)): the library copies it
        into the arena and submits it in one call; returns the ticket."""
        t = ctypes.c_uint64()
        nV, nE, nF = V0T.shape[1], E.shape[0], F.shape[0]
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None
        _check(lib().ccd_server_submit_scene(self.handle, nV, nE, nF, p(V0T), p(V1T), p(E), p(F), ctypes.byref(t)),
               "ccd_server_submit_scene")
        return t.value

    def submit(self, ticket: int) -> None:
        _check(lib().ccd_server_submit(self.handle, ticket), "ccd_server_submit")

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        """(earliest time, latency in ms) of a submitted scene; raises on a
        device error."""
        toi, lat = ctypes.c_double(), ctypes.c_double()
        rc = lib().ccd_server_wait(self.handle, ticket, float(timeout_ms), ctypes.byref(toi), ctypes.byref(lat))
        _check(rc, "ccd_server_wait")
        return toi.value, lat.value

    def stats(self) -> dict:
        st = ccd_server_stats()
        rc = lib().ccd_server_get_stats(self.handle, ctypes.byref(st))
        _check(rc, "ccd_server_get_stats")
        return st.as_dict()

    def close(self) -> None:
        if self.handle:
            lib().ccd_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
