"""GB300-native Continuous Visual Odometry (CVO, arXiv 1904.02266).

Thin ctypes binding over ``libcvo.so``, whose C ABI is declared in
``include/cvo.h``. Every step of the solve runs in the library's CUDA kernels;
this module only marshals arguments. Functions named like the C entry points
(``cvo_create``, ``cvo_set_cloud``, ``cvo_eval``, ``cvo_align``, ...) map one
to one onto them; ``Context`` wraps them for convenience.

Host arrays (numpy) are copied by the library; CUDA tensors (torch) are passed
as device pointers with the current torch stream. There is no fallback: if the
library has not been built, importing the binding works but the first call
raises ``CvoUnavailable``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB as LIB_PATH

CVO_OK = 0
CVO_ERR_INVALID_ARG = -1
CVO_ERR_OUT_OF_BUDGET = -2
CVO_ERR_CUDA = -3
CVO_ERR_TIMEOUT = -4
CVO_ERR_BUSY = -5
CVO_ERR_NOT_FOUND = -6
CVO_ERR_INTERNAL = -7

CVO_COLOR_NONE, CVO_COLOR_KERNEL, CVO_COLOR_DOT = 0, 1, 2
CVO_SCHEDULE_DECAY, CVO_SCHEDULE_TABLE1 = 0, 1
CVO_DEVICE_PTR = 1
CVO_MAX_FEAT = 8

# every entry point declared in include/cvo.h
EXPORTS = ("cvo_params_default", "cvo_create", "cvo_destroy", "cvo_set_cloud",
           "cvo_release_cloud", "cvo_eval", "cvo_align", "cvo_align_profile",
           "cvo_set_wait_limits", "cvo_stream",
           "cvo_batch_create", "cvo_batch_run", "cvo_batch_get_info", "cvo_batch_destroy",
           "cvo_serve_params_default", "cvo_serve_start", "cvo_submit", "cvo_poll",
           "cvo_serve_stop", "cvo_serve_get_stats", "cvo_frontend_params_default",
           "cvo_frontend_select", "cvo_frontend_cloud", "cvo_autotune",
           "cvo_eval_gradient_static", "cvo_strerror", "cvo_last_error")


class CvoUnavailable(RuntimeError):
    """libcvo.so is missing or cannot be loaded."""


class CvoError(RuntimeError):
    def __init__(self, code, detail=""):
        self.code = code
        super().__init__(f"{strerror(code)} ({code}): {detail}" if detail else strerror(code))


class cvo_params(ctypes.Structure):
    _fields_ = [("ell0", ctypes.c_double), ("ell_decay", ctypes.c_double),
                ("ell_min", ctypes.c_double), ("schedule", ctypes.c_int),
                ("sigma", ctypes.c_double), ("kcut", ctypes.c_double),
                ("color_mode", ctypes.c_int), ("ell_color", ctypes.c_double),
                ("color_scale", ctypes.c_double), ("a2", ctypes.c_double),
                ("b2", ctypes.c_double), ("max_iters", ctypes.c_int),
                ("eps_pose", ctypes.c_double), ("eps_grad", ctypes.c_double),
                ("step_order", ctypes.c_int), ("feat_dim", ctypes.c_int),
                ("feat_bf16", ctypes.c_int), ("reduce_fp32", ctypes.c_int),
                ("cell_factor", ctypes.c_double), ("cluster_factor", ctypes.c_double),
                ("cost_chunk", ctypes.c_int), ("cost_cluster", ctypes.c_int),
                ("cost_kept", ctypes.c_double), ("team_factor", ctypes.c_double),
                ("wait_polls", ctypes.c_int), ("join_limit_ms", ctypes.c_double)]


class cvo_eval_result(ctypes.Structure):
    _fields_ = [("F", ctypes.c_double), ("grad6", ctypes.c_double * 6),
                ("S", ctypes.c_double * 5), ("nnz", ctypes.c_int64),
                ("candidates", ctypes.c_int64)]


class cvo_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("fallback_steps", ctypes.c_int), ("no_ascent_steps", ctypes.c_int),
                ("final_ell", ctypes.c_double), ("F_last", ctypes.c_double),
                ("t_last", ctypes.c_double), ("pair_evals", ctypes.c_int64),
                ("candidates", ctypes.c_int64), ("status", ctypes.c_int),
                ("device_ms", ctypes.c_double)]


class cvo_iter_profile(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_double), ("plan_ms", ctypes.c_float), ("grad_ms", ctypes.c_float),
                ("step_ms", ctypes.c_float), ("grad_pass_ms", ctypes.c_float),
                ("grad_sync_ms", ctypes.c_float), ("step_pass_ms", ctypes.c_float),
                ("step_sync_ms", ctypes.c_float), ("replanned", ctypes.c_int),
                ("grad_pairs", ctypes.c_int64),
                ("step_pairs", ctypes.c_int64), ("grad_candidates", ctypes.c_int64),
                ("step_candidates", ctypes.c_int64)]


class cvo_batch_info(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int), ("blocks", ctypes.c_int), ("graph", ctypes.c_int),
                ("max_team", ctypes.c_int), ("bytes", ctypes.c_int64)]


class cvo_request(ctypes.Structure):
    _fields_ = [("target", ctypes.c_int32), ("xyz", ctypes.c_void_p), ("feat", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("P0", ctypes.c_double * 16), ("ell0", ctypes.c_double)]


class cvo_result(ctypes.Structure):
    _fields_ = [("P", ctypes.c_double * 16), ("stats", cvo_stats), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class cvo_serve_params(ctypes.Structure):
    _fields_ = [("reserve_blocks", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("linger_ms", ctypes.c_double), ("idle_limit_ms", ctypes.c_double),
                ("team_factor", ctypes.c_double)]


class cvo_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("kernels_launched", ctypes.c_int64),
                ("idle_exits", ctypes.c_int64)]


class cvo_tune_space(ctypes.Structure):
    _fields_ = [("n_cell", ctypes.c_int), ("n_cluster", ctypes.c_int), ("n_chunk", ctypes.c_int),
                ("n_cluster_cost", ctypes.c_int), ("cell_factor", ctypes.c_double * 8),
                ("cluster_factor", ctypes.c_double * 8), ("cost_chunk", ctypes.c_int * 8),
                ("cost_cluster", ctypes.c_int * 8), ("reps", ctypes.c_int)]


class cvo_tune_report(ctypes.Structure):
    _fields_ = [("start_ms", ctypes.c_double), ("best_ms", ctypes.c_double),
                ("candidates", ctypes.c_int), ("cell_factor", ctypes.c_double),
                ("cluster_factor", ctypes.c_double), ("cost_chunk", ctypes.c_int),
                ("cost_cluster", ctypes.c_int)]


class cvo_frontend_params(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("depth_min", ctypes.c_double),
                ("depth_max", ctypes.c_double), ("percentile", ctypes.c_double),
                ("grad_scale", ctypes.c_double), ("max_points", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libcvo.so and declare its signatures. Raises CvoUnavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise CvoUnavailable(f"{path} is not built; run __graft_entry__.build() "
                                 f"(or python -m paper_1904_02266_gb300.build)")
        try:
            lib = ctypes.CDLL(path)
        except OSError as e:
            raise CvoUnavailable(f"cannot load {path}: {e}") from e
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        lib.cvo_params_default.argtypes = [ctypes.POINTER(cvo_params)]
        lib.cvo_params_default.restype = None
        lib.cvo_create.argtypes = [ctypes.POINTER(cvo_params), ctypes.c_int, ctypes.c_size_t,
                                   ctypes.POINTER(vp)]
        lib.cvo_destroy.argtypes = [vp]
        lib.cvo_set_cloud.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_uint32, vp,
                                      ctypes.POINTER(ctypes.c_int32)]
        lib.cvo_release_cloud.argtypes = [vp, ctypes.c_int32]
        lib.cvo_eval.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, dp, ctypes.c_double,
                                 ctypes.POINTER(cvo_eval_result)]
        lib.cvo_align.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, dp, dp,
                                  ctypes.POINTER(cvo_stats)]
        lib.cvo_set_wait_limits.argtypes = [vp, ctypes.c_int, ctypes.c_double]
        lib.cvo_set_wait_limits.restype = ctypes.c_int
        lib.cvo_align_profile.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, dp, dp,
                                          ctypes.POINTER(cvo_stats),
                                          ctypes.POINTER(cvo_iter_profile), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]
        lib.cvo_align_profile.restype = ctypes.c_int
        lib.cvo_eval_gradient_static.argtypes = [vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64,
                                                 ctypes.POINTER(cvo_params), dp, ctypes.c_double,
                                                 vp, vp]
        lib.cvo_eval_gradient_static.restype = ctypes.c_int
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.cvo_batch_create.argtypes = [vp, ctypes.c_int, i32p, i32p, dp, i32p,
                                         ctypes.POINTER(vp)]
        lib.cvo_batch_run.argtypes = [vp, vp, dp, dp, ctypes.POINTER(cvo_stats)]
        lib.cvo_batch_get_info.argtypes = [vp, vp, ctypes.POINTER(cvo_batch_info), i32p]
        lib.cvo_batch_destroy.argtypes = [vp, vp]
        lib.cvo_serve_params_default.argtypes = [ctypes.POINTER(cvo_serve_params)]
        lib.cvo_serve_params_default.restype = None
        lib.cvo_serve_start.argtypes = [vp, ctypes.POINTER(cvo_serve_params)]
        lib.cvo_submit.argtypes = [vp, ctypes.POINTER(cvo_request), ctypes.POINTER(ctypes.c_uint64)]
        lib.cvo_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(cvo_result),
                                 ctypes.POINTER(ctypes.c_int)]
        lib.cvo_serve_stop.argtypes = [vp]
        lib.cvo_serve_get_stats.argtypes = [vp, ctypes.POINTER(cvo_serve_stats)]
        fpp = ctypes.POINTER(cvo_frontend_params)
        lib.cvo_frontend_params_default.argtypes = [fpp]
        lib.cvo_frontend_params_default.restype = None
        lib.cvo_frontend_select.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, fpp,
                                            ctypes.c_uint32, vp, vp, vp, vp, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int64)]
        lib.cvo_frontend_cloud.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, fpp,
                                           ctypes.c_uint32, vp, i32p,
                                           ctypes.POINTER(ctypes.c_int64)]
        lib.cvo_autotune.argtypes = [vp, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(cvo_tune_space),
                                     ctypes.POINTER(cvo_tune_report)]
        lib.cvo_stream.argtypes = [vp]
        lib.cvo_stream.restype = ctypes.c_void_p
        lib.cvo_strerror.argtypes = [ctypes.c_int]
        lib.cvo_strerror.restype = ctypes.c_char_p
        lib.cvo_last_error.argtypes = [vp]
        lib.cvo_last_error.restype = ctypes.c_char_p
        for name in ("cvo_create", "cvo_destroy", "cvo_set_cloud", "cvo_release_cloud",
                     "cvo_eval", "cvo_align", "cvo_batch_create", "cvo_batch_run",
                     "cvo_batch_get_info", "cvo_batch_destroy", "cvo_serve_start",
                     "cvo_submit", "cvo_poll", "cvo_serve_stop", "cvo_serve_get_stats",
                     "cvo_frontend_select", "cvo_frontend_cloud", "cvo_autotune"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load_library().cvo_strerror(int(code)).decode()
    except CvoUnavailable:
        return f"status {code}"


def _check(ctx, code):
    if code != CVO_OK:
        detail = load_library().cvo_last_error(ctx).decode() if ctx else ""
        raise CvoError(code, detail)


def _pose(P):
    a = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(4, 4))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# one function per C entry point
# ---------------------------------------------------------------------------

def cvo_params_default() -> cvo_params:
    p = cvo_params()
    load_library().cvo_params_default(ctypes.byref(p))
    return p


def cvo_create(params: cvo_params | None = None, device: int = 0, hbm_budget_bytes: int = 0):
    lib = load_library()
    out = ctypes.c_void_p()
    code = lib.cvo_create(ctypes.byref(params) if params is not None else None, int(device),
                          int(hbm_budget_bytes), ctypes.byref(out))
    _check(None, code)
    return out


def cvo_destroy(ctx) -> None:
    _check(None, load_library().cvo_destroy(ctx))


def cvo_set_cloud(ctx, xyz, feat=None, n=None, flags=0, stream=None) -> int:
    """xyz: (n, 3) float32; feat: (n, D) float32 or None. numpy arrays are host
    buffers; objects with ``data_ptr()`` and ``is_cuda`` (torch tensors) are
    passed as device pointers."""
    keep = []

    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
            if not a.is_contiguous() or str(a.dtype) != "torch.float32":
                raise ValueError("device arrays must be contiguous float32")
            return a.data_ptr()
        arr = np.ascontiguousarray(a, dtype=np.float32)
        keep.append(arr)
        return arr.ctypes.data

    dev = hasattr(xyz, "data_ptr") and getattr(xyz, "is_cuda", False)
    if dev:
        flags |= CVO_DEVICE_PTR
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(xyz.device).cuda_stream
    n = int(xyz.shape[0]) if n is None else int(n)
    h = ctypes.c_int32(-1)
    code = load_library().cvo_set_cloud(ctx, ptr(xyz), ptr(feat), n, int(flags),
                                        stream if stream else None, ctypes.byref(h))
    _check(ctx, code)
    return int(h.value)


def cvo_release_cloud(ctx, handle: int) -> None:
    _check(ctx, load_library().cvo_release_cloud(ctx, int(handle)))


def cvo_eval(ctx, target: int, source: int, P, ell: float) -> dict:
    _, pp = _pose(P)
    r = cvo_eval_result()
    _check(ctx, load_library().cvo_eval(ctx, int(target), int(source), pp, float(ell),
                                        ctypes.byref(r)))
    return {"F": r.F, "grad6": np.array(r.grad6[:]), "S": np.array(r.S[:]), "nnz": int(r.nnz),
            "candidates": int(r.candidates)}


def cvo_align(ctx, target: int, source: int, P0=None):
    _, p0 = _pose(np.eye(4) if P0 is None else P0)
    out = np.zeros((4, 4))
    st = cvo_stats()
    _check(ctx, load_library().cvo_align(ctx, int(target), int(source), p0,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(st)))
    stats = {k: getattr(st, k) for k, _ in cvo_stats._fields_}
    return out, stats


def cvo_set_wait_limits(ctx, wait_polls: int, join_limit_ms: float) -> None:
    _check(ctx, load_library().cvo_set_wait_limits(ctx, int(wait_polls), float(join_limit_ms)))


def cvo_align_profile(ctx, target: int, source: int, P0=None, max_records: int = 1000):
    """cvo_align with per-iteration CUDA-event timings of both pair passes."""
    _, p0 = _pose(np.eye(4) if P0 is None else P0)
    out = np.zeros((4, 4))
    st = cvo_stats()
    recs = (cvo_iter_profile * max(1, max_records))()
    nrec = ctypes.c_int(0)
    _check(ctx, load_library().cvo_align_profile(
        ctx, int(target), int(source), p0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        ctypes.byref(st), recs, int(max_records), ctypes.byref(nrec)))
    stats = {k: getattr(st, k) for k, _ in cvo_stats._fields_}
    records = [{k: getattr(recs[i], k) for k, _ in cvo_iter_profile._fields_}
               for i in range(nrec.value)]
    return out, stats, records


def _i32(a):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def cvo_batch_create(ctx, targets, sources, ell0=None, team_sizes=None):
    """Batch of len(targets) solves; returns the opaque batch pointer."""
    t, tp = _i32(targets)
    s, sp = _i32(sources)
    if t.shape != s.shape:
        raise ValueError("targets and sources differ in length")
    e = None if ell0 is None else np.ascontiguousarray(np.asarray(ell0, dtype=np.float64))
    g = None if team_sizes is None else _i32(team_sizes)
    out = ctypes.c_void_p()
    _check(ctx, load_library().cvo_batch_create(
        ctx, int(t.size), tp, sp,
        None if e is None else e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        None if g is None else g[1], ctypes.byref(out)))
    return out


def cvo_batch_run(ctx, batch, P0, check: bool = True):
    """P0: (n, 4, 4). Returns (poses (n, 4, 4), list of per-pair stats dicts);
    with check=False a failed run returns (poses, stats, status code) instead
    of raising, so that the per-pair statuses can be read."""
    p0 = np.ascontiguousarray(np.asarray(P0, dtype=np.float64))
    n = p0.shape[0]
    out = np.zeros((n, 4, 4))
    st = (cvo_stats * n)()
    code = load_library().cvo_batch_run(ctx, batch,
                                        p0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), st)
    stats = [{k: getattr(st[i], k) for k, _ in cvo_stats._fields_} for i in range(n)]
    if not check:
        return out, stats, code
    _check(ctx, code)
    return out, stats


def cvo_batch_get_info(ctx, batch, n: int | None = None) -> dict:
    info = cvo_batch_info()
    _check(ctx, load_library().cvo_batch_get_info(ctx, batch, ctypes.byref(info), None))
    teams = np.zeros(info.pairs, dtype=np.int32)
    _check(ctx, load_library().cvo_batch_get_info(
        ctx, batch, None, teams.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    d = {k: getattr(info, k) for k, _ in cvo_batch_info._fields_}
    d["teams"] = teams
    return d


def cvo_batch_destroy(ctx, batch) -> None:
    _check(ctx, load_library().cvo_batch_destroy(ctx, batch))


def cvo_serve_params_default() -> cvo_serve_params:
    p = cvo_serve_params()
    load_library().cvo_serve_params_default(ctypes.byref(p))
    return p


def cvo_serve_start(ctx, params: cvo_serve_params | None = None) -> None:
    _check(ctx, load_library().cvo_serve_start(
        ctx, ctypes.byref(params) if params is not None else None))


def cvo_submit(ctx, target: int, xyz, feat=None, P0=None, ell0: float = 0.0) -> int:
    """Queue the alignment of a frame (host arrays, copied) to a resident
    keyframe; returns the ticket."""
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    f = None if feat is None else np.ascontiguousarray(feat, dtype=np.float32)
    r = cvo_request()
    r.target = int(target)
    r.xyz = x.ctypes.data
    r.feat = None if f is None else f.ctypes.data
    r.n = int(x.shape[0])
    r.P0[:] = np.asarray(np.eye(4) if P0 is None else P0, dtype=np.float64).reshape(16)
    r.ell0 = float(ell0)
    t = ctypes.c_uint64(0)
    _check(ctx, load_library().cvo_submit(ctx, ctypes.byref(r), ctypes.byref(t)))
    return int(t.value)


def cvo_poll(ctx, ticket: int):
    """None while the request runs; else (pose, stats dict, queue_ms, latency_ms)."""
    out = cvo_result()
    done = ctypes.c_int(0)
    _check(ctx, load_library().cvo_poll(ctx, int(ticket), ctypes.byref(out), ctypes.byref(done)))
    if not done.value:
        return None
    stats = {k: getattr(out.stats, k) for k, _ in cvo_stats._fields_}
    return np.array(out.P[:]).reshape(4, 4), stats, out.queue_ms, out.latency_ms


def cvo_serve_stop(ctx) -> None:
    _check(ctx, load_library().cvo_serve_stop(ctx))


def cvo_serve_get_stats(ctx) -> dict:
    st = cvo_serve_stats()
    _check(ctx, load_library().cvo_serve_get_stats(ctx, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in cvo_serve_stats._fields_}


def cvo_frontend_params_default(**overrides) -> cvo_frontend_params:
    p = cvo_frontend_params()
    load_library().cvo_frontend_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _image_args(depth, hsv, stream):
    """Host numpy images, or CUDA tensors (device pointers, current torch stream)."""
    keep, flags = [], 0
    dev = hasattr(depth, "data_ptr") and getattr(depth, "is_cuda", False)
    if dev:
        flags |= CVO_DEVICE_PTR
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(depth.device).cuda_stream
        return depth.data_ptr(), hsv.data_ptr(), int(depth.shape[0]), int(depth.shape[1]), \
            flags, stream, keep
    d = np.ascontiguousarray(depth, dtype=np.float32)
    h = np.ascontiguousarray(hsv, dtype=np.float32)
    keep += [d, h]
    return d.ctypes.data, h.ctypes.data, d.shape[0], d.shape[1], flags, stream, keep


def cvo_frontend_select(ctx, depth, hsv, params: cvo_frontend_params, out_xyz, out_feat=None,
                        out_pixel=None, stream=None) -> int:
    """Selection into caller device tensors (float32 (cap, 3), (cap, 5), int32
    (cap,)); returns the number of points."""
    dp, hp, H, W, flags, stream, keep = _image_args(depth, hsv, stream)
    n = ctypes.c_int64(0)
    cap = int(out_xyz.shape[0])
    _check(ctx, load_library().cvo_frontend_select(
        ctx, dp, hp, W, H, ctypes.byref(params), flags, stream if stream else None,
        out_xyz.data_ptr(), None if out_feat is None else out_feat.data_ptr(),
        None if out_pixel is None else out_pixel.data_ptr(), cap, ctypes.byref(n)))
    return int(n.value)


def cvo_frontend_cloud(ctx, depth, hsv, params: cvo_frontend_params, stream=None):
    """The selection as a resident cloud: (handle, number of points)."""
    dp, hp, H, W, flags, stream, keep = _image_args(depth, hsv, stream)
    h = ctypes.c_int32(-1)
    n = ctypes.c_int64(0)
    _check(ctx, load_library().cvo_frontend_cloud(ctx, dp, hp, W, H, ctypes.byref(params), flags,
                                                  stream if stream else None, ctypes.byref(h),
                                                  ctypes.byref(n)))
    return int(h.value), int(n.value)


def cvo_autotune(ctx, target: int, source: int, space: cvo_tune_space | None = None) -> dict:
    """Time solves over the built-in (or given) candidates; the context keeps
    the fastest setting. Returns the report as a dict."""
    rep = cvo_tune_report()
    _check(ctx, load_library().cvo_autotune(ctx, int(target), int(source),
                                            ctypes.byref(space) if space is not None else None,
                                            ctypes.byref(rep)))
    return {k: getattr(rep, k) for k, _ in cvo_tune_report._fields_}


def _check_static_args(x, fx, z, fz, params: cvo_params, out):
    """Shapes, dtypes, layout and device of cvo_eval_gradient_static's tensor
    arguments, checked before anything is launched: the kernels read exactly
    n x 3 / m x 3 coordinates and n x feat_dim / m x feat_dim features, so a
    wrong shape or dtype would make them read past the end of a buffer.
    Raises ValueError."""
    def is_tensor(t):
        return hasattr(t, "data_ptr") and hasattr(t, "shape") and hasattr(t, "dtype")

    for name, t in (("x", x), ("z", z), ("out", out)):
        if not is_tensor(t):
            raise ValueError(f"{name} must be a torch tensor")
    if x.dim() != 2 or x.shape[1] != 3 or x.shape[0] < 1:
        raise ValueError(f"x must have shape (n, 3) with n >= 1, got {tuple(x.shape)}")
    if z.dim() != 2 or z.shape[1] != 3 or z.shape[0] < 1:
        raise ValueError(f"z must have shape (m, 3) with m >= 1, got {tuple(z.shape)}")
    n, m = int(x.shape[0]), int(z.shape[0])
    D = int(params.feat_dim)
    feats = params.color_mode != CVO_COLOR_NONE and D > 0
    if feats:
        for name, t, rows in (("fx", fx, n), ("fz", fz, m)):
            if not is_tensor(t):
                raise ValueError(f"{name} must be a torch tensor when features are used")
            if t.dim() != 2 or tuple(t.shape) != (rows, D):
                raise ValueError(f"{name} must have shape ({rows}, {D}), got {tuple(t.shape)}")
    used = [("x", x), ("z", z)] + ([("fx", fx), ("fz", fz)] if feats else [])
    for name, t in used:
        if str(t.dtype) != "torch.float32":
            raise ValueError(f"{name} must be float32, got {t.dtype}")
    if str(out.dtype) != "torch.float64" or out.numel() < 8:
        raise ValueError("out must be a float64 tensor of at least 8 elements")
    for name, t in used + [("out", out)]:
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if not getattr(t, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor")
    devs = {t.device for _, t in used + [("out", out)]}
    if len(devs) != 1:
        raise ValueError(f"all tensors must be on one device, got {sorted(map(str, devs))}")
    return n, m, feats


def cvo_eval_gradient_static(x, fx, z, fz, params: cvo_params, P, ell: float, out,
                             stream=None) -> None:
    """Allocation-free gradient pass on torch CUDA tensors: x (n, 3) and
    z (m, 3) float32, fx (n, feat_dim) and fz (m, feat_dim) float32 (ignored,
    may be None, when params.color_mode is NONE or feat_dim is 0), out a
    float64 tensor of at least 8 elements (F, grad6, kept pairs), all
    contiguous and on the current device. Written asynchronously on `stream`
    (default: torch's current stream). Argument errors raise ValueError
    before anything is launched."""
    n, m, feats = _check_static_args(x, fx, z, fz, params, out)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(x.device).cuda_stream
    _, pp = _pose(P)
    code = load_library().cvo_eval_gradient_static(
        x.data_ptr(), fx.data_ptr() if feats else None, n, z.data_ptr(),
        fz.data_ptr() if feats else None, m, ctypes.byref(params), pp, float(ell),
        out.data_ptr(), stream if stream else None)
    if code != CVO_OK:
        raise CvoError(code, load_library().cvo_last_error(None).decode())


def cvo_stream(ctx) -> int:
    """The context's cudaStream_t as an integer (for CUDA events on it)."""
    return int(load_library().cvo_stream(ctx) or 0)


def cvo_strerror(code: int) -> str:
    return strerror(code)


def cvo_last_error(ctx) -> str:
    return load_library().cvo_last_error(ctx).decode()


class Batch:
    """Many pair solves in one persistent launch (cvo_batch_*)."""

    def __init__(self, ctx: "Context", targets, sources, ell0=None, team_sizes=None):
        self._ctx = ctx
        self.n = len(targets)
        self.ptr = cvo_batch_create(ctx.ctx, targets, sources, ell0, team_sizes)

    def run(self, P0, check: bool = True):
        return cvo_batch_run(self._ctx.ctx, self.ptr, P0, check)

    def info(self) -> dict:
        return cvo_batch_get_info(self._ctx.ctx, self.ptr)

    def close(self) -> None:
        if self.ptr and self._ctx.ctx:
            cvo_batch_destroy(self._ctx.ctx, self.ptr)
        self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Context:
    """One library context: clouds, cached cell lists and solve plans on one GPU."""

    def __init__(self, params: cvo_params | None = None, device: int = 0, hbm_budget: int = 0,
                 **overrides):
        p = cvo_params_default() if params is None else params
        for k, v in overrides.items():
            if not hasattr(p, k):
                raise AttributeError(f"cvo_params has no field {k!r}")
            setattr(p, k, v)
        self.params = p
        self.ctx = cvo_create(p, device, hbm_budget)

    def set_cloud(self, xyz, feat=None, stream=None) -> int:
        return cvo_set_cloud(self.ctx, xyz, feat, stream=stream)

    def release(self, handle: int) -> None:
        cvo_release_cloud(self.ctx, handle)

    def eval(self, target: int, source: int, P, ell: float) -> dict:
        return cvo_eval(self.ctx, target, source, P, ell)

    def align(self, target: int, source: int, P0=None):
        return cvo_align(self.ctx, target, source, P0)

    def set_wait_limits(self, wait_polls: int, join_limit_ms: float) -> None:
        cvo_set_wait_limits(self.ctx, wait_polls, join_limit_ms)

    def align_profile(self, target: int, source: int, P0=None, max_records: int = 1000):
        return cvo_align_profile(self.ctx, target, source, P0, max_records)

    def batch(self, targets, sources, ell0=None, team_sizes=None) -> "Batch":
        return Batch(self, targets, sources, ell0, team_sizes)

    def serve_start(self, **params) -> None:
        p = cvo_serve_params_default()
        for k, v in params.items():
            setattr(p, k, v)
        cvo_serve_start(self.ctx, p)

    def submit(self, target: int, xyz, feat=None, P0=None, ell0: float = 0.0) -> int:
        return cvo_submit(self.ctx, target, xyz, feat, P0, ell0)

    def poll(self, ticket: int):
        return cvo_poll(self.ctx, ticket)

    def serve_stop(self) -> None:
        cvo_serve_stop(self.ctx)

    def serve_stats(self) -> dict:
        return cvo_serve_get_stats(self.ctx)

    def frontend_select(self, depth, hsv, params, out_xyz, out_feat=None, out_pixel=None,
                        stream=None) -> int:
        return cvo_frontend_select(self.ctx, depth, hsv, params, out_xyz, out_feat, out_pixel,
                                   stream)

    def autotune(self, target: int, source: int, space=None) -> dict:
        rep = cvo_autotune(self.ctx, target, source, space)
        for k in ("cell_factor", "cluster_factor", "cost_chunk", "cost_cluster"):
            setattr(self.params, k, rep[k])
        return rep

    def frontend_cloud(self, depth, hsv, params, stream=None):
        return cvo_frontend_cloud(self.ctx, depth, hsv, params, stream)

    @property
    def stream(self) -> int:
        return cvo_stream(self.ctx)

    def close(self) -> None:
        if self.ctx:
            cvo_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
