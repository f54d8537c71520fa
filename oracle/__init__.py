"""FP64 CPU oracle for Continuous Visual Odometry (CVO), arXiv 1904.02266.

TEST INFRASTRUCTURE ONLY. This package is the independent reference that the
CUDA path is checked against; it is plain, slow and exhaustive on purpose.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. The product library never imports, links or
executes anything here, and nothing here imports the product library.

Layout:
  cvo_oracle.c   FP64 pair sums (F, gradient, step sums) over every pair within
                 the cutoff, by an exhaustive loop or by a search of the
                 27 cells of edge r_c around each source point (same bits),
                 compiled with gcc into ``_build/liboracle.so``
  __init__.py    the solver around those sums: metric scaling (Eq. metric),
                 the 4th-order Taylor step (Eq. fourth), the SE(3)
                 exponential map (Eq. step), the pose update (Eq. newstep)
                 and the lengthscale schedule (Table 1 / decay reading).

Pose convention: P = (R, T) is a 4x4 matrix that maps source points into the
target frame, z~ = R z + T. It is the paper's h^{-1} (Sec. 3, "Calculating
the Gradient"). The solver perturbs P on the left, P <- exp(t xi) P, which is
the paper's h <- h exp(-t xi); the gradient signs below are the ones that make
(omega, v) an ascent direction under that update (checked by the finite
difference pins in the tests).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "cvo_oracle.c")

COLOR_NONE, COLOR_KERNEL, COLOR_DOT = 0, 1, 2
NOUT = 13  # F, dF/domega[3], dF/dv[3], nnz, S0..S4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C sums with gcc (FP64, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_double), ("sigma", ctypes.c_double),
                ("kcut", ctypes.c_double), ("color_mode", ctypes.c_int),
                ("ell_color", ctypes.c_double), ("color_scale", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.orc_pair_sums.argtypes = [dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64,
                                          ctypes.c_int, dp, ctypes.POINTER(_Params), dp, dp]
            lib.orc_pair_sums.restype = ctypes.c_int
            lib.orc_pair_sums_per_j.argtypes = [dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int64,
                                                ctypes.c_int, dp, ctypes.POINTER(_Params), dp,
                                                ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, dp]
            lib.orc_pair_sums_per_j.restype = ctypes.c_int
            lib.orc_pair_sums_grid.argtypes = lib.orc_pair_sums.argtypes
            lib.orc_pair_sums_grid.restype = ctypes.c_int
            lib.orc_pair_sums_grid_per_j.argtypes = lib.orc_pair_sums_per_j.argtypes
            lib.orc_pair_sums_grid_per_j.restype = ctypes.c_int
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


@dataclasses.dataclass
class Params:
    """Solver parameters. Defaults: the decaying-lengthscale reading of the
    schedule (0.15 -> x0.9 per iteration -> 0.02), sigma = 1, sparsification
    threshold 1e-3 (Sec. 5 / Table 1), appearance kernel with lengthscale 0.1,
    a = b = 1 in Eq. metric, at most 200 iterations, convergence thresholds
    1e-5 / 5e-5 (Table 1). ``search`` picks the exhaustive loop over all
    pairs or the cell search (same results; the cell search needs kcut in
    (0, 1))."""
    ell0: float = 0.15
    ell_decay: float = 0.9
    ell_min: float = 0.02
    schedule: str = "decay"          # "decay" or "table1"
    sigma: float = 1.0
    kcut: float = 1e-3
    color_mode: int = COLOR_KERNEL
    ell_color: float = 0.1
    color_scale: float = 1e-5
    a2: float = 1.0
    b2: float = 1.0
    max_iters: int = 200
    eps_pose: float = 1e-5
    eps_grad: float = 5e-5
    step_order: int = 4
    search: str = "exhaustive"       # "exhaustive" or "grid": same sums, bit for bit


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cparams(prm: Params, ell: float) -> _Params:
    return _Params(float(ell), float(prm.sigma), float(prm.kcut), int(prm.color_mode),
                   float(prm.ell_color), float(prm.color_scale))


def _prep(X, FX, Z, FZ):
    X, Z = _c(X).reshape(-1, 3), _c(Z).reshape(-1, 3)
    if FX is None or FZ is None:
        D = 0
        FX = np.zeros((X.shape[0], 0))
        FZ = np.zeros((Z.shape[0], 0))
    else:
        FX, FZ = _c(FX).reshape(X.shape[0], -1), _c(FZ).reshape(Z.shape[0], -1)
        if FX.shape[1] != FZ.shape[1]:
            raise ValueError("feature dimensions differ")
        D = FX.shape[1]
    # ctypes wants a valid pointer even for zero-size arrays
    if FX.size == 0:
        FX = np.zeros(1)
    if FZ.size == 0:
        FZ = np.zeros(1)
    return X, FX, Z, FZ, D


def _search_fn(lib, prm: Params, per_j: bool):
    if prm.search == "exhaustive":
        return lib.orc_pair_sums_per_j if per_j else lib.orc_pair_sums
    if prm.search == "grid":
        if not 0.0 < prm.kcut < 1.0:
            raise ValueError("the cell search needs kcut in (0, 1)")
        return lib.orc_pair_sums_grid_per_j if per_j else lib.orc_pair_sums_grid
    raise ValueError(f"unknown search {prm.search!r}")


def pair_sums(X, FX, Z, FZ, P, ell, prm: Params, xi=None) -> dict:
    """FP64 sums over every (i, j) pair that survives the cutoff (found by the
    exhaustive loop or the cell search, ``prm.search``: the same bits).

    Returns F (Eq. scalar), the unscaled derivatives dF/domega and dF/dv
    (Eq. 3_gradient, left-perturbation signs), the number of kept pairs, and,
    when a direction ``xi = (omega, v)`` is given, the step sums S0..S4 of
    Eq. fourth along it.
    """
    lib = _load()
    X, FX, Z, FZ, D = _prep(X, FX, Z, FZ)
    P = _c(P).reshape(4, 4)
    out = np.zeros(NOUT)
    cp = _cparams(prm, ell)
    xi_keep = _c(xi).reshape(6) if xi is not None else None
    xip = _dptr(xi_keep) if xi_keep is not None else None
    fn = _search_fn(lib, prm, per_j=False)
    rc = fn(_dptr(X), _dptr(FX), X.shape[0], _dptr(Z), _dptr(FZ), Z.shape[0], D,
            _dptr(P), ctypes.byref(cp), xip, _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle pair sums failed ({rc})")
    return {"F": out[0], "dF_domega": out[1:4].copy(), "dF_dv": out[4:7].copy(),
            "nnz": int(round(out[7])), "S": out[8:13].copy()}


def pair_sums_per_j(X, FX, Z, FZ, P, ell, prm: Params, js, xi=None) -> np.ndarray:
    """The same sums restricted to individual source points: row q holds the
    contribution of source point js[q] summed over all target points."""
    lib = _load()
    X, FX, Z, FZ, D = _prep(X, FX, Z, FZ)
    P = _c(P).reshape(4, 4)
    js = np.ascontiguousarray(js, dtype=np.int64)
    out = np.zeros((js.shape[0], NOUT))
    cp = _cparams(prm, ell)
    xi_keep = _c(xi).reshape(6) if xi is not None else None
    fn = _search_fn(lib, prm, per_j=True)
    rc = fn(_dptr(X), _dptr(FX), X.shape[0], _dptr(Z), _dptr(FZ), Z.shape[0],
            D, _dptr(P), ctypes.byref(cp),
            _dptr(xi_keep) if xi_keep is not None else None,
            js.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), js.shape[0],
            _dptr(out))
    if rc != 0:
        raise ValueError(f"oracle per-j sums failed ({rc})")
    return out


def gradient(sums: dict, prm: Params) -> np.ndarray:
    """Metric gradient (omega, v): the derivatives divided by a^2 and b^2
    (Eq. metric with n = 3 gives <(w,v),(n,u)> = a^2 w.n + b^2 v.u)."""
    return np.concatenate([sums["dF_domega"] / prm.a2, sums["dF_dv"] / prm.b2])


def hat(w) -> np.ndarray:
    """Skew matrix of a 3-vector: hat(w) @ x == cross(w, x)."""
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def exp_se3(tw) -> np.ndarray:
    """Closed-form SE(3) exponential of the twist tw = t*(omega, v), Eq. step:
    dR = I + (sin th/th) W + ((1 - cos th)/th^2) W^2,
    dT = (I + ((1 - cos th)/th^2) W + ((th - sin th)/th^3) W^2) t v,
    with W = hat(t omega) and th = |t omega|. (1 - cos th)/th^2 is evaluated
    as 2 sin^2(th/2)/th^2 and (th - sin th)/th^3 by its Taylor series below
    th = 0.01, both to avoid cancellation."""
    tw = np.asarray(tw, dtype=np.float64).reshape(6)
    phi, rho = tw[:3], tw[3:]
    th = float(np.linalg.norm(phi))
    W = hat(phi)
    W2 = W @ W
    t2 = th * th
    if th == 0.0:
        A, B = 1.0, 0.5
    else:
        A = np.sin(th) / th
        h = np.sin(0.5 * th) / (0.5 * th)
        B = 0.5 * h * h
    if th < 0.01:
        C = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0
    else:
        C = (th - np.sin(th)) / (th ** 3)
    out = np.eye(4)
    out[:3, :3] = np.eye(3) + A * W + B * W2
    out[:3, 3] = (np.eye(3) + B * W + C * W2) @ rho
    return out


def quartic_step(S, order: int = 4):
    """Step length t > 0 from the Taylor model G(t) ~ S0 + S1 t + ... + S4 t^4.

    4th order (Sec. 4 "Step size"): the first local maximum on t > 0, i.e. the
    smallest positive real root of G'(t) = S1 + 2 S2 t + 3 S3 t^2 + 4 S4 t^3
    at which G''(t) < 0. 2nd order: t = -S1 / (2 S2) when S2 < 0.
    Returns (t, ok); ok is False when the model has no such maximiser.
    """
    S0, S1, S2, S3, S4 = [float(s) for s in S]
    if order == 2:
        if S2 < 0.0:
            return -S1 / (2.0 * S2), True
        return 0.0, False
    coeffs = np.array([4.0 * S4, 3.0 * S3, 2.0 * S2, S1])
    nz = np.flatnonzero(coeffs != 0.0)
    if nz.size == 0 or nz[0] == 3:
        return 0.0, False
    roots = np.roots(coeffs[nz[0]:])
    cands = []
    for r in roots:
        if abs(r.imag) <= 1e-9 * max(1.0, abs(r.real)) and r.real > 0.0:
            t = float(r.real)
            if 2.0 * S2 + 6.0 * S3 * t + 12.0 * S4 * t * t < 0.0:
                cands.append(t)
    if not cands:
        return 0.0, False
    return min(cands), True


def ell_schedule(prm: Params, n: int) -> list:
    """Lengthscale of iterations 0..n-1.

    "decay": ell_{k+1} = max(ell_k * decay, ell_min), ell_0 = ell0, formed by
    repeated FP64 multiplication. "table1": Table 1's piecewise values
    (0.15; after iteration 3: 0.10; after 10: 0.06; after 20: 0.03), with
    iterations counted from 1 and the last value as the floor.
    """
    out = []
    if prm.schedule == "table1":
        for k in range(n):
            it = k + 1
            out.append(0.15 if it <= 3 else 0.10 if it <= 10 else 0.06 if it <= 20 else 0.03)
        return out
    ell = float(prm.ell0)
    for _ in range(n):
        out.append(ell)
        ell = max(ell * float(prm.ell_decay), float(prm.ell_min))
    return out


def ell_floor(prm: Params) -> float:
    return 0.03 if prm.schedule == "table1" else float(prm.ell_min)


def iterate(X, FX, Z, FZ, P0, prm: Params):
    """The iterations of the solve (Problem 1) one at a time: a generator that
    yields, after each iteration, a dict with the iteration's lengthscale,
    F, gradient xi, step sums S, step length t, kept pairs of both passes,
    the updated pose P and whether the stop test fired (``stop``). One
    iteration is: gradient at the current pose (Eq. 3_gradient scaled by
    Eq. metric), step sums along it (Eq. fourth), the step length from the
    quartic, and the update P <- exp(t xi) P (Eqs. newstep and step).

    It stops after the iteration at which the lengthscale sits at its floor
    and either |t xi| < eps_pose or |xi| < eps_grad (Table 1), or after
    max_iters. When the quartic has no maximiser on t > 0, the step is half
    the previous one (1e-3/|xi| on the first iteration; ``fallback`` is set).
    When |xi| < eps_grad (below the gradient threshold of Table 1's stop
    test) or S1 <= 0 (S1 is the metric norm of xi, so this happens only when
    xi is at rounding level) no step is taken (``no_ascent``): a xi at
    rounding level can still give S1 > 0, and the quartic's root along it is
    then arbitrary.
    """
    P = _c(P0).reshape(4, 4).copy()
    ells = ell_schedule(prm, prm.max_iters)
    floor = ell_floor(prm)
    t_prev = None
    for k in range(prm.max_iters):
        ell = ells[k]
        s = pair_sums(X, FX, Z, FZ, P, ell, prm)
        xi = gradient(s, prm)
        nxi = float(np.linalg.norm(xi))
        s2 = pair_sums(X, FX, Z, FZ, P, ell, prm, xi=xi)
        fallback = no_ascent = False
        if nxi == 0.0 or nxi < prm.eps_grad or not s2["S"][1] > 0.0:
            t = 0.0
            no_ascent = True
        else:
            t, ok = quartic_step(s2["S"], prm.step_order)
            if not ok:
                fallback = True
                t = 0.5 * t_prev if t_prev is not None else 1e-3 / nxi
        P = exp_se3(t * xi) @ P
        t_prev = t
        stop = ell == floor and (abs(t) * nxi < prm.eps_pose or nxi < prm.eps_grad)
        yield {"k": k, "ell": ell, "F": s["F"], "xi": xi, "t": t, "S": s2["S"],
               "nnz": s["nnz"], "pairs": s["nnz"] + s2["nnz"], "P": P.copy(),
               "fallback": fallback, "no_ascent": no_ascent, "stop": stop}
        if stop:
            return


def align(X, FX, Z, FZ, P0, prm: Params, record: bool = False) -> dict:
    """The whole solve (Problem 1): every iteration of ``iterate`` until its
    stop test fires or max_iters is reached. Returns the final pose, the
    iteration count, whether the stop test fired, the fallback and no-ascent
    step counts, the kept pairs of every pass, and (record) the history."""
    P = _c(P0).reshape(4, 4).copy()
    res = {"P": P, "iters": 0, "converged": False, "fallback_steps": 0, "no_ascent_steps": 0,
           "pair_evals": 0, "history": []}
    for r in iterate(X, FX, Z, FZ, P0, prm):
        res["P"] = r["P"]
        res["iters"] = r["k"] + 1
        res["converged"] = r["stop"]
        res["fallback_steps"] += int(r["fallback"])
        res["no_ascent_steps"] += int(r["no_ascent"])
        res["pair_evals"] += r["pairs"]
        if record:
            res["history"].append({"ell": r["ell"], "F": r["F"], "xi": r["xi"].copy(),
                                   "t": r["t"], "S": r["S"].copy(), "nnz": r["nnz"]})
    return res


def pose_error(P_est, P_ref):
    """Rotation angle of R_est R_ref^T (radians; the Frobenius norm of its
    log is sqrt(2) times this) and the translation |T_est - R_est R_ref^T T_ref|
    (Sec. 2, "Matrix Lie Group of Motion")."""
    P_est, P_ref = np.asarray(P_est), np.asarray(P_ref)
    dR = P_est[:3, :3] @ P_ref[:3, :3].T
    c = np.clip((np.trace(dR) - 1.0) / 2.0, -1.0, 1.0)
    s = np.linalg.norm([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]]) / 2.0
    ang = float(np.arctan2(s, c))
    dT = P_est[:3, 3] - dR @ P_ref[:3, 3]
    return ang, float(np.linalg.norm(dT))
