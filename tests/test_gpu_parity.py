"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances (from the benchmark spec's targets, checked against the FP64 oracle):
  F           |dF| / F <= 1e-5
  gradient    |d grad6| / |grad6| <= 1e-4 at a fixed pose
  final pose  <= 1e-4 rad and 1e-4 m
The step sums are compared along the GPU's own direction, so that only the
FP32 pair arithmetic separates the two sides.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4
POSE_TOL = 1e-4
S_TOL = 2e-4


@pytest.fixture(scope="module")
def cvo():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1904_02266_gb300 as m
    return m


def _ctx(cvo, **kw):
    return cvo.Context(device=0, **kw)


def _oracle_params(ctx_params, cvo):
    p = oracle.Params()
    for k in ("ell0", "ell_decay", "ell_min", "sigma", "kcut", "ell_color", "color_scale", "a2",
              "b2", "max_iters", "eps_pose", "eps_grad", "step_order"):
        setattr(p, k, getattr(ctx_params, k))
    p.color_mode = ctx_params.color_mode if ctx_params.feat_dim > 0 else oracle.COLOR_NONE
    p.schedule = "table1" if ctx_params.schedule == cvo.CVO_SCHEDULE_TABLE1 else "decay"
    return p


def _check_eval(g, X, FX, Z, FZ, P, ell, prm, label=""):
    r = oracle.pair_sums(X, FX, Z, FZ, P, ell, prm)
    ref = oracle.gradient(r, prm)
    if r["F"] == 0.0:
        assert g["F"] == 0.0 and np.all(g["grad6"] == 0.0), label
        return r
    assert abs(g["F"] - r["F"]) <= F_TOL * abs(r["F"]), (label, g["F"], r["F"])
    err = np.linalg.norm(g["grad6"] - ref)
    assert err <= G_TOL * np.linalg.norm(ref), (label, err / np.linalg.norm(ref), g["grad6"], ref)
    # kept-pair count: identical up to pairs sitting on the cutoff sphere
    assert abs(g["nnz"] - r["nnz"]) <= max(2, 1e-6 * r["nnz"]), (label, g["nnz"], r["nnz"])
    assert g["candidates"] >= g["nnz"]
    # step sums along the GPU's direction
    s2 = oracle.pair_sums(X, FX, Z, FZ, P, ell, prm, xi=g["grad6"])
    S_ref = s2["S"]
    scale = np.abs(S_ref).max()
    assert abs(g["S"][0] - S_ref[0]) <= F_TOL * abs(S_ref[0]), (label, g["S"], S_ref)
    for m in range(1, 5):
        assert abs(g["S"][m] - S_ref[m]) <= S_TOL * max(abs(S_ref[m]), 1e-6 * scale), \
            (label, m, g["S"], S_ref)
    return r


def _feats(d, mode):
    if mode == "none":
        return None, None
    return d["FX"], d["FZ"]


@pytest.mark.parametrize("mode", ["kernel", "none", "dot"])
@pytest.mark.parametrize("ell", [0.15, 0.06, 0.02])
def test_eval_planes(cvo, mode, ell):
    d = synth.planes_pair()
    kw = {"color_mode": {"kernel": 1, "none": 0, "dot": 2}[mode]}
    if mode == "dot":
        kw["color_scale"] = 1.0
    if mode == "none":
        kw["feat_dim"] = 0
    with _ctx(cvo, **kw) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        FX, FZ = _feats(d, mode)
        ht, hs = ctx.set_cloud(d["X"], FX), ctx.set_cloud(d["Z"], FZ)
        rng = np.random.default_rng(17)
        for P in [np.eye(4), d["P_gt"], synth.random_motion(rng, 3.0, 0.04) @ d["P_gt"]]:
            g = ctx.eval(ht, hs, P, ell)
            _check_eval(g, d["X"], FX, d["Z"], FZ, P, ell, prm, f"{mode} {ell}")


@pytest.mark.parametrize("cell_factor,cluster_factor", [(8.0, 8.0), (0.5, 1.0)])
def test_eval_extreme_cell_and_cluster_factors(cvo, cell_factor, cluster_factor):
    """The pair test runs in each cluster's own frame, so its cancellation grows
    with the cluster's extent in cutoff radii; at the largest cell and cluster
    factors the API accepts (clusters tens of r_c wide) and at the smallest,
    F, the gradient, the kept pairs and the step sums still meet the parity bars."""
    d = synth.planes_pair(3000, 3000, seed=synth.seed_for(1, 21))
    with _ctx(cvo, cell_factor=cell_factor, cluster_factor=cluster_factor) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        rng = np.random.default_rng(23)
        for ell in (0.15, 0.05, 0.02):
            for P in (d["P_gt"], synth.random_motion(rng, 2.0, 0.02) @ d["P_gt"]):
                g = ctx.eval(ht, hs, P, ell)
                _check_eval(g, d["X"], d["FX"], d["Z"], d["FZ"], P, ell, prm,
                            f"cells {cell_factor} clusters {cluster_factor} ell {ell}")


def _bf16_stored(F, scale):
    """The features the library keeps in BF16 mode: the FP32 product f * scale
    rounded to BF16 (nearest, ties to even), expressed back in feature units."""
    x = (np.asarray(F, dtype=np.float32) * np.float32(scale)).astype(np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64) / float(np.float32(scale))


@pytest.mark.parametrize("mode", ["kernel", "dot"])
def test_eval_bf16_features(cvo, mode):
    # BF16 storage: the oracle is given the features as stored, so only the
    # FP32 pair arithmetic separates the two sides
    d = synth.planes_pair(1500, 1300, seed=synth.seed_for(1, 21))
    kw = {"feat_bf16": 1, "color_mode": 1 if mode == "kernel" else 2}
    if mode == "dot":
        kw["color_scale"] = 1.0
    with _ctx(cvo, **kw) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        scale = (np.sqrt(1.4426950408889634 / (2.0 * ctx.params.ell_color ** 2)) if mode == "kernel"
                 else np.sqrt(ctx.params.color_scale))
        FXs, FZs = _bf16_stored(d["FX"], scale), _bf16_stored(d["FZ"], scale)
        assert not np.array_equal(FXs, d["FX"].astype(np.float64))   # rounding did happen
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        for P, ell in [(np.eye(4), 0.1), (d["P_gt"], 0.05)]:
            g = ctx.eval(ht, hs, P, ell)
            _check_eval(g, d["X"], FXs, d["Z"], FZs, P, ell, prm, f"bf16 {mode} {ell}")


def test_align_bf16_features(cvo):
    d = synth.planes_pair(1500, 1500, seed=synth.seed_for(1, 22))
    with _ctx(cvo, feat_bf16=1) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        scale = np.sqrt(1.4426950408889634 / (2.0 * ctx.params.ell_color ** 2))
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        P_gpu, st = ctx.align(ht, hs)
    FXs, FZs = _bf16_stored(d["FX"], scale), _bf16_stored(d["FZ"], scale)
    res = oracle.align(d["X"], FXs, d["Z"], FZs, np.eye(4), prm)
    ang, tr = oracle.pose_error(P_gpu, res["P"])
    assert ang <= POSE_TOL and tr <= POSE_TOL, (ang, tr)
    assert abs(st["iters"] - res["iters"]) <= 3


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 7, 8])
def test_feature_dims(cvo, D):
    rng = np.random.default_rng(100 + D)
    d = synth.planes_pair(900, 700, seed=77)
    FX = rng.random((900, D)).astype(np.float32)
    FZ = np.clip(FX[rng.integers(0, 900, 700)] + 0.05 * rng.normal(size=(700, D)), 0, 1)
    FZ = FZ.astype(np.float32)
    with _ctx(cvo, feat_dim=D) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(d["X"], FX), ctx.set_cloud(d["Z"], FZ)
        g = ctx.eval(ht, hs, d["P_gt"], 0.1)
        _check_eval(g, d["X"], FX, d["Z"], FZ, d["P_gt"], 0.1, prm, f"D={D}")


@pytest.mark.parametrize("n,m", [(1, 1), (37, 1013), (1013, 37), (33, 64), (4097, 2049)])
def test_ragged_sizes(cvo, n, m):
    rng = np.random.default_rng(n * 7 + m)
    X = (rng.normal(scale=0.15, size=(n, 3)) + [0.3, -1.0, 2.0]).astype(np.float32)
    Z = (X[rng.integers(0, n, m)] + rng.normal(scale=0.03, size=(m, 3))).astype(np.float32)
    FX = rng.random((n, 5)).astype(np.float32)
    FZ = rng.random((m, 5)).astype(np.float32)
    with _ctx(cvo) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(X, FX), ctx.set_cloud(Z, FZ)
        for ell in (0.15, 0.03):
            P = synth.random_motion(rng, 2.0, 0.01)
            g = ctx.eval(ht, hs, P, ell)
            _check_eval(g, X, FX, Z, FZ, P, ell, prm, f"{n}x{m} {ell}")


def test_clouds_out_of_reach(cvo):
    d = synth.planes_pair(500, 500, seed=3)
    with _ctx(cvo) as ctx:
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        P = np.eye(4)
        P[:3, 3] = [100.0, -50.0, 20.0]
        g = ctx.eval(ht, hs, P, 0.15)
        assert g["F"] == 0.0 and g["nnz"] == 0 and np.all(g["grad6"] == 0.0)
        assert np.all(g["S"] == 0.0)


def test_single_cell_cloud(cvo):
    """Every target point in one cell (extent 1 cm, ell 0.15)."""
    rng = np.random.default_rng(9)
    X = (rng.random((300, 3)) * 0.01).astype(np.float32)
    Z = (rng.random((200, 3)) * 0.01 + 0.002).astype(np.float32)
    FX, FZ = rng.random((300, 5)).astype(np.float32), rng.random((200, 5)).astype(np.float32)
    with _ctx(cvo) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(X, FX), ctx.set_cloud(Z, FZ)
        g = ctx.eval(ht, hs, np.eye(4), 0.15)
        r = _check_eval(g, X, FX, Z, FZ, np.eye(4), 0.15, prm, "one cell")
        assert r["nnz"] == 300 * 200


def test_common_motion_invariance(cvo):
    """Moving the target and the pose by the same rigid motion (Sec. 4
    corollaries) leaves F unchanged on the GPU too, with a rebuilt grid."""
    d = synth.planes_pair(1500, 1500, seed=11)
    g_motion = synth.random_motion(np.random.default_rng(4), 40.0, 1.5)
    with _ctx(cvo) as ctx:
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        hm = ctx.set_cloud(synth.transform(g_motion, d["X"].astype(np.float64)).astype(np.float32),
                           d["FX"])
        a = ctx.eval(ht, hs, d["P_gt"], 0.08)
        b = ctx.eval(hm, hs, g_motion @ d["P_gt"], 0.08)
        assert abs(a["F"] - b["F"]) <= F_TOL * a["F"]


def test_deterministic(cvo):
    d = synth.planes_pair()
    with _ctx(cvo, max_iters=25) as ctx:
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        a = ctx.eval(ht, hs, d["P_gt"], 0.1)
        b = ctx.eval(ht, hs, d["P_gt"], 0.1)
        assert a["F"] == b["F"] and np.array_equal(a["grad6"], b["grad6"])
        assert np.array_equal(a["S"], b["S"])
        P1, s1 = ctx.align(ht, hs)
        P2, s2 = ctx.align(ht, hs)
        assert np.array_equal(P1, P2) and s1["iters"] == s2["iters"]
        P3, s3, rec = ctx.align_profile(ht, hs)
        assert np.array_equal(P1, P3) and s3["iters"] == s1["iters"] == len(rec)
        assert sum(r["grad_pairs"] + r["step_pairs"] for r in rec) == s1["pair_evals"]


def test_device_pointer_input(cvo):
    torch = pytest.importorskip("torch")
    d = synth.planes_pair(1200, 1100, seed=21)
    with _ctx(cvo) as ctx:
        h1 = ctx.set_cloud(d["X"], d["FX"])
        h2 = ctx.set_cloud(d["Z"], d["FZ"])
        h3 = ctx.set_cloud(torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["FX"]).cuda())
        h4 = ctx.set_cloud(torch.from_numpy(d["Z"]).cuda(), torch.from_numpy(d["FZ"]).cuda())
        a = ctx.eval(h1, h2, d["P_gt"], 0.1)
        b = ctx.eval(h3, h4, d["P_gt"], 0.1)
        assert a["F"] == b["F"] and np.array_equal(a["grad6"], b["grad6"])


def test_invalid_arguments(cvo):
    d = synth.planes_pair(500, 500, seed=5)
    with _ctx(cvo) as ctx:
        with pytest.raises(cvo.CvoError) as e:
            ctx.set_cloud(np.zeros((0, 3), np.float32), np.zeros((0, 5), np.float32))
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        bad = d["X"].copy()
        bad[17, 1] = np.nan
        with pytest.raises(cvo.CvoError) as e:
            ctx.set_cloud(bad, d["FX"])
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        badf = d["FX"].copy()
        badf[3, 4] = np.inf
        with pytest.raises(cvo.CvoError) as e:
            ctx.set_cloud(d["X"], badf)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        h = ctx.set_cloud(d["X"], d["FX"])
        with pytest.raises(cvo.CvoError) as e:
            ctx.eval(h, 99, np.eye(4), 0.1)
        assert e.value.code == cvo.CVO_ERR_NOT_FOUND
        with pytest.raises(cvo.CvoError) as e:
            ctx.eval(h, h, np.eye(4), -1.0)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        P = np.eye(4)
        P[0, 3] = np.nan
        with pytest.raises(cvo.CvoError) as e:
            ctx.align(h, h, P)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        ctx.release(h)
        with pytest.raises(cvo.CvoError) as e:
            ctx.release(h)
        assert e.value.code == cvo.CVO_ERR_NOT_FOUND
    with cvo.Context(device=0, hbm_budget=4 * 1024) as small:
        with pytest.raises(cvo.CvoError) as e:
            small.set_cloud(d["X"], d["FX"])
        assert e.value.code == cvo.CVO_ERR_OUT_OF_BUDGET


def _align_parity(cvo, d, ctx_kw, P0=None, check_gt=None):
    with _ctx(cvo, **ctx_kw) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        P0 = np.eye(4) if P0 is None else P0
        P_gpu, st = ctx.align(ht, hs, P0)
    res = oracle.align(d["X"], d["FX"], d["Z"], d["FZ"], P0, prm)
    ang, tr = oracle.pose_error(P_gpu, res["P"])
    assert ang <= POSE_TOL and tr <= POSE_TOL, (ang, tr, st["iters"], res["iters"])
    assert abs(st["iters"] - res["iters"]) <= 3, (st["iters"], res["iters"])
    if check_gt is not None:
        ang_gt, tr_gt = oracle.pose_error(P_gpu, d["P_gt"])
        assert ang_gt < check_gt and tr_gt < check_gt
    return st, res


def test_align_planes(cvo):
    st, res = _align_parity(cvo, synth.planes_pair(), {}, check_gt=5e-3)
    assert st["converged"] == 1
    assert st["iters"] == res["iters"]


@pytest.mark.parametrize("pair", [1, 2, 3])
def test_align_planes_seeds(cvo, pair):
    d = synth.planes_pair(2000 + 311 * pair, 1800 + 97 * pair, seed=synth.seed_for(1, pair))
    _align_parity(cvo, d, {})


def test_align_table1_schedule_and_second_order(cvo):
    d = synth.planes_pair(1500, 1500, seed=synth.seed_for(1, 9))
    _align_parity(cvo, d, {"schedule": cvo.CVO_SCHEDULE_TABLE1, "max_iters": 60})
    _align_parity(cvo, d, {"step_order": 2, "max_iters": 60})


def test_align_with_kept_pair_rebalance(cvo):
    # the rebalanced work split only reorders the FP64 sums over blocks
    d = synth.planes_pair(2500, 2300, seed=synth.seed_for(1, 11))
    _align_parity(cvo, d, {"cost_kept": 2.0})


def test_align_paper_color_dot(cvo):
    d = synth.planes_pair(1500, 1500, seed=synth.seed_for(1, 10))
    _align_parity(cvo, d, {"color_mode": cvo.CVO_COLOR_DOT, "color_scale": 1e-5, "max_iters": 60})


def test_align_identical_clouds_stays_put(cvo):
    d = synth.planes_pair(1000, 1000, seed=12)
    with _ctx(cvo, max_iters=40) as ctx:
        h = ctx.set_cloud(d["X"], d["FX"])
        P, st = ctx.align(h, h)
    ang, tr = oracle.pose_error(P, np.eye(4))
    assert ang < 1e-6 and tr < 1e-6


def test_step_length_with_roots_orders_of_magnitude_apart(cvo):
    """A keyframe / frame pair of the serving workload (57k and 40k planes
    points, seeds as the serving trace draws them) whose first step model has
    roots five orders of magnitude apart (-3.3e-3, -5.5e-8, 2.8e-8): the first
    maximiser must be found without fallback steps, and the solve must not
    depend on the traversal parameters beyond the pose tolerance."""
    X, FX = synth.stream_keyframe(623434856, 56816)
    Z, FZ, P_gt = synth.stream_frame(623434856, 0, 39819)
    poses = []
    for kw in ({}, {"cell_factor": 1.0}, {"cluster_factor": 1.0}):
        with _ctx(cvo, **kw) as ctx:
            P, st = ctx.align(ctx.set_cloud(X, FX), ctx.set_cloud(Z, FZ))
        assert st["status"] == 0 and st["fallback_steps"] == 0, (kw, st)
        poses.append(P)
    for P in poses[1:]:
        ang, tr = oracle.pose_error(P, poses[0])
        assert ang < POSE_TOL and tr < POSE_TOL, (ang, tr)
    ang, tr = oracle.pose_error(poses[0], P_gt)
    assert ang < 5e-3 and tr < 5e-3, (ang, tr)


@pytest.mark.slow
def test_eval_room_full_size(cvo):
    """The benchmark workload (VGA-scale room, 20k points per frame) at fixed
    poses, in the same launch configuration the benchmark times."""
    d = synth.room_pair()
    with _ctx(cvo) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        for P, ell in [(np.eye(4), 0.15), (d["P_gt"], 0.02), (np.eye(4), 0.05)]:
            g = ctx.eval(ht, hs, P, ell)
            _check_eval(g, d["X"], d["FX"], d["Z"], d["FZ"], P, ell, prm, f"room {ell}")


@pytest.mark.slow
def test_eval_dense_room_100k(cvo):
    """The dense precision-sweep size: N = M = 100,000 points (room frames,
    95% of the valid pixels kept, subsampled), F, gradient and step sums at a
    fixed pose against the exhaustive FP64 oracle (10^10 pair tests a pass)."""
    d = synth.room_pair(n_points=100000, seed=synth.seed_for(4), mode="valid")
    with _ctx(cvo) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        g = ctx.eval(ht, hs, np.eye(4), 0.05)
        _check_eval(g, d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), 0.05, prm, "room 100k")


def test_fp32_reduction_mode_is_looser_but_close(cvo):
    # precision study: FP32 block and cross-block sums against the FP64 oracle
    d = synth.room_pair()
    with _ctx(cvo, reduce_fp32=1) as ctx:
        prm = _oracle_params(ctx.params, cvo)
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        g = ctx.eval(ht, hs, np.eye(4), 0.05)
    r = oracle.pair_sums(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), 0.05, prm)
    ref = oracle.gradient(r, prm)
    assert abs(g["F"] - r["F"]) <= 1e-4 * abs(r["F"])
    assert np.linalg.norm(g["grad6"] - ref) <= 1e-3 * np.linalg.norm(ref)
    assert g["nnz"] == pytest.approx(r["nnz"], abs=max(2, 1e-6 * r["nnz"]))


@pytest.mark.slow
def test_align_room_full_size(cvo):
    d = synth.room_pair()
    _align_parity(cvo, d, {})
