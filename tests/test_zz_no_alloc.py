"""cvo_eval_gradient_static, the gradient pass that allocates no device memory
(for callers that cannot allocate during a call), called through the C ABI.

Its F, gradient and kept-pair count must match cvo_eval's (the context-based
entry point) and the FP64 oracle's within the parity tolerances, on calls in a
row that share the library's static scratch. This file is collected last so
that a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

F_TOL = 1e-5
G_TOL = 1e-4


@pytest.fixture(scope="module")
def cvo():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1904_02266_gb300 as m
    return m


def _features(F5, D, seed):
    """D-column features from the workload's five: the first D, or the five
    followed by seeded uniform columns."""
    if D <= 5:
        return np.ascontiguousarray(F5[:, :D])
    extra = np.random.default_rng(seed).random((F5.shape[0], D - 5)).astype(np.float32)
    return np.ascontiguousarray(np.concatenate([F5, extra], axis=1))


def _oracle_check(oracle, got, X, FX, Z, FZ, P, ell, prm):
    ref = oracle.pair_sums(X, FX, Z, FZ, P, ell, prm)
    g_ref = oracle.gradient(ref, prm)
    assert abs(got[0] - ref["F"]) <= F_TOL * abs(ref["F"]), (got[0], ref["F"])
    assert np.linalg.norm(got[1:7] - g_ref) <= G_TOL * np.linalg.norm(g_ref), (got[1:7], g_ref)
    # pairs within FP32 rounding of the cutoff sphere may fall either way
    assert abs(got[7] - ref["nnz"]) <= max(2, 1e-6 * ref["nnz"]), (got[7], ref["nnz"])


def test_static_gradient_matches_eval_on_consecutive_calls(cvo, oracle_mod):
    torch = pytest.importorskip("torch")
    d = synth.planes_pair(3001, 2477, seed=synth.seed_for(1, 41))
    params = cvo.cvo_params_default()
    prm = oracle_mod.Params()
    X, FX = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["FX"]).cuda()
    Z, FZ = torch.from_numpy(d["Z"]).cuda(), torch.from_numpy(d["FZ"]).cuda()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(5)
    cases = [(d["P_gt"], 0.10), (synth.random_motion(rng, 2.0, 0.02) @ d["P_gt"], 0.05),
             (d["P_gt"], 0.10)]
    got_all = []
    with cvo.Context(device=0) as ctx:
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        for P, ell in cases:
            cvo.cvo_eval_gradient_static(X, FX, Z, FZ, params, P, ell, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().copy()
            got_all.append(got)
            ref = ctx.eval(ht, hs, P, ell)
            assert abs(got[0] - ref["F"]) <= F_TOL * abs(ref["F"]), (got[0], ref["F"])
            err = np.linalg.norm(got[1:7] - ref["grad6"])
            assert err <= G_TOL * np.linalg.norm(ref["grad6"]), (got[1:7], ref["grad6"])
            assert abs(got[7] - ref["nnz"]) <= max(2, 1e-6 * ref["nnz"]), (got[7], ref["nnz"])
            _oracle_check(oracle_mod, got, d["X"], d["FX"], d["Z"], d["FZ"], P, ell, prm)
    # the same inputs give the same bits, whatever the previous call left behind
    assert np.array_equal(got_all[0], got_all[2])


@pytest.mark.parametrize("mode", ["none", "kernel", "dot"])
@pytest.mark.parametrize("D", [3, 8])
def test_static_gradient_label_modes_and_widths(cvo, oracle_mod, mode, D):
    """Every label product and the 3- and 8-wide feature layouts, against the
    FP64 oracle and cvo_eval, two calls in a row."""
    torch = pytest.importorskip("torch")
    d = synth.planes_pair(2100, 1900, seed=synth.seed_for(1, 43))
    FX, FZ = _features(d["FX"], D, 1), _features(d["FZ"], D, 2)
    cm = {"none": cvo.CVO_COLOR_NONE, "kernel": cvo.CVO_COLOR_KERNEL, "dot": cvo.CVO_COLOR_DOT}[mode]
    om = {"none": oracle_mod.COLOR_NONE, "kernel": oracle_mod.COLOR_KERNEL,
          "dot": oracle_mod.COLOR_DOT}[mode]
    params = cvo.cvo_params_default()
    params.color_mode, params.feat_dim = cm, D
    prm = oracle_mod.Params(color_mode=om)
    tX, tZ = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["Z"]).cuda()
    tFX, tFZ = torch.from_numpy(FX).cuda(), torch.from_numpy(FZ).cuda()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with cvo.Context(device=0, color_mode=cm, feat_dim=D) as ctx:
        ht, hs = ctx.set_cloud(d["X"], FX), ctx.set_cloud(d["Z"], FZ)
        for P, ell in ((d["P_gt"], 0.08), (np.eye(4), 0.12)):
            cvo.cvo_eval_gradient_static(tX, tFX, tZ, tFZ, params, P, ell, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().copy()
            _oracle_check(oracle_mod, got, d["X"], FX if mode != "none" else None, d["Z"],
                          FZ if mode != "none" else None, P, ell, prm)
            ref = ctx.eval(ht, hs, P, ell)
            assert abs(got[0] - ref["F"]) <= F_TOL * abs(ref["F"])
            assert np.linalg.norm(got[1:7] - ref["grad6"]) <= G_TOL * np.linalg.norm(ref["grad6"])


def test_static_gradient_more_source_points_than_scratch_slots(cvo, oracle_mod):
    """m > 512 blocks x 256 threads: the block count is capped at the scratch's
    512 slots and each block strides over several tiles of source points."""
    torch = pytest.importorskip("torch")
    d = synth.planes_pair(400, 140000, seed=synth.seed_for(1, 44))
    assert d["Z"].shape[0] > 512 * 256
    params = cvo.cvo_params_default()
    prm = oracle_mod.Params()
    tX, tZ = torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["Z"]).cuda()
    tFX, tFZ = torch.from_numpy(d["FX"]).cuda(), torch.from_numpy(d["FZ"]).cuda()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with cvo.Context(device=0) as ctx:
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        for _ in range(2):
            cvo.cvo_eval_gradient_static(tX, tFX, tZ, tFZ, params, d["P_gt"], 0.1, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy().copy()
            _oracle_check(oracle_mod, got, d["X"], d["FX"], d["Z"], d["FZ"], d["P_gt"], 0.1, prm)
            ref = ctx.eval(ht, hs, d["P_gt"], 0.1)
            assert abs(got[0] - ref["F"]) <= F_TOL * abs(ref["F"])
            assert np.linalg.norm(got[1:7] - ref["grad6"]) <= G_TOL * np.linalg.norm(ref["grad6"])


def test_static_gradient_rejects_bad_sizes(cvo):
    torch = pytest.importorskip("torch")
    params = cvo.cvo_params_default()
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    feats = torch.zeros((0, 5), dtype=torch.float32, device="cuda")
    one = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    one_f = torch.zeros((1, 5), dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        cvo.cvo_eval_gradient_static(empty, feats, one, one_f, params, np.eye(4), 0.1, out)
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_eval_gradient_static(one, one_f, one, one_f, params, np.eye(4), -1.0, out)
    assert e.value.code == cvo.CVO_ERR_INVALID_ARG
    bad = cvo.cvo_params_default()
    bad.color_mode = 3
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_eval_gradient_static(one, one_f, one, one_f, bad, np.eye(4), 0.1, out)
    assert e.value.code == cvo.CVO_ERR_INVALID_ARG
    bad = cvo.cvo_params_default()
    bad.color_mode, bad.color_scale = cvo.CVO_COLOR_DOT, -1.0
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_eval_gradient_static(one, one_f, one, one_f, bad, np.eye(4), 0.1, out)
    assert e.value.code == cvo.CVO_ERR_INVALID_ARG
