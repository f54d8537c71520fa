"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics:
closed forms, finite differences, invariances, library routines and brute
force. None of these re-types the oracle's own formulas."""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _params(oracle, **kw):
    p = oracle.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _random_pose(rng, deg=20.0, meters=0.2):
    return synth.random_motion(rng, deg, meters)


def _small_clouds(rng, n=40, m=30, d=5, spread=0.2):
    X = rng.normal(scale=spread, size=(n, 3))
    Z = X[rng.integers(0, n, size=m)] + rng.normal(scale=0.05, size=(m, 3))
    FX = rng.random((n, d))
    FZ = rng.random((m, d))
    return X, FX, Z, FZ


# --------------------------------------------------------------------------
# F: closed forms (Eq. scalar with the squared-exponential kernel, Sec. 3)
# --------------------------------------------------------------------------

def test_coincident_points_give_count_times_sigma2(oracle_mod):
    """n copies of one point against m copies of the same point: every kernel
    value is sigma^2 and every label product is 1, so F = n m sigma^2."""
    p = _params(oracle_mod, sigma=0.7, color_mode=oracle_mod.COLOR_KERNEL)
    X = np.tile([[0.3, -0.2, 1.1]], (7, 1))
    Z = np.tile([[0.3, -0.2, 1.1]], (5, 1))
    F = np.full((7, 5 - 0), 0.25)[:, :3]
    s = oracle_mod.pair_sums(X, np.tile([[0.1, 0.2, 0.3]], (7, 1)), Z, np.tile([[0.1, 0.2, 0.3]], (5, 1)),
                             np.eye(4), 0.1, p)
    assert s["F"] == pytest.approx(7 * 5 * 0.49, rel=1e-14)
    assert s["nnz"] == 35
    assert F.shape == (7, 3)


def test_gaussian_lattice_poisson_sum(oracle_mod):
    """A straight line of target points with spacing h = ell/2 and one source
    point at offset s: by Poisson summation,
    sum_i exp(-(i h - s)^2 / 2 ell^2) = sqrt(2 pi) ell / h up to terms of
    order exp(-2 pi^2 ell^2 / h^2) ~ 1e-34."""
    ell = 0.1
    h = ell / 2
    i = np.arange(-400, 401)
    X = np.stack([i * h, np.zeros_like(i, dtype=float), np.zeros_like(i, dtype=float)], axis=1)
    for s_off in [0.0, 0.013, 0.037]:
        Z = np.array([[s_off, 0.0, 0.0]])
        p = _params(oracle_mod, kcut=0.0, color_mode=oracle_mod.COLOR_NONE)
        s = oracle_mod.pair_sums(X, None, Z, None, np.eye(4), ell, p)
        assert s["F"] == pytest.approx(math.sqrt(2 * math.pi) * ell / h, rel=1e-13)
        # the translational gradient along the line vanishes by the same
        # argument (derivative of a constant); across the line it is zero by symmetry
        assert abs(s["dF_dv"][0]) < 1e-10
        assert abs(s["dF_dv"][1]) < 1e-12 and abs(s["dF_dv"][2]) < 1e-12


def test_sparsification_radius(oracle_mod):
    """Sparsification (Sec. 5): a pair is dropped when its spatial kernel value
    is below kcut, i.e. beyond r_c = ell sqrt(2 ln(1/kcut))."""
    ell, kcut = 0.05, 1e-3
    rc = ell * math.sqrt(2 * math.log(1 / kcut))
    X = np.array([[0.0, 0.0, 0.0]])
    p = _params(oracle_mod, kcut=kcut, color_mode=oracle_mod.COLOR_NONE)
    inside = oracle_mod.pair_sums(X, None, np.array([[rc * (1 - 1e-9), 0, 0]]), None, np.eye(4), ell, p)
    outside = oracle_mod.pair_sums(X, None, np.array([[0, rc * (1 + 1e-9), 0]]), None, np.eye(4), ell, p)
    assert inside["nnz"] == 1 and inside["F"] == pytest.approx(kcut, rel=1e-7)
    assert outside["nnz"] == 0 and outside["F"] == 0.0


def test_label_products_closed_form(oracle_mod):
    """Appearance kernel exp(-|f-g|^2 / 2 ell_c^2) and the paper's scaled dot
    product s <f, g> (Sec. 5 remark), on coincident positions."""
    X = np.array([[0.0, 0.0, 0.0]])
    f = np.array([[0.2, 0.5, 0.9]])
    g = np.array([[0.3, 0.1, 0.6]])
    pk = _params(oracle_mod, color_mode=oracle_mod.COLOR_KERNEL, ell_color=0.2)
    sk = oracle_mod.pair_sums(X, f, X, g, np.eye(4), 0.1, pk)
    assert sk["F"] == pytest.approx(math.exp(-(0.01 + 0.16 + 0.09) / (2 * 0.04)), rel=1e-14)
    pd = _params(oracle_mod, color_mode=oracle_mod.COLOR_DOT, color_scale=1e-5)
    sd = oracle_mod.pair_sums(X, f, X, g, np.eye(4), 0.1, pd)
    assert sd["F"] == pytest.approx(1e-5 * (0.06 + 0.05 + 0.54), rel=1e-14)


def test_per_source_sums_add_up(oracle_mod):
    rng = np.random.default_rng(3)
    X, FX, Z, FZ = _small_clouds(rng)
    p = _params(oracle_mod)
    P = _random_pose(rng, 3, 0.02)
    xi = rng.normal(size=6)
    whole = oracle_mod.pair_sums(X, FX, Z, FZ, P, 0.1, p, xi=xi)
    per = oracle_mod.pair_sums_per_j(X, FX, Z, FZ, P, 0.1, p, np.arange(Z.shape[0]), xi=xi)
    tot = per.sum(axis=0)
    assert tot[0] == pytest.approx(whole["F"], rel=1e-13)
    np.testing.assert_allclose(tot[8:13], whole["S"], rtol=1e-12, atol=1e-12 * abs(whole["S"]).max())


# --------------------------------------------------------------------------
# invariances (Sec. 4 corollaries: SE(n) acts isometrically)
# --------------------------------------------------------------------------

def test_common_rigid_motion_invariance(oracle_mod):
    """Moving the target cloud and the pose by the same rigid motion g leaves
    every kernel value, hence F and the kept-pair count, unchanged."""
    rng = np.random.default_rng(5)
    X, FX, Z, FZ = _small_clouds(rng)
    p = _params(oracle_mod)
    P = _random_pose(rng, 4, 0.03)
    g = _random_pose(rng, 70, 2.0)
    a = oracle_mod.pair_sums(X, FX, Z, FZ, P, 0.08, p)
    b = oracle_mod.pair_sums(synth.transform(g, X), FX, Z, FZ, g @ P, 0.08, p)
    assert b["F"] == pytest.approx(a["F"], rel=1e-12)
    assert b["nnz"] == a["nnz"]


def test_role_swap_symmetry(oracle_mod):
    """The kernel is symmetric and the action isometric, so
    F(X, Z, P) = F(Z, X, P^{-1})."""
    rng = np.random.default_rng(6)
    X, FX, Z, FZ = _small_clouds(rng, n=35, m=45)
    p = _params(oracle_mod)
    P = _random_pose(rng, 10, 0.1)
    a = oracle_mod.pair_sums(X, FX, Z, FZ, P, 0.1, p)
    b = oracle_mod.pair_sums(Z, FZ, X, FX, synth.inverse(P), 0.1, p)
    assert b["F"] == pytest.approx(a["F"], rel=1e-12)
    assert b["nnz"] == a["nnz"]


def test_identity_is_global_max_for_identical_clouds(oracle_mod):
    """Sec. 4 theorem: for Z = X (same labels) the identity maximises F, so the
    gradient vanishes there and F(P) <= F(I) for any P."""
    rng = np.random.default_rng(7)
    X = rng.normal(scale=0.3, size=(60, 3))
    FX = rng.random((60, 5))
    p = _params(oracle_mod, kcut=0.0)
    s0 = oracle_mod.pair_sums(X, FX, X, FX, np.eye(4), 0.1, p)
    scale = s0["F"] / 0.1
    assert np.abs(s0["dF_domega"]).max() < 1e-12 * scale
    assert np.abs(s0["dF_dv"]).max() < 1e-12 * scale
    for _ in range(10):
        P = _random_pose(rng, rng.uniform(0.1, 30), rng.uniform(0.001, 0.3))
        assert oracle_mod.pair_sums(X, FX, X, FX, P, 0.1, p)["F"] <= s0["F"]


# --------------------------------------------------------------------------
# gradient = derivative of F (Sec. 3 theorem and Eq. 3_gradient)
# --------------------------------------------------------------------------

def _F_at(oracle, X, FX, Z, FZ, P, ell, p, tw):
    return oracle.pair_sums(X, FX, Z, FZ, scipy.linalg.expm(_twist_matrix(tw)) @ P, ell, p)["F"]


def _twist_matrix(tw):
    w, v = tw[:3], tw[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


@pytest.mark.parametrize("mode", ["none", "kernel", "dot"])
def test_gradient_matches_finite_differences(oracle_mod, mode):
    """Central differences of F along each generator of se(3), with the pose
    moved by the matrix exponential (scipy) on the left."""
    rng = np.random.default_rng(11)
    X, FX, Z, FZ = _small_clouds(rng)
    cm = {"none": oracle_mod.COLOR_NONE, "kernel": oracle_mod.COLOR_KERNEL,
          "dot": oracle_mod.COLOR_DOT}[mode]
    p = _params(oracle_mod, kcut=0.0, color_mode=cm, color_scale=1.0)
    P = _random_pose(rng, 8, 0.05)
    ell = 0.12
    s = oracle_mod.pair_sums(X, FX, Z, FZ, P, ell, p)
    g = np.concatenate([s["dF_domega"], s["dF_dv"]])
    h = 1e-5
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd[k] = (_F_at(oracle_mod, X, FX, Z, FZ, P, ell, p, e)
                 - _F_at(oracle_mod, X, FX, Z, FZ, P, ell, p, -e)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


def test_metric_gradient_is_riesz_representer(oracle_mod):
    """Eq. metric with n = 3: <(w, v), (n, u)> = a^2 w.n + b^2 v.u. The metric
    gradient xi must satisfy <xi, eta> = dF(eta) for every direction eta."""
    rng = np.random.default_rng(12)
    X, FX, Z, FZ = _small_clouds(rng)
    p = _params(oracle_mod, kcut=0.0, a2=3.0, b2=0.5)
    P = _random_pose(rng, 5, 0.05)
    s = oracle_mod.pair_sums(X, FX, Z, FZ, P, 0.1, p)
    xi = oracle_mod.gradient(s, p)
    for _ in range(4):
        eta = rng.normal(size=6)
        h = 1e-6
        dF = (_F_at(oracle_mod, X, FX, Z, FZ, P, 0.1, p, h * eta)
              - _F_at(oracle_mod, X, FX, Z, FZ, P, 0.1, p, -h * eta)) / (2 * h)
        lhs = p.a2 * xi[:3] @ eta[:3] + p.b2 * xi[3:] @ eta[3:]
        assert lhs == pytest.approx(dF, rel=1e-6, abs=1e-9 * abs(s["F"]))


# --------------------------------------------------------------------------
# step sums (Eq. fourth)
# --------------------------------------------------------------------------

def test_step_sums_first_terms(oracle_mod):
    """S0 = F, and along xi = grad the first-order term is the metric norm:
    S1 = dF(xi) = a^2 |omega|^2 + b^2 |v|^2."""
    rng = np.random.default_rng(13)
    X, FX, Z, FZ = _small_clouds(rng)
    p = _params(oracle_mod, a2=2.0, b2=0.7)
    P = _random_pose(rng, 5, 0.05)
    s = oracle_mod.pair_sums(X, FX, Z, FZ, P, 0.1, p)
    xi = oracle_mod.gradient(s, p)
    s2 = oracle_mod.pair_sums(X, FX, Z, FZ, P, 0.1, p, xi=xi)
    assert s2["S"][0] == pytest.approx(s["F"], rel=1e-13)
    assert s2["S"][1] == pytest.approx(p.a2 * xi[:3] @ xi[:3] + p.b2 * xi[3:] @ xi[3:], rel=1e-11)


def test_quartic_residual_is_fifth_order(oracle_mod):
    """G(t) = F(exp(t xi) P) minus the quartic model S0 + ... + S4 t^4 is
    O(t^5): halving t divides the residual by about 32. A wrong S2, S3 or S4
    leaves an O(t^2), O(t^3) or O(t^4) residual (ratio 4, 8 or 16)."""
    rng = np.random.default_rng(14)
    X, FX, Z, FZ = _small_clouds(rng, n=60, m=50)
    p = _params(oracle_mod, kcut=0.0)
    P = _random_pose(rng, 6, 0.04)
    ell = 0.15
    s = oracle_mod.pair_sums(X, FX, Z, FZ, P, ell, p)
    xi = oracle_mod.gradient(s, p)
    xi = xi / np.linalg.norm(xi)                 # any direction works
    S = oracle_mod.pair_sums(X, FX, Z, FZ, P, ell, p, xi=xi)["S"]

    def resid(t):
        G = _F_at(oracle_mod, X, FX, Z, FZ, P, ell, p, t * xi)
        return G - (S[0] + S[1] * t + S[2] * t ** 2 + S[3] * t ** 3 + S[4] * t ** 4)

    ts = [0.02, 0.01, 0.005]
    r = [resid(t) for t in ts]
    for a, b in zip(r, r[1:]):
        assert 24.0 < a / b < 40.0, r


# --------------------------------------------------------------------------
# exponential map (Eq. step) and the step length
# --------------------------------------------------------------------------

@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 0.3, 2.5, 3.1])
def test_exp_map_matches_matrix_exponential(oracle_mod, scale):
    rng = np.random.default_rng(int(scale * 1e3) + 1)
    tw = rng.normal(size=6)
    tw[:3] *= scale / max(np.linalg.norm(tw[:3]), 1e-300)
    E = oracle_mod.exp_se3(tw)
    ref = scipy.linalg.expm(_twist_matrix(tw))
    np.testing.assert_allclose(E, ref, rtol=0, atol=1e-13)
    R = E[:3, :3]
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)


def test_quartic_step_constructed_roots(oracle_mod):
    """G'(t) = 4 S4 (t - r1)(t - r2)(t - r3) with S4 < 0 and 0 < r1 < r2 < r3
    rises from t = 0 and turns down first at r1."""
    for r1, r2, r3, S4 in [(0.3, 1.0, 2.0, -1.0), (1e-4, 5e-4, 3e-3, -2e6), (0.5, 0.7, 9.0, -0.01)]:
        c3, c2, c1, c0 = 4 * S4, -4 * S4 * (r1 + r2 + r3), 4 * S4 * (r1 * r2 + r1 * r3 + r2 * r3), \
            -4 * S4 * r1 * r2 * r3
        S = [1.0, c0, c1 / 2, c2 / 3, c3 / 4]
        t, ok = oracle_mod.quartic_step(S)
        assert ok and t == pytest.approx(r1, rel=1e-9)


def test_quartic_step_roots_orders_of_magnitude_apart(oracle_mod):
    """G' = 4 S4 (t - r1)(t - r2)(t - r3) with S4 < 0 and roots -3.3e-3, -5.5e-8,
    2.8e-8 (the spread met on a serving-workload pair): the model rises from
    t = 0 and turns down at the only positive root, 2.8e-8."""
    r1, r2, r3, S4 = -3.3e-3, -5.5e-8, 2.8e-8, -1.7e29
    c3, c2, c1, c0 = 4 * S4, -4 * S4 * (r1 + r2 + r3), 4 * S4 * (r1 * r2 + r1 * r3 + r2 * r3), \
        -4 * S4 * r1 * r2 * r3
    t, ok = oracle_mod.quartic_step([1.0, c0, c1 / 2, c2 / 3, c3 / 4])
    assert ok and t == pytest.approx(r3, rel=1e-7)


def test_quartic_step_brute_force(oracle_mod):
    """First local maximum of the quartic on t > 0 found by scanning a fine grid."""
    rng = np.random.default_rng(21)
    checked = 0
    for _ in range(300):
        S = rng.normal(size=5)
        S[1] = abs(S[1]) + 0.1
        t, ok = oracle_mod.quartic_step(S)
        ts = np.linspace(1e-6, 20.0, 400001)
        q = S[0] + S[1] * ts + S[2] * ts ** 2 + S[3] * ts ** 3 + S[4] * ts ** 4
        interior = np.flatnonzero((q[1:-1] > q[:-2]) & (q[1:-1] >= q[2:])) + 1
        if interior.size == 0:
            # no maximiser inside the scanned range: the model is monotone there
            assert (not ok) or t > 19.9
            continue
        assert ok
        assert t == pytest.approx(ts[interior[0]], abs=2 * (ts[1] - ts[0]))
        checked += 1
    assert checked > 50


def test_quartic_step_monotone_model_has_no_maximiser(oracle_mod):
    t, ok = oracle_mod.quartic_step([0.0, 1.0, 1.0, 1.0, 1.0])
    assert not ok
    t2, ok2 = oracle_mod.quartic_step([0.0, 2.0, -4.0, 0.0, 0.0], order=2)
    assert ok2 and t2 == pytest.approx(0.25)


# --------------------------------------------------------------------------
# lengthscale schedule (Table 1) and the full solve (Problem 1)
# --------------------------------------------------------------------------

def _golden_table1():
    vals = {}
    with open(os.path.join(HERE, "golden", "table1_parameters.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_table1_schedule_and_defaults(oracle_mod):
    g = _golden_table1()
    p = _params(oracle_mod, schedule="table1")
    ells = oracle_mod.ell_schedule(p, 30)
    assert ells[0:3] == [g["ell_iter_1_to_3"]] * 3
    assert ells[3:10] == [g["ell_after_iter_3"]] * 7
    assert ells[10:20] == [g["ell_after_iter_10"]] * 10
    assert ells[20:] == [g["ell_after_iter_20"]] * 10
    d = oracle_mod.Params()
    assert d.eps_pose == g["eps_pose"] and d.eps_grad == g["eps_grad"]
    assert d.kcut == g["sparsification"]


def test_decay_schedule(oracle_mod):
    p = _params(oracle_mod)
    ells = oracle_mod.ell_schedule(p, 40)
    assert ells[0] == 0.15 and ells[-1] == 0.02
    k = next(i for i, e in enumerate(ells) if e == 0.02)
    assert k == math.ceil(math.log(0.02 / 0.15) / math.log(0.9))
    np.testing.assert_allclose(ells[:k], 0.15 * 0.9 ** np.arange(k), rtol=1e-14)


def test_align_identical_clouds_stays_at_identity(oracle_mod):
    d = synth.planes_pair(800, 800, seed=99)
    p = _params(oracle_mod, max_iters=30)
    r = oracle_mod.align(d["X"], d["FX"], d["X"], d["FX"], np.eye(4), p)
    ang, tr = oracle_mod.pose_error(r["P"], np.eye(4))
    assert ang < 1e-9 and tr < 1e-9


def test_align_recovers_known_transform(oracle_mod):
    """Problem 1 on the three-planes workload: the solve moves from the
    identity to the true relative pose, up to the noise floor set by the
    independent resampling and 5 mm noise."""
    d = synth.planes_pair()
    p = _params(oracle_mod)
    ang0, tr0 = oracle_mod.pose_error(np.eye(4), d["P_gt"])
    r = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), p)
    ang, tr = oracle_mod.pose_error(r["P"], d["P_gt"])
    assert r["converged"]
    assert ang0 > 0.08 and tr0 > 0.04
    assert ang < 5e-3 and tr < 5e-3


def test_scale_parameters_only_scale(oracle_mod):
    """sigma scales F and its derivatives uniformly and the step length
    absorbs it; a^2 = b^2 = 7 (the paper's worked example) traces the same
    path as a = b = 1 because t absorbs a common metric factor."""
    d = synth.planes_pair(600, 600, seed=5)
    base = _params(oracle_mod, max_iters=12)
    r0 = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), base)
    r1 = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4),
                          _params(oracle_mod, max_iters=12, sigma=0.1))
    r2 = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4),
                          _params(oracle_mod, max_iters=12, a2=7.0, b2=7.0))
    for r in (r1, r2):
        ang, tr = oracle_mod.pose_error(r["P"], r0["P"])
        assert ang < 1e-10 and tr < 1e-10


def test_trajectory_ground_truth_composes():
    # the relative poses the odometry test scores against chain to the
    # absolute camera poses: T_wc[k+1] = T_wc[k] P_gt[k]
    tr = synth.room_trajectory(n_frames=4, n_points=300, width=96, height=72,
                               seed=synth.seed_for(6, 2))
    for k in range(3):
        assert np.allclose(tr["T_wc"][k + 1], tr["T_wc"][k] @ tr["P_gt"][k], atol=1e-12)
    # a frame's points seen from the next camera: x_k = P_gt[k] x_{k+1} for a
    # static world point (checked on a synthetic point, not the sampled ones)
    w = np.array([1.5, 2.0, 0.7, 1.0])
    xk = np.linalg.inv(tr["T_wc"][0]) @ w
    xk1 = np.linalg.inv(tr["T_wc"][1]) @ w
    assert np.allclose(tr["P_gt"][0] @ xk1, xk, atol=1e-12)


# ---- semi-dense front end (oracle/frontend.py) -----------------------------

def test_frontend_percentile_is_numpys_linear_method():
    from oracle import frontend
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 100, 1001):
        v = rng.random(n).astype(np.float32)
        for q in (0.0, 12.5, 50.0, 80.0, 99.9, 100.0):
            assert frontend.percentile_linear(v, q) == np.percentile(v.astype(np.float64), q)


def test_frontend_gradient_matches_numpy_and_a_pixel_loop():
    from oracle import frontend
    rng = np.random.default_rng(4)
    img = rng.random((9, 13)).astype(np.float32)
    gx, gy = frontend.gradient_fp32(img)
    ngy, ngx = np.gradient(img.astype(np.float64))
    assert np.allclose(gx, ngx, atol=1e-6) and np.allclose(gy, ngy, atol=1e-6)
    # pixel loop, FP32 arithmetic
    for y in range(9):
        for x in range(13):
            if 0 < x < 12:
                ref = np.float32(0.5) * (img[y, x + 1] - img[y, x - 1])
            elif x == 0:
                ref = img[y, 1] - img[y, 0]
            else:
                ref = img[y, 12] - img[y, 11]
            assert gx[y, x] == ref


def test_frontend_selection_on_a_hand_built_image():
    # a step edge in V between columns 3 and 4 of an 8 x 8 image: the
    # gradient is nonzero only on columns 3 and 4; with half the pixels
    # invalid (depth 0) and the 60th percentile, exactly the edge pixels of
    # the valid rows survive, in raster order, back-projected by the pinhole
    from oracle import frontend
    H, W = 8, 8
    hsv = np.zeros((H, W, 3), np.float32)
    hsv[:, 4:, 2] = 1.0
    hsv[..., 0] = 0.25
    depth = np.full((H, W), 2.0, np.float32)
    depth[1::2, :] = 0.0
    xyz, feats, idx = frontend.select(depth, hsv, fx=4.0, fy=4.0, cx=3.5, cy=3.5,
                                      percentile=60.0)
    rows = np.arange(0, H, 2)
    want = np.sort(np.concatenate([rows * W + 3, rows * W + 4]))
    assert np.array_equal(idx, want)
    assert np.allclose(xyz[:, 2], 2.0)
    assert np.allclose(xyz[:, 0], (idx % W - 3.5) / 4.0 * 2.0)
    assert np.allclose(feats[:, 3], 1.0)          # 0.5 / 0.05 clipped to 1
    assert np.allclose(feats[:, 0], 0.25)
    # subsampling takes evenly spaced ranks
    _, _, idx2 = frontend.select(depth, hsv, fx=4.0, fy=4.0, cx=3.5, cy=3.5, percentile=60.0,
                                 max_points=3)
    m = want.size
    assert np.array_equal(idx2, want[(np.arange(3) * m) // 3])
