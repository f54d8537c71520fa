"""Pins of the pose distances of Sec. 2 ("Matrix Lie Group of Motion"): the
rotational distance is read as the rotation angle of R_est R_ref^T (the
paper's Frobenius norm of log(R_est R_ref^T) is sqrt(2) times it) and the
translational one is |T_est - R_est R_ref^T T_ref|, the translation part of
h_est h_ref^{-1}. The oracle's pose_error and the benchmark's own copy
(bench.synth_pose_err) are checked against closed forms and against scipy's
matrix logarithm and rotation-vector routines, never against each other's
formula alone."""
import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import bench
import oracle


def _rot(axis, theta):
    """Rotation by theta about axis, as the matrix exponential of its skew
    matrix (scipy.linalg.expm, independent of the oracle's closed form)."""
    a = np.asarray(axis, dtype=float)
    a = a / np.linalg.norm(a)
    W = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return scipy.linalg.expm(theta * W)


def _pose(R, T):
    P = np.eye(4)
    P[:3, :3] = R
    P[:3, 3] = T
    return P


FUNCS = [oracle.pose_error, bench.synth_pose_err]


@pytest.mark.parametrize("f", FUNCS, ids=["oracle", "bench"])
@pytest.mark.parametrize("theta", [1e-6, 0.01, 0.3, 1.2, 2.5, 3.1])
def test_rotation_about_an_axis_gives_its_angle(f, theta):
    """A pure rotation by theta about a random axis: angle theta (not
    sqrt(2) theta, the Frobenius norm of its logarithm), translation 0."""
    rng = np.random.default_rng(int(theta * 1e6) + 11)
    R = _rot(rng.normal(size=3), theta)
    ang, tr = f(_pose(R, np.zeros(3)), np.eye(4))
    assert ang == pytest.approx(theta, rel=1e-9, abs=1e-12)
    assert tr < 1e-14
    # the paper's Frobenius form is sqrt(2) times the angle
    L = scipy.linalg.logm(R @ np.eye(3).T)
    assert np.linalg.norm(np.real(L), "fro") == pytest.approx(np.sqrt(2.0) * ang, rel=1e-8)


@pytest.mark.parametrize("f", FUNCS, ids=["oracle", "bench"])
def test_pure_translation_gives_its_length(f):
    t = np.array([0.03, -0.04, 0.12])
    ang, tr = f(_pose(np.eye(3), t), np.eye(4))
    assert ang == 0.0
    assert tr == pytest.approx(0.13, rel=1e-14)


@pytest.mark.parametrize("f", FUNCS, ids=["oracle", "bench"])
def test_translation_term_is_that_of_h_est_h_ref_inverse(f):
    """P_ref = (R, T) with a large T, P_est = (R_est, T_est) hand-built: the
    translation distance is |T_est - R_est R^T T| (here worked out by hand:
    1 cm), while |T_est - T| is about 20 cm."""
    R = _rot([0.0, 0.0, 1.0], np.pi / 2)          # 90 deg about z: (x, y) -> (-y, x)
    T = np.array([2.0, 0.0, 0.0])
    R_est = _rot([0.0, 0.0, 1.0], np.pi / 2 + 0.1)
    T_est = np.array([2 * np.cos(0.1) + 0.01, 2 * np.sin(0.1), 0.0])
    # R_est R^T = rotation by 0.1 about z; applied to (2, 0, 0): (2 cos .1, 2 sin .1, 0)
    by_hand = np.linalg.norm(T_est - np.array([2 * np.cos(0.1), 2 * np.sin(0.1), 0.0]))
    ang, tr = f(_pose(R_est, T_est), _pose(R, T))
    assert ang == pytest.approx(0.1, rel=1e-12)
    assert tr == pytest.approx(by_hand, rel=1e-12)
    assert by_hand == pytest.approx(0.01, rel=1e-12)
    assert np.linalg.norm(T_est - T) > 0.19
    # and it is the translation of h_est h_ref^{-1} (numpy's general inverse)
    D = _pose(R_est, T_est) @ np.linalg.inv(_pose(R, T))
    assert tr == pytest.approx(np.linalg.norm(D[:3, 3]), rel=1e-12)


@pytest.mark.parametrize("f", FUNCS, ids=["oracle", "bench"])
def test_random_poses_against_scipy_rotation_vector(f):
    """Random pose pairs: the angle is the norm of scipy's rotation vector of
    R_est R_ref^T; the translation that of h_est h_ref^{-1}; composing both
    poses with a common right factor h_ref -> h_ref g, h_est -> h_est g
    leaves both distances unchanged (they depend on h_est h_ref^{-1} only)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        Pr = _pose(_rot(rng.normal(size=3), rng.uniform(0, 3.0)), rng.normal(size=3))
        Pe = _pose(_rot(rng.normal(size=3), rng.uniform(0, 3.0)), rng.normal(size=3))
        G = _pose(_rot(rng.normal(size=3), rng.uniform(0, 3.0)), rng.normal(size=3))
        ang, tr = f(Pe, Pr)
        rv = Rotation.from_matrix(Pe[:3, :3] @ Pr[:3, :3].T).as_rotvec()
        assert ang == pytest.approx(np.linalg.norm(rv), rel=1e-9, abs=1e-12)
        D = Pe @ np.linalg.inv(Pr)
        assert tr == pytest.approx(np.linalg.norm(D[:3, 3]), rel=1e-9)
        ang2, tr2 = f(Pe @ G, Pr @ G)
        assert ang2 == pytest.approx(ang, rel=1e-9, abs=1e-12)
        assert tr2 == pytest.approx(tr, rel=1e-9, abs=1e-12)


def test_bench_and_oracle_pose_errors_agree():
    rng = np.random.default_rng(9)
    for _ in range(20):
        Pr = _pose(_rot(rng.normal(size=3), rng.uniform(0, 3.0)), rng.normal(size=3))
        Pe = _pose(_rot(rng.normal(size=3), rng.uniform(0, 3.0)), rng.normal(size=3))
        assert np.allclose(oracle.pose_error(Pe, Pr), bench.synth_pose_err(Pe, Pr), rtol=0,
                           atol=1e-15)
