"""Odometry over a stream (the evaluation protocol of Sec. 5 on a synthetic
trajectory): consecutive frames of a camera moving through a rendered room are
aligned, all pairs in one batch, and the relative-pose errors use the pose
distances of Sec. 2. Every pair must match the FP64 oracle's solve within the
pose tolerance (1e-4 rad, 1e-4 m); the errors against the ground truth are
noise-limited and only bounded loosely."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-4


@pytest.fixture(scope="module")
def cvo():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1904_02266_gb300 as m
    return m


def test_trajectory_pairs_match_oracle_and_truth(cvo):
    tr = synth.room_trajectory(n_frames=6, n_points=1500, width=320, height=240,
                               seed=synth.seed_for(6, 1))
    fr = tr["frames"]
    n = len(fr) - 1
    with cvo.Context(device=0) as ctx:
        h = [ctx.set_cloud(X, F) for X, F in fr]
        with ctx.batch(h[:-1], h[1:]) as b:
            P, st = b.run(np.stack([np.eye(4)] * n))
    prm = oracle.Params()
    rot, trans = [], []
    for k in range(n):
        assert st[k]["status"] == 0
        ref = oracle.align(fr[k][0], fr[k][1], fr[k + 1][0], fr[k + 1][1], np.eye(4), prm)
        ang, t = oracle.pose_error(P[k], ref["P"])
        assert ang < POSE_TOL and t < POSE_TOL, (k, ang, t)
        a_gt, t_gt = oracle.pose_error(P[k], tr["P_gt"][k])
        rot.append(a_gt)
        trans.append(t_gt)
    # 3 deg / 3 cm steps, recovered to below the step size at this small
    # size (1500 points per 320 x 240 frame)
    assert np.median(rot) < np.deg2rad(1.0) and np.median(trans) < 0.05, (rot, trans)
    # chaining the relative poses reproduces the trajectory up to the summed error
    T = np.eye(4)
    for k in range(n):
        T = T @ P[k]
    T_gt = np.linalg.inv(tr["T_wc"][0]) @ tr["T_wc"][-1]
    a_end, t_end = oracle.pose_error(T, T_gt)
    assert a_end <= sum(rot) + 1e-9 + 0.02 and t_end <= sum(trans) + 0.05
