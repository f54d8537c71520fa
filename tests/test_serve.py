"""Request loop (cvo_submit / cvo_poll): continuous batching of frame-pair
solves, called through the C ABI.

Each request runs the same iteration as cvo_align; only the team of blocks
that solves it (so the order of the FP64 sums over blocks) depends on what
else is in flight. Every result must therefore be the same alone and in a
mix within the pose tolerance (1e-4 rad, 1e-4 m), and match the FP64 oracle.
"""
import time

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


def _wait_all(ctx, tickets, timeout_s=120.0):
    out = {}
    t_end = time.time() + timeout_s
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = ctx.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() < t_end, "requests did not finish"
        time.sleep(0.0005)
    return [out[t] for t in tickets]


@pytest.fixture(scope="module")
def frames():
    # two keyframes, frames of uneven size rendered against each
    kf = [synth.planes_pair(3000, 3000, seed=synth.seed_for(5, k)) for k in range(2)]
    rng = np.random.default_rng(synth.seed_for(5, 99))
    fr = []
    for i in range(12):
        k = i % 2
        n = int(rng.integers(600, 4000))
        d = synth.planes_pair(3000, n, seed=synth.seed_for(5, 100 + i))
        fr.append((k, d))
    return kf, fr


def test_same_result_alone_and_in_the_mix(cvo, frames):
    kf, fr = frames
    with cvo.Context(device=0) as ctx:
        keys = [ctx.set_cloud(d["X"], d["FX"]) for d in kf]
        # the frames are aligned to their own X; give each its keyframe's X
        # by re-rendering: use the frame's own target as a private keyframe
        own = [ctx.set_cloud(d["X"], d["FX"]) for _, d in fr]
        probe = 3
        _, dp = fr[probe]
        alone = _wait_all(ctx, [ctx.submit(own[probe], dp["Z"], dp["FZ"])])[0]
        mix = [ctx.submit(own[i], d["Z"], d["FZ"]) for i, (_, d) in enumerate(fr)]
        mix += [ctx.submit(keys[k], d["Z"], d["FZ"]) for k, d in fr]   # shared keyframes too
        res = _wait_all(ctx, mix)
        for P, st, q_ms, lat_ms in res:
            assert st["status"] == 0
            assert lat_ms >= q_ms >= 0.0 and st["device_ms"] > 0.0
        ang, tr = oracle.pose_error(alone[0], res[probe][0])
        assert ang < POSE_TOL and tr < POSE_TOL, (ang, tr)
        assert abs(alone[1]["iters"] - res[probe][1]["iters"]) <= 2
        ctx.serve_stop()
        # plain solves of the same pairs agree with the served ones
        for i in (0, probe, 7):
            s = ctx.set_cloud(fr[i][1]["Z"], fr[i][1]["FZ"])
            P, st = ctx.align(own[i], s)
            ang, tr = oracle.pose_error(P, res[i][0])
            assert ang < POSE_TOL and tr < POSE_TOL, (i, ang, tr)
            ctx.release(s)


def test_served_result_matches_oracle(cvo):
    d = synth.planes_pair(900, 700, seed=synth.seed_for(5, 7))
    with cvo.Context(device=0) as ctx:
        k = ctx.set_cloud(d["X"], d["FX"])
        noise = [synth.planes_pair(900, 500 + 100 * i, seed=synth.seed_for(5, 20 + i))
                 for i in range(4)]
        ts = [ctx.submit(k, d["Z"], d["FZ"])] + [ctx.submit(k, e["Z"], e["FZ"]) for e in noise]
        res = _wait_all(ctx, ts)
    prm = oracle.Params()
    ref = oracle.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), prm)
    ang, tr = oracle.pose_error(res[0][0], ref["P"])
    assert ang < POSE_TOL and tr < POSE_TOL, (ang, tr)
    assert res[0][1]["iters"] == ref["iters"]


def test_admission_by_budget(cvo):
    d = synth.planes_pair(2000, 2000, seed=synth.seed_for(5, 8))
    small = [synth.planes_pair(2000, 1500, seed=synth.seed_for(5, 30 + i)) for i in range(6)]
    # enough for the keyframe and about two requests at a time
    with cvo.Context(device=0, hbm_budget=6 << 20) as ctx:
        k = ctx.set_cloud(d["X"], d["FX"])
        ts = [ctx.submit(k, e["Z"], e["FZ"]) for e in small]
        res = _wait_all(ctx, ts)
        assert all(r[1]["status"] == 0 for r in res)
        # later requests waited for memory
        assert max(r[2] for r in res) > 0.0
        # a frame that can never fit is refused, and the loop goes on
        big = synth.planes_pair(2000, 200000, seed=synth.seed_for(5, 40))
        tb = ctx.submit(k, big["Z"], big["FZ"])
        tk = ctx.submit(k, small[0]["Z"], small[0]["FZ"])
        rb, rk = _wait_all(ctx, [tb, tk])
        assert rb[1]["status"] == cvo.CVO_ERR_OUT_OF_BUDGET
        assert rk[1]["status"] == 0
        ang, tr = oracle.pose_error(rk[0], res[0][0])
        assert ang < POSE_TOL and tr < POSE_TOL


def test_busy_rules_and_tickets(cvo):
    d = synth.planes_pair(1500, 1500, seed=synth.seed_for(5, 9))
    with cvo.Context(device=0) as ctx:
        k = ctx.set_cloud(d["X"], d["FX"])
        s = ctx.set_cloud(d["Z"], d["FZ"])
        ctx.serve_start(linger_ms=1000.0)   # keep the serving kernel up
        t = ctx.submit(k, d["Z"], d["FZ"])
        with pytest.raises(cvo.CvoError) as e:
            ctx.release(k)                   # a request still names it
        assert e.value.code == cvo.CVO_ERR_BUSY
        with pytest.raises(cvo.CvoError) as e:
            ctx.align(k, s)                  # whole-GPU solves wait for the loop to end
        assert e.value.code == cvo.CVO_ERR_BUSY
        r = _wait_all(ctx, [t])[0]
        assert r[1]["status"] == 0
        with pytest.raises(cvo.CvoError) as e:
            ctx.poll(t)                      # retired
        assert e.value.code == cvo.CVO_ERR_NOT_FOUND
        with pytest.raises(cvo.CvoError) as e:
            ctx.submit(k + 50, d["Z"], d["FZ"])
        assert e.value.code == cvo.CVO_ERR_NOT_FOUND
        with pytest.raises(cvo.CvoError) as e:
            ctx.submit(k, d["Z"][:0], d["FZ"][:0])
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        ctx.serve_stop()
        P, st = ctx.align(k, s)
        ang, tr = oracle.pose_error(P, r[0])
        assert ang < POSE_TOL and tr < POSE_TOL
        ctx.release(k)


def test_idle_bound_of_the_serving_kernel(cvo):
    """A bounded device wait that runs out: the loop never tells the serving
    kernel to leave (linger far beyond the test), so the kernel's own idle
    bound ends it; the host reads the status, counts the exit, and the next
    request starts a new kernel and completes."""
    d = synth.planes_pair(1200, 1000, seed=synth.seed_for(5, 50))
    with cvo.Context(device=0) as ctx:
        k = ctx.set_cloud(d["X"], d["FX"])
        ctx.serve_start(linger_ms=1e6, idle_limit_ms=50.0)
        r1 = _wait_all(ctx, [ctx.submit(k, d["Z"], d["FZ"])])[0]
        t_end = time.time() + 20.0
        while ctx.serve_stats()["idle_exits"] < 1:
            assert time.time() < t_end, "the serving kernel did not leave on its idle bound"
            time.sleep(0.01)
        r2 = _wait_all(ctx, [ctx.submit(k, d["Z"], d["FZ"])])[0]
        st = ctx.serve_stats()
        assert r1[1]["status"] == 0 and r2[1]["status"] == 0
        assert st["kernels_launched"] == 2 and st["idle_exits"] >= 1
        assert st["submitted"] == 2 and st["completed"] == 2 and st["failed"] == 0
        ang, tr = oracle.pose_error(r1[0], r2[0])
        assert ang < POSE_TOL and tr < POSE_TOL
