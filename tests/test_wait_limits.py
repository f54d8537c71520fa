"""Failure detection of the device-side waits, on the GPU, without a fault:
every wait of the persistent solve (the team barrier, the join of a queued
team) is bounded, and a block whose bound runs out leaves with a timeout
status that the host reads as CVO_ERR_TIMEOUT. Here the bounds are made tiny
(cvo_set_wait_limits) so that ordinary solves run them out; nothing is
broken on purpose and no wait is unbounded. Afterwards the same context, with
the default bounds back, solves normally and matches the FP64 oracle."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-4
DEFAULT_POLLS, DEFAULT_JOIN_MS = 1 << 22, 60000.0


@pytest.fixture(scope="module")
def cvo():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1904_02266_gb300 as m
    return m


def test_tiny_wait_bounds_time_out_and_the_context_recovers(cvo, oracle_mod):
    d = synth.planes_pair(1500, 1400, seed=synth.seed_for(1, 61))
    prm = oracle_mod.Params(max_iters=30)
    with cvo.Context(device=0, max_iters=30) as ctx:
        ht, hs = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        P_ok, st_ok = ctx.align(ht, hs)
        # one poll per barrier wait: the early blocks of the first barrier give up
        ctx.set_wait_limits(1, DEFAULT_JOIN_MS)
        with pytest.raises(cvo.CvoError) as e:
            ctx.align(ht, hs)
        assert e.value.code == cvo.CVO_ERR_TIMEOUT
        # the bounds back: the same context and plan solve as before, bit for bit
        ctx.set_wait_limits(DEFAULT_POLLS, DEFAULT_JOIN_MS)
        P2, st2 = ctx.align(ht, hs)
        assert np.array_equal(P2, P_ok) and st2["iters"] == st_ok["iters"]
        ref = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), prm)
        ang, tr = oracle_mod.pose_error(P2, ref["P"])
        assert ang < POSE_TOL and tr < POSE_TOL, (ang, tr)


def test_batch_reports_per_pair_timeouts_and_recovers(cvo, oracle_mod):
    pairs = synth.batch_pairs(n_pairs=12, seed=synth.seed_for(3, 61), n_range=(600, 6000))
    with cvo.Context(device=0, max_iters=30) as ctx:
        hs = [(ctx.set_cloud(p["X"], p["FX"]), ctx.set_cloud(p["Z"], p["FZ"])) for p in pairs]
        ell0 = [p["ell0"] for p in pairs]
        P0 = np.stack([np.eye(4)] * len(pairs))
        with ctx.batch([t for t, _ in hs], [s for _, s in hs], ell0=ell0) as b:
            teams = b.info()["teams"]
            assert teams.max() > 1
            P_ok, st_ok = b.run(P0)
            # one poll per barrier wait and a join bound far below a pair's solve
            ctx.set_wait_limits(1, 1e-3)
            P, st, code = b.run(P0, check=False)
            codes = [s["status"] for s in st]
            assert code == cvo.CVO_ERR_TIMEOUT
            assert set(codes) <= {cvo.CVO_OK, cvo.CVO_ERR_TIMEOUT}, codes
            assert codes.count(cvo.CVO_ERR_TIMEOUT) >= 1
            # a pair that finished anyway ran the ordinary solve
            for i, c in enumerate(codes):
                if c == cvo.CVO_OK:
                    assert max(oracle_mod.pose_error(P[i], P_ok[i])) < 1e-7
            # the bounds back: the replayed graph gives the first run's results
            ctx.set_wait_limits(DEFAULT_POLLS, DEFAULT_JOIN_MS)
            P2, st2 = b.run(P0)
            assert all(s["status"] == cvo.CVO_OK for s in st2)
            assert np.array_equal(P2, P_ok)
        for i in (0, len(pairs) - 1):
            p = pairs[i]
            prm = oracle_mod.Params(max_iters=30, ell0=p["ell0"])
            ref = oracle_mod.align(p["X"], p["FX"], p["Z"], p["FZ"], np.eye(4), prm)
            ang, tr = oracle_mod.pose_error(P2[i], ref["P"])
            assert ang < POSE_TOL and tr < POSE_TOL, (i, ang, tr)


def test_wait_limits_are_validated(cvo):
    with cvo.Context(device=0) as ctx:
        for polls, ms in ((0, 1.0), ((1 << 30) + 1, 1.0), (10, 0.0), (10, -1.0), (10, 2e7)):
            with pytest.raises(cvo.CvoError) as e:
                ctx.set_wait_limits(polls, ms)
            assert e.value.code == cvo.CVO_ERR_INVALID_ARG
