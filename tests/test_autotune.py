"""Autotuner of the performance parameters (cvo_autotune), called through the
C ABI: it times whole solves, keeps the fastest setting in the context, and
must not change results beyond the pose tolerance (1e-4 rad, 1e-4 m): the
cutoff test is exact, only the order of the FP64 sums over blocks moves."""
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


def test_autotune_keeps_results_and_the_fastest_setting(cvo):
    d = synth.planes_pair(3000, 2800, seed=synth.seed_for(1, 31))
    sp = cvo.cvo_tune_space()
    sp.n_cell, sp.n_cluster, sp.n_chunk, sp.n_cluster_cost, sp.reps = 2, 2, 2, 2, 1
    sp.cell_factor[0], sp.cell_factor[1] = 0.6, 1.0
    sp.cluster_factor[0], sp.cluster_factor[1] = 1.5, 2.5
    sp.cost_chunk[0], sp.cost_chunk[1] = 16, 32
    sp.cost_cluster[0], sp.cost_cluster[1] = 32, 96
    with cvo.Context(device=0) as ctx:
        cell0, chunk0 = ctx.params.cell_factor, ctx.params.cost_chunk   # the starting setting
        t, s = ctx.set_cloud(d["X"], d["FX"]), ctx.set_cloud(d["Z"], d["FZ"])
        P0, _ = ctx.align(t, s)
        rep = ctx.autotune(t, s, sp)
        assert rep["candidates"] == 1 + 8
        assert 0.0 < rep["best_ms"] <= rep["start_ms"]
        assert rep["cell_factor"] in (cell0, 0.6, 1.0) and rep["cost_chunk"] in (chunk0, 16, 32)
        P1, st = ctx.align(t, s)
        ang, tr = oracle.pose_error(P0, P1)
        assert ang < POSE_TOL and tr < POSE_TOL
        # a batch holds the clouds: no tuning then
        with ctx.batch([t], [s]) as b:
            with pytest.raises(cvo.CvoError) as e:
                ctx.autotune(t, s, sp)
            assert e.value.code == cvo.CVO_ERR_BUSY
        bad = cvo.cvo_tune_space()
        bad.n_cell = 1
        bad.cell_factor[0] = 0.1
        with pytest.raises(cvo.CvoError) as e:
            ctx.autotune(t, s, bad)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
