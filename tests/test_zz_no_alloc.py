"""cvo_eval_gradient_static, the gradient pass that allocates no device memory
(for callers that cannot allocate during a call), called through the C ABI.

Its F, gradient and kept-pair count must match cvo_eval's (the context-based
entry point) within the parity tolerances, on two calls in a row that share
the library's static scratch. This file is collected last so that a run that
stops at the first failure has already run every other test.
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


def test_static_gradient_matches_eval_on_consecutive_calls(cvo):
    torch = pytest.importorskip("torch")
    d = synth.planes_pair(3001, 2477, seed=synth.seed_for(1, 41))
    params = cvo.cvo_params_default()
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
    # the same inputs give the same bits, whatever the previous call left behind
    assert np.array_equal(got_all[0], got_all[2])


def test_static_gradient_rejects_bad_sizes(cvo):
    torch = pytest.importorskip("torch")
    params = cvo.cvo_params_default()
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    feats = torch.zeros((0, 5), dtype=torch.float32, device="cuda")
    one = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    one_f = torch.zeros((1, 5), dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_eval_gradient_static(empty, feats, one, one_f, params, np.eye(4), 0.1, out)
    assert e.value.code == cvo.CVO_ERR_INVALID_ARG
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_eval_gradient_static(one, one_f, one, one_f, params, np.eye(4), -1.0, out)
    assert e.value.code == cvo.CVO_ERR_INVALID_ARG
