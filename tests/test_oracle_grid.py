"""The oracle's two searches of the pairs within the cutoff (Sec. 5
sparsification): the exhaustive loop over every target point and the cell
search over the 27 cells of edge r_c around each source point. The cell
search visits each source point's candidates in the exhaustive loop's order,
so every sum, the kept-pair count and a whole solve must agree bit for bit;
a cell search that missed a neighbour (a wrong cell edge, an off-by-one in
the 27-cell window, a point outside the grid) changes the kept count."""
import numpy as np
import pytest

import synth


def _both(oracle, X, FX, Z, FZ, P, ell, xi=None, **kw):
    out = []
    for search in ("exhaustive", "grid"):
        p = oracle.Params(search=search, **kw)
        out.append(oracle.pair_sums(X, FX, Z, FZ, P, ell, p, xi=xi))
    return out


def _same(a, b):
    assert a["nnz"] == b["nnz"]
    assert a["F"] == b["F"]
    assert np.array_equal(a["dF_domega"], b["dF_domega"])
    assert np.array_equal(a["dF_dv"], b["dF_dv"])
    assert np.array_equal(a["S"], b["S"])


@pytest.mark.parametrize("ell", [0.02, 0.05, 0.15, 0.6])
@pytest.mark.parametrize("mode", ["none", "kernel", "dot"])
def test_grid_search_gives_the_exhaustive_bits(oracle_mod, ell, mode):
    cm = {"none": oracle_mod.COLOR_NONE, "kernel": oracle_mod.COLOR_KERNEL,
          "dot": oracle_mod.COLOR_DOT}[mode]
    d = synth.planes_pair(1800, 1500, seed=synth.seed_for(1, 71))
    rng = np.random.default_rng(4)
    P = synth.random_motion(rng, 3.0, 0.04) @ d["P_gt"]
    xi = rng.normal(size=6)
    e, g = _both(oracle_mod, d["X"], d["FX"], d["Z"], d["FZ"], P, ell, xi=xi, color_mode=cm)
    assert e["nnz"] > 0
    _same(e, g)


def test_grid_search_on_the_room_and_far_away_sources(oracle_mod):
    """Room frames (surfaces at many depths), a pose that moves part of the
    source out of the target's bounding box, and one that moves all of it
    far away (no pair kept)."""
    d = synth.room_pair(4000, seed=synth.seed_for(2, 71))
    for P, ell in ((np.eye(4), 0.03), (synth.rigid(np.eye(3), np.array([2.5, 0.0, 0.0])), 0.1),
                   (synth.rigid(np.eye(3), np.array([0.0, 60.0, 0.0])), 0.1)):
        e, g = _both(oracle_mod, d["X"], d["FX"], d["Z"], d["FZ"], P, ell, xi=np.ones(6))
        _same(e, g)
    assert e["nnz"] == 0


def test_grid_search_with_coincident_and_boundary_points(oracle_mod):
    """Many copies of a point, and target points placed exactly at the cutoff
    distance (in exact binary fractions) around a source point, on and off
    the cell boundaries."""
    ell, kcut = 0.0625, 1e-3
    rc = ell * np.sqrt(2 * np.log(1 / kcut))
    z = np.array([[0.5, 0.25, 0.125]])
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                     [0.6, 0.8, 0.0], [0.0, -0.6, 0.8]])
    X = np.concatenate([z + rc * dirs * (1 - 1e-12), z + rc * dirs * (1 + 1e-12),
                        np.repeat(z, 7, axis=0), z + 3 * rc * dirs])
    Z = np.concatenate([z, z + 1e-3])
    e, g = _both(oracle_mod, X, None, Z, None, np.eye(4), ell, color_mode=oracle_mod.COLOR_NONE,
                 kcut=kcut)
    _same(e, g)
    assert e["nnz"] >= 2 * (8 + 7)


def test_grid_search_per_source_sums_and_solve(oracle_mod):
    d = synth.planes_pair(900, 800, seed=synth.seed_for(1, 72))
    js = np.array([0, 5, 799, 400])
    a = oracle_mod.pair_sums_per_j(d["X"], d["FX"], d["Z"], d["FZ"], d["P_gt"], 0.05,
                                   oracle_mod.Params(), js, xi=np.ones(6))
    b = oracle_mod.pair_sums_per_j(d["X"], d["FX"], d["Z"], d["FZ"], d["P_gt"], 0.05,
                                   oracle_mod.Params(search="grid"), js, xi=np.ones(6))
    assert np.array_equal(a, b)
    r_e = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4),
                           oracle_mod.Params(max_iters=40))
    r_g = oracle_mod.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4),
                           oracle_mod.Params(max_iters=40, search="grid"))
    assert np.array_equal(r_e["P"], r_g["P"])
    assert r_e["iters"] == r_g["iters"] and r_e["pair_evals"] == r_g["pair_evals"]


def test_grid_search_needs_a_cutoff(oracle_mod):
    d = synth.planes_pair(50, 40, seed=3)
    with pytest.raises(ValueError):
        oracle_mod.pair_sums(d["X"], None, d["Z"], None, np.eye(4), 0.1,
                             oracle_mod.Params(search="grid", kcut=0.0))
