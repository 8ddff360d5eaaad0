"""The oracle's grouped form (Sec. 2.1, Neighbour Recycling): groups of g consecutive
targets along the curve, one superset walk per group, each member filtering the
superset.  The method is exact, so every output must equal the per-particle form bit for
bit (same neighbour sets, same summation order); the per-particle form is itself pinned
to brute force.  Variable h (clustered sets at converged h) makes the hydro superset
depend on the node hmax term: without it, neighbours through a large h_j go missing."""

import numpy as np
import pytest

import oracle
import sphgen


def _data(kind, n, cfg):
    d = sphgen.make(kind, n, config=cfg)
    m = d["m"].astype(np.float64)
    h, dens = oracle.density_iterate(d["pos"], m, np.full(n, d["h0"]))
    return d, m, h, dens


@pytest.fixture(scope="module", params=[("uniform", 4096, 1), ("clustered", 3001, 2)], ids=["uniform", "clustered"])
def case(request):
    return _data(*request.param)


@pytest.mark.parametrize("g", [1, 3, 16, 64])
@pytest.mark.parametrize("frac", [1.0, 0.3])
def test_grouped_density_equals_per_particle(case, g, frac):
    d, m, h, _ = case
    n = len(m)
    targets = None
    if frac < 1.0:
        rng = np.random.default_rng(7)
        mask = sphgen.active_rank_mask(n, frac, 32.0, rng)
        targets = np.sort(oracle.curve_order(d["pos"])[np.flatnonzero(mask)]).astype(np.int32)
    ref = oracle.density(d["pos"], m, h, targets=targets)
    got = oracle.density_grouped(d["pos"], m, h, g, targets=targets)
    for k in ("rho", "drhodh", "f", "neff", "nngb"):
        assert np.array_equal(got[k], ref[k]), k
    nt = n if targets is None else len(targets)
    assert got["walks"] == -(-nt // g)
    assert got["pair_tests"] >= got["candidates"] >= int(ref["nngb"].sum()) // max(g, 1)


@pytest.mark.parametrize("g", [1, 4, 16, 64])
def test_grouped_hydro_equals_per_particle(case, g):
    d, m, h, dens = case
    args = (d["pos"], d["vel"], m, h, dens["rho"], dens["f"], d["u"])
    ref = oracle.hydro(*args)
    got = oracle.hydro_grouped(*args, g)
    assert np.array_equal(got["acc"], ref["acc"])
    assert np.array_equal(got["dudt"], ref["dudt"])
    assert np.array_equal(got["nngb"], ref["nngb"])
    assert got["walks"] == -(-len(m) // g)


def test_grouped_supersets_grow_with_g_and_tests_follow():
    """Bigger groups walk less and test more: the trade-off the paper tunes."""
    d, m, h, _ = _data("clustered", 3001, 2)
    s = [oracle.density_grouped(d["pos"], m, h, g) for g in (1, 8, 64)]
    walks = [x["walks"] for x in s]
    tests_per_member = [x["pair_tests"] / len(m) for x in s]
    assert walks[0] > walks[1] > walks[2]
    assert tests_per_member[0] < tests_per_member[1] < tests_per_member[2]
    # with g = 1 the superset of each walk is that particle's own candidate list
    assert s[0]["candidates"] == s[0]["pair_tests"]


def test_grouped_edge_cases():
    d, m, h, _ = _data("uniform", 512, 1)
    one = oracle.density_grouped(d["pos"], m, h, 10_000)   # a single group of every particle
    ref = oracle.density(d["pos"], m, h)
    assert one["walks"] == 1 and np.array_equal(one["rho"], ref["rho"])
    empty = oracle.density_grouped(d["pos"], m, h, 8, targets=np.zeros(0, np.int32))
    assert empty["walks"] == 0 and len(empty["rho"]) == 0
    with pytest.raises(ValueError):
        oracle.density_grouped(d["pos"], m, h, 0)


def test_grouped_matches_brute_force_on_a_tiny_set():
    d, m, h, dens = _data("clustered", 400, 9)
    brute = oracle.density(d["pos"], m, h, use_tree=False)
    got = oracle.density_grouped(d["pos"], m, h, 16)
    assert np.array_equal(got["nngb"], brute["nngb"])
    assert np.array_equal(got["rho"], brute["rho"])
    bh = oracle.hydro(d["pos"], d["vel"], m, h, dens["rho"], dens["f"], d["u"], use_tree=False)
    gh = oracle.hydro_grouped(d["pos"], d["vel"], m, h, dens["rho"], dens["f"], d["u"], 16)
    assert np.array_equal(gh["nngb"], bh["nngb"])
    assert np.array_equal(gh["acc"], bh["acc"])
