"""Randomised properties of the oracle on small sets (hypothesis), beyond the fixed
seeds of the other pins: points anywhere in the periodic unit cube (clumps, exact
duplicates, points next to a face), smoothing lengths spread over an order of
magnitude.

* the pruning tree changes nothing: tree sets and sums equal the brute-force ones;
* the grouped form (Sec. 2.1) equals the per-particle form bit for bit for any g and
  any subset of targets;
* the neighbour relations are those of Sec. 1.1: density sets contain i, hydro sets
  are symmetric (j in N_i iff i in N_j) and exclude i.
"""

import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings, HealthCheck = hyp.given, hyp.settings, hyp.HealthCheck


@st.composite
def particle_sets(draw):
    n = draw(st.integers(1, 160))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    kind = draw(st.sampled_from(["uniform", "clumps", "duplicates", "faces"]))
    if kind == "uniform":
        pos = rng.random((n, 3))
    elif kind == "clumps":
        centres = rng.random((3, 3))
        pos = (centres[rng.integers(0, 3, n)] + 0.02 * rng.standard_normal((n, 3))) % 1.0
    elif kind == "duplicates":
        base = rng.random((max(1, n // 3), 3))
        pos = base[rng.integers(0, len(base), n)]
    else:
        pos = rng.random((n, 3))
        pos[:, 0] = np.where(rng.random(n) < 0.5, 1e-12 * rng.random(n), 1.0 - 1e-12 * rng.random(n))
    pos = np.ascontiguousarray(pos % 1.0)
    pos[pos >= 1.0] = 0.0
    h = np.exp(rng.uniform(np.log(0.02), np.log(0.3), n))
    m = rng.uniform(0.5, 1.5, n) / n
    targets = np.flatnonzero(rng.random(n) < draw(st.floats(0.2, 1.0))).astype(np.int32)
    if len(targets) == 0:
        targets = np.array([0], np.int32)
    g = draw(st.integers(1, 48))
    return pos, h, m, targets, g, rng


SETTINGS = dict(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@settings(**SETTINGS)
@given(particle_sets())
def test_tree_changes_nothing(case):
    pos, h, m, targets, _, _ = case
    for kind in (oracle.DENSITY, oracle.HYDRO):
        a = oracle.ngb_sets(pos, h, targets, kind=kind, use_tree=True)
        b = oracle.ngb_sets(pos, h, targets, kind=kind, use_tree=False)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ta = oracle.density(pos, m, h, targets, use_tree=True)
    tb = oracle.density(pos, m, h, targets, use_tree=False)
    assert np.array_equal(ta["rho"], tb["rho"]) and np.array_equal(ta["nngb"], tb["nngb"])


@settings(**SETTINGS)
@given(particle_sets())
def test_grouped_equals_per_particle(case):
    pos, h, m, targets, g, rng = case
    ref = oracle.density(pos, m, h, targets)
    got = oracle.density_grouped(pos, m, h, g, targets=targets)
    for k in ("rho", "drhodh", "nngb"):
        assert np.array_equal(got[k], ref[k]), k
    n = len(m)
    vel = rng.standard_normal((n, 3))
    u = rng.uniform(0.5, 2.0, n)
    rho = np.maximum(oracle.density(pos, m, h)["rho"], 1e-300)
    f = rng.uniform(0.8, 1.2, n)
    hr = oracle.hydro(pos, vel, m, h, rho, f, u, targets)
    hg = oracle.hydro_grouped(pos, vel, m, h, rho, f, u, g, targets=targets)
    assert np.array_equal(hg["nngb"], hr["nngb"])
    assert np.array_equal(hg["acc"], hr["acc"]) and np.array_equal(hg["dudt"], hr["dudt"])
    assert hg["walks"] == -(-len(targets) // g)


@settings(**SETTINGS)
@given(particle_sets())
def test_neighbour_relations(case):
    pos, h, _, _, _, _ = case
    n = len(h)
    off, idx = oracle.ngb_sets(pos, h, kind=oracle.DENSITY)
    for i in range(n):
        assert i in idx[off[i]:off[i + 1]]
    off, idx = oracle.ngb_sets(pos, h, kind=oracle.HYDRO)
    pairs = {(i, int(j)) for i in range(n) for j in idx[off[i]:off[i + 1]]}
    assert all((j, i) in pairs for i, j in pairs)
    assert all(i != j for i, j in pairs)
