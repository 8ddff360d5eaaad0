"""Pins of the oracle's neighbour sets (Sec. 1.1 definitions).

density: j is a neighbour of i iff |r_ij| < h_i (strict); hydro: iff j != i and
|r_ij| < max(h_i, h_j); distances use the minimum image in the periodic unit cube.
The oracle's brute-force sets are checked against a separate numpy brute force and
against hand-made exact (dyadic) cases; its pruned tree sets are checked against the
brute force.
"""

import numpy as np
import pytest

import oracle
import sphgen


def _numpy_sets(pos, h, kind):
    n = len(pos)
    d = pos[None, :, :] - pos[:, None, :]
    d = d - np.round(d)  # numpy rounds half to even
    r2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    if kind == oracle.DENSITY:
        m = r2 < (h * h)[:, None]
    else:
        m = r2 < np.maximum(h * h, (h * h)[:, None])
        np.fill_diagonal(m, False)
    return [np.flatnonzero(m[i]) for i in range(n)]


def _csr_lists(off, idx):
    return [idx[off[i]:off[i + 1]] for i in range(len(off) - 1)]


@pytest.mark.parametrize("kind", [oracle.DENSITY, oracle.HYDRO])
def test_brute_force_matches_numpy(kind):
    rng = np.random.default_rng(5)
    pos = rng.random((400, 3))
    h = rng.uniform(0.05, 0.2, 400)
    off, idx = oracle.ngb_sets(pos, h, kind=kind, use_tree=False)
    ref = _numpy_sets(pos, h, kind)
    for a, b in zip(_csr_lists(off, idx), ref):
        assert np.array_equal(a, b)


def test_exact_boundary_and_periodic_wrap():
    # dyadic positions: every difference below is exact
    pos = np.array([[0.0625, 0.5, 0.5],    # 0
                    [0.9375, 0.5, 0.5],    # 1: 0.125 from 0 through the x boundary
                    [0.0625, 0.5, 0.625],  # 2: 0.125 from 0 along z
                    [0.5, 0.5, 0.5]])      # 3: far
    h = np.array([0.125, 0.25, 0.0625, 0.01])
    off, idx = oracle.ngb_sets(pos, h, kind=oracle.DENSITY, use_tree=False)
    sets = _csr_lists(off, idx)
    assert list(sets[0]) == [0]            # r = h exactly is not a neighbour
    assert list(sets[1]) == [0, 1, 2]      # sqrt(2)*0.125 < 0.25 through the wrap
    assert list(sets[3]) == [3]
    h2 = h.copy()
    h2[0] = np.nextafter(0.125, 1.0)
    sets = _csr_lists(*oracle.ngb_sets(pos, h2, kind=oracle.DENSITY, use_tree=False))
    assert list(sets[0]) == [0, 1, 2]
    # hydro uses max(h_i, h_j): 0 sees 1 through h_1, and excludes itself
    sets = _csr_lists(*oracle.ngb_sets(pos, h, kind=oracle.HYDRO, use_tree=False))
    assert list(sets[0]) == [1] and list(sets[2]) == [1] and list(sets[3]) == []


def test_distance_symmetry_bitwise():
    rng = np.random.default_rng(6)
    pos = rng.random((1000, 3))
    pi = rng.integers(0, 1000, 5000)
    pj = rng.integers(0, 1000, 5000)
    assert np.array_equal(oracle.pair_r2(pos, pi, pj), oracle.pair_r2(pos, pj, pi))


@pytest.mark.parametrize("kind", [oracle.DENSITY, oracle.HYDRO])
@pytest.mark.parametrize("dist", ["uniform", "clustered"])
def test_tree_sets_equal_brute_force(kind, dist):
    d = sphgen.make(dist, 3000, config=9, with_hydro=False)
    rng = np.random.default_rng(7)
    h = d["h0"] * rng.uniform(0.3, 1.5, 3000)
    a = oracle.ngb_sets(d["pos"], h, kind=kind, use_tree=False)
    b = oracle.ngb_sets(d["pos"], h, kind=kind, use_tree=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
