"""Pins of the oracle's Peano-Hilbert keys and stable order (Sec. 1: Hilbert ordering).

The curve variant is fixed by the properties that make it a Hilbert curve at all, each
checked by brute force on small grids: the index is a bijection, consecutive indices
are face-adjacent cells, every aligned block of 8^l indices is one octree cube, and
the curve on a 2^b grid is the coarse version of the curve on any finer grid.
"""

import numpy as np
import pytest

import oracle


def _grid(b):
    g = np.arange(2 ** b, dtype=np.uint32)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


@pytest.mark.parametrize("bits", [1, 2, 3, 4, 5])
def test_bijection_and_adjacency(bits):
    cells = _grid(bits)
    keys = oracle.hilbert_cells(cells, bits)
    assert np.array_equal(np.sort(keys), np.arange(8 ** bits, dtype=np.uint64))
    order = np.argsort(keys)
    walk = cells[order].astype(np.int64)
    steps = np.abs(np.diff(walk, axis=0)).sum(axis=1)
    assert np.all(steps == 1), "consecutive Hilbert cells must share a face"
    assert keys[0] == 0 and np.all(cells[order[0]] == 0), "the curve starts at the origin"


@pytest.mark.parametrize("bits", [2, 3, 4])
def test_octree_blocks(bits):
    cells = _grid(bits)
    keys = oracle.hilbert_cells(cells, bits)
    for level in range(1, bits + 1):
        shift = 3 * (bits - level)
        prefix = keys >> np.uint64(shift)
        coarse = cells >> np.uint32(bits - level)
        # every key prefix maps to exactly one coarse cube and vice versa
        pairs = np.unique(np.concatenate([prefix[:, None].astype(np.int64), coarse.astype(np.int64)], 1), axis=0)
        assert len(pairs) == 8 ** level
        assert len(np.unique(pairs[:, 0])) == 8 ** level


@pytest.mark.parametrize("bits,finer", [(2, 5), (3, 7), (4, 21)])
def test_coarse_curve_nests_in_fine_curve(bits, finer):
    cells = _grid(bits)
    kb = oracle.hilbert_cells(cells, bits)
    kf = oracle.hilbert_cells(cells << np.uint32(finer - bits), finer)
    assert np.array_equal(kf >> np.uint64(3 * (finer - bits)), kb)


def test_position_keys_use_the_2_21_grid():
    rng = np.random.default_rng(1)
    cells = rng.integers(0, 2 ** 21, (1000, 3)).astype(np.uint32)
    # any point inside a cell gets that cell's key; the cell corner belongs to it
    frac = rng.random((1000, 3))
    pos_in = (cells + frac) / 2.0 ** 21
    pos_corner = cells / 2.0 ** 21
    kc = oracle.hilbert_cells(cells, 21)
    assert np.array_equal(oracle.hilbert_keys(pos_in), kc)
    assert np.array_equal(oracle.hilbert_keys(pos_corner), kc)
    assert int(kc.max()) < 2 ** 63


def test_position_keys_reject_out_of_range():
    with pytest.raises(ValueError):
        oracle.hilbert_keys(np.array([[0.5, 0.5, 1.0]]))
    with pytest.raises(ValueError):
        oracle.hilbert_keys(np.array([[np.nan, 0.5, 0.5]]))


def test_stable_order_matches_a_stable_library_sort():
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 50, 5000).astype(np.uint64)  # many ties
    perm = oracle.stable_order(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    # ties keep the input order
    for k in range(50):
        sel = perm[keys[perm] == k]
        assert np.all(np.diff(sel) > 0)
