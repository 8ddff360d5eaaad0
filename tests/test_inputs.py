"""The seeded input recipes (sphgen): the clustered set's structure, the active runs and
the batched boxes follow the stated recipe, and every call is reproducible."""

import numpy as np

import sphgen


def test_clustered_recipe():
    d = sphgen.make("clustered", 20000, config=2)
    pos = d["pos"]
    assert pos.shape == (20000, 3) and np.all((pos >= 0) & (pos < 1))
    again = sphgen.make("clustered", 20000, config=2)
    assert np.array_equal(pos, again["pos"])
    assert np.allclose(d["m"], 1.0 / 20000)
    # half the particles sit in Plummer spheres: the distribution is far from uniform
    counts = np.histogram(pos[:, 0], bins=64, range=(0, 1))[0]
    assert counts.max() > 3 * counts.mean()
    assert np.isclose(d["h0"], (3 * 64 / (4 * np.pi * 20000)) ** (1 / 3))


def test_active_runs_fraction():
    rng = np.random.default_rng(3)
    mask = sphgen.active_rank_mask(100000, 0.2, 32.0, rng)
    assert mask.sum() == 20000
    # runs along the order: far fewer run starts than actives
    starts = np.count_nonzero(mask[1:] & ~mask[:-1]) + int(mask[0])
    assert starts < 20000 / 8


def test_batch_recipe():
    b = sphgen.batch(12, 2000, 50000, config=41)
    off = b["box_off"]
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == len(b["pos"]) and np.all(sizes >= 2000) and np.all(sizes <= 50000)
    assert set(np.unique(b["box_class"])) <= {0, 1}
    assert np.array_equal(b["box_class"], (b["kinds"] == "clustered").astype(np.int32))
    for k in range(12):
        s = slice(off[k], off[k + 1])
        assert b["active"][s].any()
        assert np.allclose(b["m"][s], 1.0 / sizes[k])
        assert np.allclose(b["h0"][s], (3 * 64 / (4 * np.pi * sizes[k])) ** (1 / 3))
    assert np.all((b["fracs"] >= 0.01) & (b["fracs"] <= 1.0))
    again = sphgen.batch(12, 2000, 50000, config=41)
    assert np.array_equal(again["pos"], b["pos"]) and np.array_equal(again["active"], b["active"])
