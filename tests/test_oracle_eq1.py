"""Eq. 1 (Sec. 2.2) against the oracle's neighbour counting.

In the approximation of uniform density and one h, the superset of a group of radius
R = f h (the sphere of radius R + h) holds (1 + f)^3 times the neighbours of one
particle; the paper prints the value for f = 0.5 (tests/golden/eq1_superset_worked_value.txt).
On a uniform random set at the uniform-density h, the oracle's counts within (1 + f) h
and within h (the particle itself excluded) must stand in that ratio, and the count
within h must be the N_ngb of the Sec. 2.2 relation N_ngb = 4 pi n h^3 / 3.
"""

import os

import numpy as np

import oracle
import sphgen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "eq1_superset_worked_value.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_superset_ratio_matches_the_worked_value():
    g = _golden()
    f = g["f"]
    n = 32768
    d = sphgen.make("uniform", n, config=1)
    h = np.full(n, (3.0 * 64.0 / (4.0 * np.pi * n)) ** (1.0 / 3.0))
    sample = np.sort(np.random.default_rng(5).choice(n, 2000, replace=False)).astype(np.int32)
    off_h, _ = oracle.ngb_sets(d["pos"], h, targets=sample)
    off_r, _ = oracle.ngb_sets(d["pos"], (1.0 + f) * h, targets=sample)
    within_h = np.diff(off_h) - 1
    within_r = np.diff(off_r) - 1
    # N_ngb = 4 pi n h^3 / 3 with n = (N - 1) other particles in the unit box
    assert abs(within_h.mean() / (64.0 * (n - 1) / n) - 1.0) < 0.01
    assert abs(within_r.mean() / within_h.mean() / g["ncand_over_nngb"] - 1.0) < 0.01


def test_grouped_supersets_are_at_least_the_predicted_sphere():
    """The oracle's grouped walk returns whole leaves, and curve-consecutive groups are
    elongated, so its superset per walk is at least Eq. 1's sphere for the matching f
    (g = N_ngb f^3)."""
    n = 32768
    d = sphgen.make("uniform", n, config=1)
    h = np.full(n, (3.0 * 64.0 / (4.0 * np.pi * n)) ** (1.0 / 3.0))
    m = d["m"].astype(np.float64)
    for g in (8, 27):
        f = (g / 64.0) ** (1.0 / 3.0)
        r = oracle.density_grouped(d["pos"], m, h, g)
        assert r["candidates"] / r["walks"] >= 64.0 * (1.0 + f) ** 3
