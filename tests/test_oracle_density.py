"""Pins of the oracle's SPH density and smoothing-length iteration.

* a uniform cubic lattice has the same density at every particle, equal to the
  lattice sum m * sum_{|d| < h} W(|d|, h) over integer offsets (enumerated here);
* dRho/dh agrees with finite differences of rho(h);
* the converged smoothing lengths satisfy |4 pi rho h^3 / (3 m) - N_ngb| <= dN
  (the relation used to derive Eq. 1), re-evaluated independently at the final h.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
import sphgen


def _lattice_sum(n_side, h):
    k = int(math.ceil(h * n_side)) + 1
    offs = np.array(list(itertools.product(range(-k, k + 1), repeat=3)), dtype=np.float64)
    r = np.sqrt((offs ** 2).sum(1)) / n_side
    r = r[r < h]
    w = oracle.kernel(r, h)[0]
    return np.sort(w).sum() / n_side ** 3, len(r)


@pytest.mark.parametrize("n_side,h_cells", [(16, 2.3), (12, 1.7), (10, 3.1)])
def test_lattice_density_closed_form(n_side, h_cells):
    pos = sphgen.lattice(n_side)
    n = len(pos)
    h = np.full(n, h_cells / n_side)
    m = np.full(n, 1.0 / n)
    out = oracle.density(pos, m, h)
    ref, count = _lattice_sum(n_side, h[0])
    assert np.all(out["nngb"] == count)
    assert np.max(np.abs(out["rho"] / ref - 1.0)) < 1e-13


def test_drho_dh_matches_finite_differences():
    d = sphgen.make("clustered", 4000, config=9, with_hydro=False)
    h = np.full(4000, d["h0"])
    t = np.arange(0, 4000, 37, dtype=np.int32)
    out = oracle.density(d["pos"], d["m"], h, targets=t)
    eps = 1e-6 * d["h0"]
    up = oracle.density(d["pos"], d["m"], h + eps, targets=t)["rho"]
    dn = oracle.density(d["pos"], d["m"], h - eps, targets=t)["rho"]
    fd = (up - dn) / (2 * eps)
    scale = np.abs(out["rho"]) / d["h0"]
    assert np.max(np.abs(fd - out["drhodh"]) / scale) < 1e-5


def test_two_particle_density():
    pos = np.array([[0.25, 0.25, 0.25], [0.25, 0.25, 0.28125]])  # exact separation 1/32
    m = np.array([1.0, 3.0])
    h = np.array([0.05, 0.02])
    out = oracle.density(pos, m, h)
    w0 = oracle.kernel(np.array([0.0]), 0.05)[0][0]
    w1 = oracle.kernel(np.array([1.0 / 32]), 0.05)[0][0]
    assert out["rho"][0] == pytest.approx(1.0 * w0 + 3.0 * w1, rel=1e-15)
    assert list(out["nngb"]) == [2, 1]


@pytest.mark.parametrize("dist", ["uniform", "clustered"])
def test_iteration_converges_to_band(dist):
    d = sphgen.make(dist, 6000, config=9, with_hydro=False)
    h0 = np.full(6000, d["h0"])
    h, out = oracle.density_iterate(d["pos"], d["m"], h0)
    assert out["failed"] == 0
    re = oracle.density(d["pos"], d["m"], h)
    neff = 4.0 * math.pi / 3.0 * h ** 3 * re["rho"] / d["m"]
    assert np.all(np.abs(neff - 64.0) <= 2.0)
    assert np.array_equal(re["rho"], out["rho"])
