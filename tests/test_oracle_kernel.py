"""Pins of the oracle's M4 cubic-spline kernel (support radius h).

The kernel is fixed by: normalisation (integral over the support is 1), its value at
the centre, vanishing value and slope at the support edge, continuity of value and
slope at q = 1/2, and the derivatives agreeing with finite differences of the value.
"""

import math

import numpy as np
import pytest
from scipy import integrate

import oracle


@pytest.mark.parametrize("h", [1.0, 0.013, 2.7e-4])
def test_normalisation(h):
    f = lambda r: 4.0 * math.pi * r * r * oracle.kernel(np.array([r]), h)[0][0]
    val = integrate.quad(f, 0.0, h / 2, epsabs=0, epsrel=1e-13)[0] + \
        integrate.quad(f, h / 2, h, epsabs=0, epsrel=1e-13)[0]
    assert abs(val - 1.0) < 1e-12


def test_special_values():
    h = 0.37
    w, dwdr, _ = oracle.kernel(np.array([0.0, h, 1.5 * h, 0.75 * h]), h)
    assert w[0] == pytest.approx(8.0 / (math.pi * h ** 3), rel=1e-15)
    assert w[1] == 0.0 and dwdr[1] == 0.0 and w[2] == 0.0
    assert dwdr[0] == 0.0
    # q = 3/4: 2 (1/4)^3 sigma
    assert w[3] == pytest.approx(8.0 / (math.pi * h ** 3) * 2.0 / 64.0, rel=1e-14)


def test_continuity_at_half():
    h = 1.0
    e = 1e-12
    w, dwdr, _ = oracle.kernel(np.array([0.5 - e, 0.5 + e]), h)
    assert abs(w[0] - w[1]) < 1e-10
    assert abs(dwdr[0] - dwdr[1]) < 1e-10


def test_derivatives_match_finite_differences():
    rng = np.random.default_rng(3)
    h = 0.05
    r = rng.uniform(0.001, 0.999, 200) * h
    d = 1e-7 * h
    w, dwdr, dwdh = oracle.kernel(r, h)
    fd_r = (oracle.kernel(r + d, h)[0] - oracle.kernel(r - d, h)[0]) / (2 * d)
    fd_h = (oracle.kernel(r, h + d)[0] - oracle.kernel(r, h - d)[0]) / (2 * d)
    scale = 8.0 / (math.pi * h ** 4)
    assert np.max(np.abs(fd_r - dwdr)) < 1e-6 * scale
    assert np.max(np.abs(fd_h - dwdh)) < 1e-6 * scale
