"""Pins of the oracle's SPH hydro accelerations and du/dt.

* total momentum and total energy are conserved to rounding (the pair terms are
  antisymmetric and the neighbour relation max(h_i, h_j) is symmetric);
* a uniform lattice with uniform u and no motion feels no force;
* two particles at rest repel each other along their separation, and an approaching
  pair is heated by the viscosity (du/dt > 0) and decelerated;
* tree-pruned and brute-force evaluations agree.
"""

import numpy as np
import pytest

import oracle
import sphgen


def _state(dist, n, seed=9):
    d = sphgen.make(dist, n, config=seed)
    h, dens = oracle.density_iterate(d["pos"], d["m"], np.full(n, d["h0"]))
    return d, h, dens


@pytest.mark.parametrize("dist", ["uniform", "clustered"])
def test_momentum_and_energy_conservation(dist):
    d, h, dens = _state(dist, 5000)
    out = oracle.hydro(d["pos"], d["vel"], d["m"], h, dens["rho"], dens["f"], d["u"])
    ma = d["m"][:, None] * out["acc"]
    assert np.max(np.abs(ma.sum(0))) < 1e-12 * np.abs(ma).sum()
    e = d["m"] * ((d["vel"] * out["acc"]).sum(1) + out["dudt"])
    assert abs(e.sum()) < 1e-12 * np.abs(e).sum()


def test_lattice_at_rest_feels_no_force():
    pos = sphgen.lattice(12)
    n = len(pos)
    m = np.full(n, 1.0 / n)
    h = np.full(n, 2.2 / 12)
    dens = oracle.density(pos, m, h)
    out = oracle.hydro(pos, np.zeros((n, 3)), m, h, dens["rho"], dens["f"], np.ones(n))
    # scale: one neighbour's pressure term
    w, dw, _ = oracle.kernel(np.array([1.0 / 12]), h[0])
    scale = m[0] * abs(dw[0]) * dens["f"][0] * (2.0 / 3.0) / dens["rho"][0]
    assert np.max(np.abs(out["acc"])) < 1e-10 * scale
    assert np.max(np.abs(out["dudt"])) < 1e-10 * scale


def test_pair_at_rest_repels_and_approaching_pair_heats():
    pos = np.array([[0.5, 0.5, 0.5], [0.53125, 0.5, 0.5]])
    m = np.array([1.0, 2.0])
    h = np.array([0.05, 0.04])
    rho = np.array([2.0, 3.0])
    f = np.array([0.9, 0.8])
    u = np.array([1.5, 0.7])
    rest = oracle.hydro(pos, np.zeros((2, 3)), m, h, rho, f, u)
    assert rest["acc"][0, 0] < 0 < rest["acc"][1, 0]
    assert np.allclose(rest["acc"][:, 1:], 0.0)
    # pressure-only closed form along x: a_0 = m_1 (A_0 W'(r,h_0) + A_1 W'(r,h_1)),
    # A_k = f_k P_k / rho_k^2, P_k = (gamma - 1) rho_k u_k, W' < 0
    r = 0.03125
    dw0 = oracle.kernel(np.array([r]), h[0])[1][0]
    dw1 = oracle.kernel(np.array([r]), h[1])[1][0]
    A = f * (2.0 / 3.0) * rho * u / rho ** 2
    assert rest["acc"][0, 0] == pytest.approx(m[1] * (A[0] * dw0 + A[1] * dw1), rel=1e-14)
    assert rest["acc"][1, 0] == pytest.approx(-m[0] * (A[1] * dw1 + A[0] * dw0), rel=1e-14)
    assert np.allclose(rest["dudt"], 0.0)
    vel = np.array([[0.3, 0.0, 0.0], [-0.3, 0.0, 0.0]])
    mov = oracle.hydro(pos, vel, m, h, rho, f, u)
    assert np.all(mov["dudt"] > 0.0)
    # viscosity adds deceleration on top of the pressure push
    assert mov["acc"][0, 0] < rest["acc"][0, 0]
    # receding pair: no viscosity, pressure work cools particle 0
    away = oracle.hydro(pos, -vel, m, h, rho, f, u)
    assert np.allclose(away["acc"], rest["acc"], rtol=1e-14)
    assert away["dudt"][0] == pytest.approx(m[1] * A[0] * (-0.6) * (-dw0), rel=1e-14)


def test_tree_equals_brute_force():
    d, h, dens = _state("clustered", 2500)
    a = oracle.hydro(d["pos"], d["vel"], d["m"], h, dens["rho"], dens["f"], d["u"], use_tree=False)
    b = oracle.hydro(d["pos"], d["vel"], d["m"], h, dens["rho"], dens["f"], d["u"], use_tree=True)
    assert np.array_equal(a["nngb"], b["nngb"])
    assert np.allclose(a["acc"], b["acc"], rtol=1e-13, atol=0)
