"""Pins of the oracle's velocity divergence and curl (density sets, gather at h_i).

On a uniform cubic lattice, for particles whose sphere does not reach the box edge, the
cubic symmetry makes the SPH gradient of a linear field v = A x exactly c A for one
scalar c: a rotation has zero divergence and curl 2c omega, an isotropic expansion zero
curl, and a symmetric traceless field neither; c is close to 1.  The tree and the brute
force sets agree.
"""

import numpy as np

import oracle
import sphgen


def _lattice_case(A, n_side=16):
    pos = sphgen.lattice(n_side)
    n = len(pos)
    m = np.full(n, 1.0 / n)
    h = np.full(n, 2.6 / n_side)                       # about 73 neighbours, off lattice shells
    vel = pos @ np.asarray(A).T
    rho = oracle.density(pos, m, h)["rho"]
    inner = np.flatnonzero(np.all((pos > h[0] + 1e-9) & (pos < 1 - h[0] - 1e-9), axis=1))
    div, curl = oracle.velocity_derivs(pos, vel, m, h, rho, targets=inner)
    return div, curl


def test_rotation_has_no_divergence():
    w = np.array([0.3, -0.2, 0.5])
    A = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])   # v = w x x
    div, curl = _lattice_case(A)
    assert np.max(np.abs(div)) < 1e-12
    c = curl / (2 * w)
    assert np.allclose(c, c[0, 0], rtol=1e-10) and abs(c[0, 0] - 1.0) < 0.05


def test_expansion_has_no_curl():
    div, curl = _lattice_case(0.7 * np.eye(3))
    assert np.max(np.abs(curl)) < 1e-12
    c = div / (3 * 0.7)
    assert np.allclose(c, c[0], rtol=1e-10) and abs(c[0] - 1.0) < 0.05


def test_symmetric_traceless_shear_has_neither():
    A = np.array([[0.2, 0.3, 0.0], [0.3, -0.1, 0.4], [0.0, 0.4, -0.1]])
    div, curl = _lattice_case(A)
    assert np.max(np.abs(div)) < 1e-12 and np.max(np.abs(curl)) < 1e-12


def test_tree_equals_brute_force():
    d = sphgen.make("clustered", 3000, config=13)
    h, dens = oracle.density_iterate(d["pos"], d["m"], np.full(3000, d["h0"]))
    a = oracle.velocity_derivs(d["pos"], d["vel"], d["m"], h, dens["rho"], use_tree=True)
    b = oracle.velocity_derivs(d["pos"], d["vel"], d["m"], h, dens["rho"], use_tree=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
