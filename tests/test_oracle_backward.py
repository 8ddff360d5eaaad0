"""Pins of the oracle's backward pass: L = sum_i w_i . a_i + sum_i s_i rho_i and its
gradient with respect to positions, velocities and masses (neighbour sets fixed, h from
the exact constraint (4 pi / 3) h^3 rho = N_ngb m).

* the hand-written adjoint equals forward-mode dual numbers through the same loss
  (exact to rounding) on small sets;
* it agrees with central finite differences of the loss (h re-solved at every point);
* the loss value equals sum w.a + sum s rho from the forward oracle functions;
* translation and Galilean invariance: the gradients with respect to all positions and
  to all velocities each sum to zero.
"""

import numpy as np
import pytest

import oracle
import sphgen


def _state(kind, n, cfg=11, seed=5):
    d = sphgen.make(kind, n, config=cfg)
    h, _ = oracle.density_iterate(d["pos"], d["m"], np.full(n, d["h0"]))
    he = oracle.h_exact(d["pos"], d["m"], h)
    rng = np.random.default_rng(seed)
    return d, he, rng.standard_normal((n, 3)), rng.standard_normal(n)


@pytest.mark.parametrize("kind,n", [("uniform", 96), ("clustered", 128)])
def test_adjoint_equals_dual_numbers(kind, n):
    d, h, w, s = _state(kind, n)
    _, gx, gv, gm = oracle.loss_grad(d["pos"], d["vel"], d["m"], d["u"], h, w, s)
    dx, dv, dm = oracle.grad_dual(d["pos"], d["vel"], d["m"], d["u"], h, w, s)
    for a, b in ((gx, dx), (gv, dv), (gm, dm)):
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_exact_constraint_holds():
    d, h, _, _ = _state("clustered", 800)
    rho = oracle.density(d["pos"], d["m"], h)["rho"]
    g = 4.0 * np.pi / 3.0 * h ** 3 * rho / d["m"] - 64.0
    assert np.max(np.abs(g)) < 1e-9


def test_loss_value_matches_forward_functions():
    d, h, w, s = _state("clustered", 600)
    L, _, _, _ = oracle.loss_grad(d["pos"], d["vel"], d["m"], d["u"], h, w, s)
    dens = oracle.density(d["pos"], d["m"], h)
    hy = oracle.hydro(d["pos"], d["vel"], d["m"], h, dens["rho"], dens["f"], d["u"])
    ref = float(np.sum(w * hy["acc"]) + np.sum(s * dens["rho"]))
    assert L == pytest.approx(ref, rel=1e-12)


def test_translation_and_galilean_invariance():
    d, h, w, s = _state("clustered", 1500)
    _, gx, gv, _ = oracle.loss_grad(d["pos"], d["vel"], d["m"], d["u"], h, w, s)
    assert np.max(np.abs(gx.sum(0))) < 1e-10 * np.abs(gx).sum()
    assert np.max(np.abs(gv.sum(0))) < 1e-10 * np.abs(gv).sum()


def _loss_at(d, pos, vel, m, h_start, w, s):
    h = oracle.h_exact(pos, m, h_start)
    return oracle.loss_grad(pos, vel, m, d["u"], h, w, s)[0]


def test_central_finite_differences():
    d, h, w, s = _state("uniform", 1200, cfg=12)
    _, gx, gv, gm = oracle.loss_grad(d["pos"], d["vel"], d["m"], d["u"], h, w, s)
    rng = np.random.default_rng(8)
    for _ in range(6):
        i, a = int(rng.integers(0, 1200)), int(rng.integers(0, 3))
        for kind, g in (("x", gx), ("v", gv)):
            step = 1e-6 if kind == "x" else 1e-5
            vals = []
            for sgn in (1, -1):
                pos, vel = d["pos"].copy(), d["vel"].copy()
                (pos if kind == "x" else vel)[i, a] += sgn * step
                vals.append(_loss_at(d, pos, vel, d["m"], h, w, s))
            fd = (vals[0] - vals[1]) / (2 * step)
            assert fd == pytest.approx(g[i, a], rel=2e-4, abs=1e-6 * np.abs(g).max())
    i = int(rng.integers(0, 1200))
    step = 1e-6 * d["m"][i]
    vals = []
    for sgn in (1, -1):
        m = d["m"].copy()
        m[i] += sgn * step
        vals.append(_loss_at(d, d["pos"], d["vel"], m, h, w, s))
    fd = (vals[0] - vals[1]) / (2 * step)
    assert fd == pytest.approx(gm[i], rel=2e-4, abs=1e-6 * np.abs(gm).max())
