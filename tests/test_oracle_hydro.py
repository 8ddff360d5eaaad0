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


# ----------------------------------------------------------------------------------------
# Monaghan viscosity, pinned by hand-evaluated closed forms of one approaching pair.
#
# Particles 0 and 1 on the x axis at dyadic positions, r = x_1 - x_0 = 1/32, with
# h_0 = 1/16 (q = 1/2) and h_1 = 1/8 (q = 1/4).  The M4 shape derivative is written out
# here from its polynomial, not taken from the oracle: dw/dq = -12 q + 18 q^2 for
# q <= 1/2, so dw/dq(1/2) = -3/2 and dw/dq(1/4) = -15/8, and dW/dr = 8/(pi h^4) dw/dq.
# With r_01 = x_0 - x_1 = (-r, 0, 0) every kernel gradient lies on x:
#   grad_0 W(h) = (-W'(r, h), 0, 0),   grad_1 W(h) = (+W'(r, h), 0, 0).
# The pair means are h_bar = (h_0 + h_1)/2, c_bar = (c_0 + c_1)/2, rho_bar =
# (rho_0 + rho_1)/2, and for v_01 . r_01 < 0
#   mu = h_bar v_01.r_01 / (r^2 + eps h_bar^2),  Pi = (-alpha c_bar mu + beta mu^2) / rho_bar.
# Then (Sec. 1.1 hydro loop, in the energy-conserving grad-h form with Monaghan viscosity)
#   a_0x = m_1 [A_0 W'_0 + A_1 W'_1 + Pi (W'_0 + W'_1)/2]
#   a_1x = -m_0 [A_1 W'_1 + A_0 W'_0 + Pi (W'_0 + W'_1)/2]
#   du_0 = m_1 [A_0 v_01 . grad_0 W(h_0) + Pi/2 v_01 . grad_0 W_bar]
#        = m_1 [-2 v A_0 W'_0 - Pi v (W'_0 + W'_1)/2]
#   du_1 = m_0 [-2 v A_1 W'_1 - Pi v (W'_0 + W'_1)/2]
# for v_0 = (v, w, 0), v_1 = (-v, 0, 0) (the transverse w must not enter).  The masses,
# densities, energies and h differ between the two particles, so a missing 1/rho_bar,
# h_bar or c_bar taken from one side or as a maximum, a wrong eps placement or a lost
# 1/2 in du/dt each change one of the values below.
# ----------------------------------------------------------------------------------------

_GAMMA = 5.0 / 3.0
_PAIR = {"x0": 0.5, "r": 1.0 / 32.0, "h": (1.0 / 16.0, 1.0 / 8.0), "m": (1.0, 2.0), "rho": (2.0, 4.0),
         "f": (0.75, 0.875), "u": (1.5, 0.5), "v": 0.25, "w": 0.375}


def _pair_closed_form(alpha, beta, eps):
    P = _PAIR
    r = P["r"]
    h0, h1 = P["h"]
    m0, m1 = P["m"]
    rho0, rho1 = P["rho"]
    f0, f1 = P["f"]
    u0, u1 = P["u"]
    v = P["v"]
    dW0 = 8.0 / (np.pi * h0 ** 4) * (-1.5)      # q = 1/2
    dW1 = 8.0 / (np.pi * h1 ** 4) * (-1.875)    # q = 1/4
    pr0, pr1 = (_GAMMA - 1.0) * rho0 * u0, (_GAMMA - 1.0) * rho1 * u1
    c0, c1 = np.sqrt(_GAMMA * pr0 / rho0), np.sqrt(_GAMMA * pr1 / rho1)
    A0, A1 = f0 * pr0 / rho0 ** 2, f1 * pr1 / rho1 ** 2
    vr = (2.0 * v) * (-r)                        # v_01 . r_01
    hbar = 0.5 * (h0 + h1)
    mu = hbar * vr / (r * r + eps * hbar * hbar)
    cbar = 0.5 * (c0 + c1)
    rhobar = 0.5 * (rho0 + rho1)
    Pi = (-alpha * cbar * mu + beta * mu * mu) / rhobar
    gbar = 0.5 * (dW0 + dW1)
    a0 = m1 * (A0 * dW0 + A1 * dW1 + Pi * gbar)
    a1 = -m0 * (A1 * dW1 + A0 * dW0 + Pi * gbar)
    du0 = m1 * (-2.0 * v * A0 * dW0 - Pi * v * gbar)
    du1 = m0 * (-2.0 * v * A1 * dW1 - Pi * v * gbar)
    return {"a0": a0, "a1": a1, "du0": du0, "du1": du1, "Pi": Pi, "gbar": gbar, "mu": mu}


def _pair_oracle(alpha, beta, eps, moving=True):
    P = _PAIR
    pos = np.array([[P["x0"], 0.5, 0.5], [P["x0"] + P["r"], 0.5, 0.5]])
    vel = np.array([[P["v"], P["w"], 0.0], [-P["v"], 0.0, 0.0]]) if moving else np.zeros((2, 3))
    return oracle.hydro(pos, vel, np.array(P["m"]), np.array(P["h"]), np.array(P["rho"]), np.array(P["f"]),
                        np.array(P["u"]), gamma=_GAMMA, alpha=alpha, beta=beta, eps=eps)


@pytest.mark.parametrize("alpha,beta,eps", [(1.0, 2.0, 0.01),    # the benchmark's constants
                                            (1.0, 0.0, 0.01),    # linear term alone
                                            (0.0, 2.0, 0.01),    # quadratic term alone
                                            (0.5, 3.0, 0.25)])   # eps large enough to dominate
def test_viscosity_two_particle_closed_form(alpha, beta, eps):
    ref = _pair_closed_form(alpha, beta, eps)
    out = _pair_oracle(alpha, beta, eps)
    assert ref["Pi"] > 0.0 and ref["mu"] < 0.0
    assert out["acc"][0, 0] == pytest.approx(ref["a0"], rel=1e-14)
    assert out["acc"][1, 0] == pytest.approx(ref["a1"], rel=1e-14)
    assert np.all(out["acc"][:, 1:] == 0.0)
    assert out["dudt"][0] == pytest.approx(ref["du0"], rel=1e-14)
    assert out["dudt"][1] == pytest.approx(ref["du1"], rel=1e-14)
    # the viscous part alone: moving minus the same pair at rest is m_j Pi W_bar' on x
    rest = _pair_oracle(alpha, beta, eps, moving=False)
    visc0 = out["acc"][0, 0] - rest["acc"][0, 0]
    assert visc0 == pytest.approx(_PAIR["m"][1] * ref["Pi"] * ref["gbar"], rel=1e-12)


def test_viscosity_terms_separate():
    # Pi is linear in alpha at beta = 0, quadratic-only at alpha = 0, and the sum at both
    lin = _pair_closed_form(1.0, 0.0, 0.01)["Pi"]
    quad = _pair_closed_form(0.0, 1.0, 0.01)["Pi"]
    both = _pair_oracle(1.0, 1.0, 0.01)["acc"][0, 0] - _pair_oracle(1.0, 1.0, 0.01, moving=False)["acc"][0, 0]
    gbar = _pair_closed_form(1.0, 1.0, 0.01)["gbar"]
    assert both == pytest.approx(_PAIR["m"][1] * (lin + quad) * gbar, rel=1e-12)
    # a plausible slip changes the answer: h_bar as the max, c_bar from one side, no 1/rho_bar
    ref = _pair_closed_form(1.0, 2.0, 0.01)
    out = _pair_oracle(1.0, 2.0, 0.01)
    P = _PAIR
    for slip in ("hmax", "c0", "norho"):
        h0, h1 = P["h"]
        hb = max(h0, h1) if slip == "hmax" else 0.5 * (h0 + h1)
        vr = 2.0 * P["v"] * -P["r"]
        mu = hb * vr / (P["r"] ** 2 + 0.01 * hb * hb)
        c = [np.sqrt(_GAMMA * (_GAMMA - 1.0) * u) for u in P["u"]]
        cb = c[0] if slip == "c0" else 0.5 * (c[0] + c[1])
        rb = 1.0 if slip == "norho" else 0.5 * sum(P["rho"])
        wrong = (-cb * mu + 2.0 * mu * mu) / rb
        assert abs(wrong / ref["Pi"] - 1.0) > 1e-3
        assert abs(out["acc"][0, 0] - (ref["a0"] + P["m"][1] * (wrong - ref["Pi"]) * ref["gbar"])) > \
            1e-6 * abs(ref["a0"])


def test_tree_equals_brute_force():
    d, h, dens = _state("clustered", 2500)
    a = oracle.hydro(d["pos"], d["vel"], d["m"], h, dens["rho"], dens["f"], d["u"], use_tree=False)
    b = oracle.hydro(d["pos"], d["vel"], d["m"], h, dens["rho"], dens["f"], d["u"], use_tree=True)
    assert np.array_equal(a["nngb"], b["nngb"])
    assert np.allclose(a["acc"], b["acc"], rtol=1e-13, atol=0)


# ----------------------------------------------------------------------------------------
# Balsara's limiter: Pi_ij is scaled by the pair mean (f_i + f_j) / 2 of
# f = |div v| / (|div v| + |curl v| + 1e-4 c / h).
# ----------------------------------------------------------------------------------------

def test_limited_viscosity_two_particle_closed_form():
    fb = np.array([0.25, 0.75])     # the pair mean is 1/2, neither value alone
    ref = _pair_closed_form(1.0, 2.0, 0.01)
    P = _PAIR
    pos = np.array([[P["x0"], 0.5, 0.5], [P["x0"] + P["r"], 0.5, 0.5]])
    vel = np.array([[P["v"], P["w"], 0.0], [-P["v"], 0.0, 0.0]])
    args = (pos, vel, np.array(P["m"]), np.array(P["h"]), np.array(P["rho"]), np.array(P["f"]), np.array(P["u"]))
    out = oracle.hydro(*args, gamma=_GAMMA, fbal=fb)
    rest = _pair_oracle(1.0, 2.0, 0.01, moving=False)
    half = 0.5 * ref["Pi"]
    assert out["acc"][0, 0] == pytest.approx(rest["acc"][0, 0] + P["m"][1] * half * ref["gbar"], rel=1e-13)
    # du_0 = m_1 [-2 v A_0 W'_0 - (Pi / 2) v W_bar']: the plain value with half the viscous term
    assert out["dudt"][0] == pytest.approx(ref["du0"] + P["m"][1] * half * P["v"] * ref["gbar"], rel=1e-13)
    assert out["dudt"][1] == pytest.approx(ref["du1"] + P["m"][0] * half * P["v"] * ref["gbar"], rel=1e-13)
    # limiter 1 everywhere is the plain viscosity, 0 everywhere removes it
    one = oracle.hydro(*args, gamma=_GAMMA, fbal=np.ones(2))
    plain = oracle.hydro(*args, gamma=_GAMMA)
    assert np.array_equal(one["acc"], plain["acc"]) and np.array_equal(one["dudt"], plain["dudt"])
    zero = oracle.hydro(*args, gamma=_GAMMA, fbal=np.zeros(2))
    assert np.allclose(zero["acc"], rest["acc"], rtol=1e-14, atol=0)


def _lattice_flow(A, n_side=12):
    pos = sphgen.lattice(n_side)
    n = len(pos)
    m = np.full(n, 1.0 / n)
    h = np.full(n, 2.2 / n_side)
    dens = oracle.density(pos, m, h)
    vel = (pos - 0.5) @ np.asarray(A).T
    u = np.ones(n)
    inner = np.flatnonzero(np.all((pos > 2 * h[0] + 1e-9) & (pos < 1 - 2 * h[0] - 1e-9), axis=1))
    divv, curl = oracle.velocity_derivs(pos, vel, m, h, dens["rho"])
    fb = oracle.balsara(divv, curl, u, h)
    args = (pos, vel, m, h, dens["rho"], dens["f"], u)
    return args, fb, inner


def test_limiter_switches_off_viscosity_in_pure_shear():
    # v_x = S y: no divergence on the lattice (symmetry), curl -S z: the limiter is 0
    args, fb, inner = _lattice_flow([[0.0, 0.4, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert np.max(fb[inner]) < 1e-12
    lim = oracle.hydro(*args, targets=inner, fbal=fb)
    plain = oracle.hydro(*args, targets=inner)
    scale = np.max(np.abs(plain["dudt"]))
    assert scale > 0.0                                  # the plain viscosity heats the shear
    assert np.max(np.abs(lim["dudt"])) < 1e-10 * scale  # the limited one does not


def test_limiter_keeps_viscosity_in_pure_compression():
    # v = -a (x - c): no curl, the limiter is the same value close to 1 for the inner
    # particles, and their viscous part (plain minus inviscid) scales by exactly it
    args, fb, inner = _lattice_flow(-0.6 * np.eye(3))
    f0 = fb[inner]
    assert np.allclose(f0, f0[0], rtol=1e-12) and 0.99 < f0[0] < 1.0
    far = np.flatnonzero(np.all((args[0] > 3 * args[3][0] + 1e-9) & (args[0] < 1 - 3 * args[3][0] - 1e-9), axis=1))
    lim = oracle.hydro(*args, targets=far, fbal=fb)
    plain = oracle.hydro(*args, targets=far)
    inv = oracle.hydro(*args, targets=far, alpha=0.0, beta=0.0)
    assert np.allclose(lim["dudt"] - inv["dudt"], f0[0] * (plain["dudt"] - inv["dudt"]), rtol=1e-11, atol=0)
