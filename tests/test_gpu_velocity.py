"""GPU parity of the velocity divergence and curl (grouped walk over the density sets)
against the FP64 oracle, through the C ABI.

Bar: rel-L2 <= 1e-4 for div v and for curl v (FP32 compensated sums against FP64, as
for the accelerations).  Inputs: the seeded synthetic sets of sphgen at the oracle's
converged h, uniform and clustered, all active and runs of actives.
"""

import numpy as np
import pytest

import oracle
from gpu_common import Gpu, active_runs, converged, dataset

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _run(G, active, h, rho32, vel32, g):
    torch = G.torch
    n = G.n
    divv = torch.zeros(n, dtype=torch.float32, device=G.dev)
    curl = torch.zeros((n, 3), dtype=torch.float32, device=G.dev)
    G.ctx.velocity_derivs(G.t(active, torch.int32), G.t(h, torch.float64), G.t(rho32), G.t(vel32), g, divv, curl)
    return divv.cpu().numpy(), curl.cpu().numpy()


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=[("uniform", 32768, 1), ("clustered", 24001, 2)], ids=["uniform", "clustered"])
def setup(cuda_device, request):
    dist, n, cfg = request.param
    d = dataset(dist, n, cfg)
    h, dens = converged(dist, n, cfg)
    rho32 = dens["rho"].astype(np.float32)
    G = Gpu(d["pos"], d["m32"])
    ref = oracle.velocity_derivs(d["pos"], d["vel32"].astype(np.float64), d["m32"].astype(np.float64), h,
                                 rho32.astype(np.float64))
    return d, h, rho32, G, ref


@pytest.mark.parametrize("g", [1, 16, 32, 128])
def test_velocity_derivs_all_active(setup, g):
    d, h, rho32, G, (rdiv, rcurl) = setup
    act = np.arange(G.n, dtype=np.int32)
    div, curl = _run(G, act, h, rho32, d["vel32"], g)
    assert _rel_l2(div, rdiv) <= TOL
    assert _rel_l2(curl, rcurl) <= TOL


def test_velocity_derivs_partial_active(setup):
    d, h, rho32, G, (rdiv, rcurl) = setup
    act = active_runs(G.n, 0.1, 11, G.perm.cpu().numpy())
    div, curl = _run(G, act, h, rho32, d["vel32"], 32)
    assert _rel_l2(div[act], rdiv[act]) <= TOL
    assert _rel_l2(curl[act], rcurl[act]) <= TOL
    inactive = np.setdiff1d(np.arange(G.n), act)
    assert np.all(div[inactive] == 0.0) and np.all(curl[inactive] == 0.0)


def test_velocity_derivs_rigid_rotation(cuda_device):
    """A lattice in rigid rotation about z: div v = 0 and curl v = (0, 0, 2 w) up to the
    kernel-sum discretisation, and the GPU matches the oracle on it."""
    k = 16
    g1 = (np.arange(k) + 0.5) / k
    pos = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    n = len(pos)
    m32 = np.full(n, 1.0 / n, np.float32)
    w = 0.7
    c = pos - 0.5
    vel32 = np.stack([-w * c[:, 1], w * c[:, 0], np.zeros(n)], -1).astype(np.float32)
    h = np.full(n, 2.2 / k)
    rho = oracle.density(pos, m32.astype(np.float64), h)["rho"]
    rho32 = rho.astype(np.float32)
    # interior particles only: the rotation field is not periodic across the box faces
    inner = np.flatnonzero(np.all(np.abs(c) < 0.5 - 2.5 / k, axis=1)).astype(np.int32)
    G = Gpu(pos, m32)
    div, curl = _run(G, inner, h, rho32, vel32, 16)
    rdiv, rcurl = oracle.velocity_derivs(pos, vel32.astype(np.float64), m32.astype(np.float64), h,
                                         rho32.astype(np.float64), targets=inner)
    assert np.max(np.abs(div[inner])) < 1e-4 * w
    assert np.allclose(curl[inner, 2], 2 * w, rtol=5e-3)   # lattice kernel-sum error ~1.6e-3
    assert _rel_l2(curl[inner], rcurl) <= TOL
    assert np.max(np.abs(div[inner] - rdiv)) < 1e-4 * w


def test_velocity_derivs_single_particle_and_empty(cuda_device):
    G = Gpu(np.array([[0.3, 0.6, 0.9]]), np.ones(1, np.float32))
    div, curl = _run(G, np.zeros(1, np.int32), np.array([0.1]), np.array([2.0], np.float32),
                     np.array([[1.0, 2.0, 3.0]], np.float32), 8)
    assert div[0] == 0.0 and np.all(curl[0] == 0.0)
    div, curl = _run(G, np.zeros(0, np.int32), np.array([0.1]), np.array([2.0], np.float32),
                     np.array([[1.0, 2.0, 3.0]], np.float32), 8)
    assert div[0] == 0.0


def test_velocity_derivs_rejects_bad_input(cuda_device):
    import paper_1810_09898_gb300 as sg

    G = Gpu(np.array([[0.3, 0.6, 0.9], [0.31, 0.6, 0.9]]), np.ones(2, np.float32))
    with pytest.raises(sg.SphgrpError):
        _run(G, np.zeros(1, np.int32), np.array([0.1, 0.1]), np.ones(2, np.float32), np.zeros((2, 3), np.float32), 0)
    with pytest.raises(sg.SphgrpError):
        _run(G, np.array([5], np.int32), np.array([0.1, 0.1]), np.ones(2, np.float32),
             np.zeros((2, 3), np.float32), 8)


# ---------------------------------------------------------------- fused density + derivatives

def _fused(G, active, h, vel32, g, iterate):
    torch = G.torch
    n = G.n
    f32 = dict(dtype=torch.float32, device=G.dev)
    hh = G.t(np.array(h, dtype=np.float64, copy=True), torch.float64)
    rho, drho, fg = (torch.zeros(n, **f32) for _ in range(3))
    nn = torch.zeros(n, dtype=torch.int32, device=G.dev)
    divv, curl = torch.zeros(n, **f32), torch.zeros((n, 3), **f32)
    G.ctx.density_derivs(G.t(active, torch.int32), hh, iterate, g, G.t(vel32), rho, drho, fg, nn, divv, curl)
    return {"h": hh.cpu().numpy(), "rho": rho.cpu().numpy(), "nngb": nn.cpu().numpy(), "div": divv.cpu().numpy(),
            "curl": curl.cpu().numpy()}


@pytest.mark.parametrize("iterate", [0, 1])
@pytest.mark.parametrize("g", [8, 16, 64])
def test_density_derivs_fused(setup, iterate, g):
    """div v and curl v summed inside the density loop: the density as sphgrp_density, the
    derivatives as the separate loop would give at the call's final h and rho."""
    d, h, rho32, G, _ = setup
    act = np.arange(G.n, dtype=np.int32)
    h0 = h * np.exp(0.05 * np.random.default_rng(5).standard_normal(G.n)) if iterate else h
    out = _fused(G, act, h0, d["vel32"], g, iterate)
    m = d["m32"].astype(np.float64)
    chk = oracle.density(d["pos"], m, out["h"])
    assert np.array_equal(out["nngb"], chk["nngb"])
    assert np.max(np.abs(out["rho"] / chk["rho"] - 1.0)) <= 1e-5
    rdiv, rcurl = oracle.velocity_derivs(d["pos"], d["vel32"].astype(np.float64), m, out["h"],
                                         out["rho"].astype(np.float64))
    assert _rel_l2(out["div"], rdiv) <= TOL
    assert _rel_l2(out["curl"], rcurl) <= TOL


def test_density_derivs_partial_active(setup):
    d, h, rho32, G, _ = setup
    act = active_runs(G.n, 0.2, 17, G.perm.cpu().numpy())
    out = _fused(G, act, h, d["vel32"], 16, 1)
    m = d["m32"].astype(np.float64)
    rdiv, rcurl = oracle.velocity_derivs(d["pos"], d["vel32"].astype(np.float64), m, out["h"],
                                         out["rho"].astype(np.float64), targets=act)
    assert _rel_l2(out["div"][act], rdiv) <= TOL
    assert _rel_l2(out["curl"][act], rcurl) <= TOL
    inactive = np.setdiff1d(np.arange(G.n), act)
    assert np.all(out["div"][inactive] == 0.0)


# ---------------------------------------------------------------- Balsara-limited hydro

@pytest.mark.parametrize("mode,g", [(0, 1), (1, 16), (1, 32)])
def test_hydro_balsara_matches_oracle(setup, mode, g):
    """The limited viscosity against the oracle's, both fed the same div v and curl v."""
    d, h, rho32, G, _ = setup
    torch = G.torch
    n = G.n
    act = np.arange(n, dtype=np.int32)
    f32 = oracle.density(d["pos"], d["m32"].astype(np.float64), h)["f"].astype(np.float32)
    div, curl = _run(G, act, h, rho32, d["vel32"], 16)
    acc = torch.zeros((n, 3), dtype=torch.float32, device=G.dev)
    dudt = torch.zeros(n, dtype=torch.float32, device=G.dev)
    nn = torch.zeros(n, dtype=torch.int32, device=G.dev)
    G.ctx.hydro_force(G.t(act, torch.int32), G.t(h, torch.float64), G.t(rho32), G.t(f32), G.t(d["vel32"]),
                      G.t(d["u32"]), mode, g, acc, dudt, nn, divv=G.t(div), curlv=G.t(curl))
    fb = oracle.balsara(div, curl, d["u32"].astype(np.float64), h)
    assert 0.0 <= fb.min() and fb.max() < 1.0 and fb.std() > 0.05   # the limiter does vary
    ref = oracle.hydro(d["pos"], d["vel32"].astype(np.float64), d["m32"].astype(np.float64), h,
                       rho32.astype(np.float64), f32.astype(np.float64), d["u32"].astype(np.float64), fbal=fb)
    assert np.array_equal(nn.cpu().numpy(), ref["nngb"])
    assert _rel_l2(acc.cpu().numpy(), ref["acc"]) <= TOL
    assert _rel_l2(dudt.cpu().numpy(), ref["dudt"]) <= TOL
    # and it differs from the plain viscosity
    plain = oracle.hydro(d["pos"], d["vel32"].astype(np.float64), d["m32"].astype(np.float64), h,
                         rho32.astype(np.float64), f32.astype(np.float64), d["u32"].astype(np.float64))
    assert _rel_l2(plain["dudt"], ref["dudt"]) > 1e-2
