"""Parity of the backward (adjoint) path: sphgrp_backward and the autograd Function
against the FP64 oracle's hand-written adjoint (itself pinned to dual numbers and
finite differences on the CPU), and against central finite differences of the
oracle's loss.

L = sum_k w_k . a_k + sum_k s_k rho_k with seeded standard-normal w and s, h from the
exact constraint (4 pi / 3) h^3 rho = 64 m.  Tolerance: every gradient array within
1e-3 of the FP64 gradient in relative L2 norm (FP32 pair terms and sums, FP64
per-particle chain), and elementwise within 1e-3 of the array's largest magnitude.
"""

import functools

import numpy as np
import pytest

import oracle
import sphgen
from gpu_common import Gpu, dataset

pytestmark = pytest.mark.gpu

TOL = 1e-3


@functools.lru_cache(maxsize=None)
def _problem(kind, n, cfg):
    d = dataset(kind, n, cfg)
    m = d["m32"].astype(np.float64)
    h, out = oracle.density_iterate(d["pos"], m, np.full(n, d["h0"]))
    assert out["failed"] == 0
    he = oracle.h_exact(d["pos"], m, h)
    rng = np.random.default_rng(sphgen.SEED_BASE + 400 + cfg)
    w = rng.standard_normal((n, 3)).astype(np.float32)
    s = rng.standard_normal(n).astype(np.float32)
    return d, m, he, w, s


@functools.lru_cache(maxsize=None)
def _oracle_grad(kind, n, cfg):
    d, m, h, w, s = _problem(kind, n, cfg)
    return oracle.loss_grad(d["pos"], d["vel32"].astype(np.float64), m, d["u32"].astype(np.float64), h,
                            w.astype(np.float64), s.astype(np.float64))


def _gpu_grad(g, d, h, w, s, group_size, with_s=True):
    torch = g.torch
    n = g.n
    gx = torch.full((n, 3), np.nan, dtype=torch.float32, device=g.dev)
    gv = torch.full((n, 3), np.nan, dtype=torch.float32, device=g.dev)
    gm = torch.full((n,), np.nan, dtype=torch.float32, device=g.dev)
    g.ctx.backward(g.t(h, torch.float64), g.t(d["vel32"]), g.t(d["u32"]), g.t(w), g.t(s) if with_s else None,
                   group_size, gx, gv, gm)
    return gx.cpu().numpy(), gv.cpu().numpy(), gm.cpu().numpy()


def _compare(got, ref, what):
    got = np.asarray(got, np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    worst = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert np.all(np.isfinite(got)), what
    assert err <= TOL, f"{what}: relative L2 error {err:.3e}"
    assert worst <= TOL, f"{what}: largest error {worst:.3e} of the largest magnitude"
    return err, worst


@pytest.mark.parametrize("kind,n,cfg", [("uniform", 32768, 1), ("clustered", 24001, 4)])
@pytest.mark.parametrize("group_size", [1, 16, 64])
def test_backward_matches_oracle(cuda_device, kind, n, cfg, group_size):
    d, m, h, w, s = _problem(kind, n, cfg)
    _, ox, ov, om = _oracle_grad(kind, n, cfg)
    g = Gpu(d["pos"], d["m32"])
    gx, gv, gm = _gpu_grad(g, d, h, w, s, group_size)
    errs = [_compare(gx, ox, "dL/dx"), _compare(gv, ov, "dL/dv"), _compare(gm, om, "dL/dm")]
    print(kind, n, group_size, ["%.2e/%.2e" % e for e in errs], g.ctx.stats())


def test_backward_larger_clustered(cuda_device):
    d, m, h, w, s = _problem("clustered", 131072, 4)
    _, ox, ov, om = _oracle_grad("clustered", 131072, 4)
    g = Gpu(d["pos"], d["m32"])
    gx, gv, gm = _gpu_grad(g, d, h, w, s, 16)
    for got, ref, what in ((gx, ox, "dL/dx"), (gv, ov, "dL/dv"), (gm, om, "dL/dm")):
        print(what, "%.2e / %.2e" % _compare(got, ref, what))


def test_backward_clustered_2m(cuda_device):
    """The backward workload's size: 2^21 clustered particles, all elements."""
    n = 1 << 21
    d, m, h, w, s = _problem("clustered", n, 4)
    _, ox, ov, om = _oracle_grad("clustered", n, 4)
    g = Gpu(d["pos"], d["m32"])
    gx, gv, gm = _gpu_grad(g, d, h, w, s, 16)
    for got, ref, what in ((gx, ox, "dL/dx"), (gv, ov, "dL/dv"), (gm, om, "dL/dm")):
        print(what, "%.2e / %.2e" % _compare(got, ref, what))
    g.ctx.close()
    _oracle_grad.cache_clear()
    _problem.cache_clear()


def test_backward_without_density_weights(cuda_device):
    d, m, h, w, s = _problem("clustered", 24001, 4)
    ref = oracle.loss_grad(d["pos"], d["vel32"].astype(np.float64), m, d["u32"].astype(np.float64), h,
                           w.astype(np.float64), np.zeros(len(m)))
    g = Gpu(d["pos"], d["m32"])
    got = _gpu_grad(g, d, h, w, s, 16, with_s=False)
    for a, b, what in zip(got, ref[1:], ("dL/dx", "dL/dv", "dL/dm")):
        _compare(a, b, what)


def test_backward_central_differences(cuda_device):
    """GPU gradient against FP64 central differences (step 1e-6) of the oracle's loss,
    h re-solved from the exact constraint at every point, on 64 random coordinates."""
    kind, n, cfg = "clustered", 6000, 4
    d, m, h, w, s = _problem(kind, n, cfg)
    g = Gpu(d["pos"], d["m32"])
    gx, _, _ = _gpu_grad(g, d, h, w, s, 16)
    vel, u = d["vel32"].astype(np.float64), d["u32"].astype(np.float64)
    w64, s64 = w.astype(np.float64), s.astype(np.float64)
    scale = np.max(np.abs(gx))
    rng = np.random.default_rng(sphgen.SEED_BASE + 77)
    picks = [(int(rng.integers(0, n)), int(rng.integers(0, 3))) for _ in range(64)]
    bad = []
    for i, a in picks:
        vals = []
        for sgn in (1.0, -1.0):
            pos = d["pos"].copy()
            pos[i, a] += sgn * 1e-6
            hh = oracle.h_exact(pos, m, h)
            vals.append(oracle.loss_grad(pos, vel, m, u, hh, w64, s64)[0])
        fd = (vals[0] - vals[1]) / 2e-6
        if abs(gx[i, a] - fd) > TOL * (abs(fd) + 1e-2 * scale):
            bad.append((i, a, float(gx[i, a]), fd))
    assert not bad, bad


def test_autograd_function(cuda_device):
    import torch

    import paper_1810_09898_gb300 as sg

    d, m, h, w, s = _problem("clustered", 24001, 4)
    _, ox, ov, om = _oracle_grad("clustered", 24001, 4)
    n = len(m)
    dev = torch.device("cuda:0")
    ctx = sg.Context(n)
    pos = torch.tensor(d["pos"], device=dev, requires_grad=True)
    vel = torch.tensor(d["vel32"], device=dev, requires_grad=True)
    mass = torch.tensor(d["m32"], device=dev, requires_grad=True)
    acc, rho = sg.sph_forces(ctx, pos, vel, mass, torch.tensor(d["u32"], device=dev),
                             torch.tensor(h, device=dev), 16)
    loss = (torch.tensor(w, device=dev) * acc).sum() + (torch.tensor(s, device=dev) * rho).sum()
    loss.backward()
    assert pos.grad.dtype == torch.float64 and vel.grad.dtype == torch.float32
    _compare(pos.grad.cpu().numpy(), ox, "dL/dx")
    _compare(vel.grad.cpu().numpy(), ov, "dL/dv")
    _compare(mass.grad.cpu().numpy(), om, "dL/dm")
    # forward outputs are those of the forward entry points
    dens = oracle.density(d["pos"], m, h)
    assert np.max(np.abs(rho.detach().cpu().numpy() - dens["rho"]) / dens["rho"]) <= 1e-5
    ctx.close()


def test_backward_rejects_bad_calls(cuda_device):
    import torch

    import paper_1810_09898_gb300 as sg

    d, m, h, w, s = _problem("uniform", 32768, 1)
    ctx = sg.Context(1000)
    z = torch.zeros(3000, dtype=torch.float32, device="cuda:0")
    with pytest.raises(sg.SphgrpError, match="ESTATE"):
        ctx.backward(torch.ones(1000, dtype=torch.float64, device="cuda:0") * 0.1, z, z, z, None, 16, z)
    g = Gpu(d["pos"][:1000], d["m32"][:1000])
    hh = g.t(h[:1000], torch.float64)
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        g.ctx.backward(hh, z, z, z, None, 0, z)
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        g.ctx.backward(hh, z, z, z, None, 16)
    bad = hh.clone()
    bad[3] = 0.7
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        g.ctx.backward(bad, z, z, z, None, 16, z)
    ctx.close()


@pytest.mark.parametrize("kind,n,cfg", [("uniform", 32768, 1), ("clustered", 24001, 4)])
def test_density_only_backward(cuda_device, kind, n, cfg):
    """g_acc = NULL: the gradient of sum s . rho alone, without the hydro-adjoint loop
    (vel and u not passed), against the oracle's gradient of the same loss (w = 0)."""
    d, m, h, _, s = _problem(kind, n, cfg)
    _, ox, ov, om = oracle.loss_grad(d["pos"], d["vel32"].astype(np.float64), m, d["u32"].astype(np.float64), h,
                                     np.zeros((n, 3)), s.astype(np.float64))
    assert np.all(ov == 0.0)
    g = Gpu(d["pos"], d["m32"])
    torch = g.torch
    gx = torch.full((n, 3), np.nan, dtype=torch.float32, device=g.dev)
    gv = torch.full((n, 3), np.nan, dtype=torch.float32, device=g.dev)
    gm = torch.full((n,), np.nan, dtype=torch.float32, device=g.dev)
    g.ctx.backward(g.t(h, torch.float64), None, None, None, g.t(s), 16, gx, gv, gm)
    st = g.ctx.stats()
    _compare(gx.cpu().numpy(), ox, "dL/dx")
    _compare(gm.cpu().numpy(), om, "dL/dm")
    assert np.all(gv.cpu().numpy() == 0.0)
    assert st["search_launches"] == 2, st   # density sums and density adjoint only
    # the autograd Function takes the same path when the loss uses rho alone
    import paper_1810_09898_gb300 as sg

    pos = torch.tensor(d["pos"], device=g.dev, requires_grad=True)
    mm = torch.as_tensor(d["m32"], device=g.dev).clone().requires_grad_(True)
    _, rho = sg.sph_forces(g.ctx, pos, g.t(d["vel32"]), mm, g.t(d["u32"]), g.t(h, torch.float64), 16)
    (g.t(s) * rho).sum().backward()
    assert g.ctx.stats()["search_launches"] == 2
    _compare(pos.grad.cpu().numpy(), ox, "autograd dL/dx")
    _compare(mm.grad.cpu().numpy(), om, "autograd dL/dm")
    with pytest.raises(sg.SphgrpError, match="EINVAL"):
        g.ctx.backward(g.t(h, torch.float64), None, None, None, None, 16, gx, gv, gm)
