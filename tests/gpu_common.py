"""Shared helpers of the GPU parity tests: datasets, oracle results (cached per
session) and the calls through the C ABI binding."""

from __future__ import annotations

import functools

import numpy as np

import oracle
import sphgen


# The GPU accepts a smoothing length when its own FP32 density gives |N_eff - 64| <= 2.
# The oracle re-evaluates N_eff = 4 pi h^3 rho / (3 m) at that h in FP64; the two rho
# differ by at most the density tolerance (rel 1e-5), so a particle accepted right at the
# edge of the band can sit up to (64 + 2) * 1e-5 = 6.6e-4 outside it by the oracle's count.
RHO_TOL = 1e-5
NEFF_TOL = 2.0 + (64.0 + 2.0) * RHO_TOL


@functools.lru_cache(maxsize=None)
def dataset(kind: str, n: int, config: int = 1):
    d = sphgen.make(kind, n, config=config)
    d["m32"] = d["m"].astype(np.float32)
    d["vel32"] = d["vel"].astype(np.float32)
    d["u32"] = d["u"].astype(np.float32)
    return d


@functools.lru_cache(maxsize=None)
def converged(kind: str, n: int, config: int = 1):
    """Oracle smoothing lengths iterated from h0, and the density at them."""
    d = dataset(kind, n, config)
    h, out = oracle.density_iterate(d["pos"], d["m32"].astype(np.float64), np.full(n, d["h0"]))
    assert out["failed"] == 0
    return h, out


def active_runs(n, frac, seed, perm):
    """Original indices of actives marked as runs along the key order given by perm."""
    rng = np.random.default_rng(seed)
    mask = sphgen.active_rank_mask(n, frac, 32.0, rng)
    return np.sort(perm[np.flatnonzero(mask)]).astype(np.int32)


def csr_sorted_lists(off, idx):
    return [np.sort(idx[off[k]:off[k + 1]]) for k in range(len(off) - 1)]


class Gpu:
    """A context with positions/masses uploaded, sorted and the tree built."""

    def __init__(self, pos, m32, **params):
        import torch

        import paper_1810_09898_gb300 as sg

        self.torch = torch
        self.sg = sg
        self.dev = torch.device("cuda:0")
        self.n = len(pos)
        self.ctx = sg.Context(self.n, **params)
        self.pos = torch.as_tensor(np.ascontiguousarray(pos), device=self.dev)
        self.m = torch.as_tensor(np.ascontiguousarray(m32), device=self.dev)
        self.keys = torch.empty(self.n, dtype=torch.int64, device=self.dev)
        self.perm = torch.empty(self.n, dtype=torch.int32, device=self.dev)
        self.ctx.sfc_keys_sort(self.pos, self.keys, self.perm)
        self.ctx.tree_build(self.pos, self.m)

    def t(self, a, dtype=None):
        return self.torch.as_tensor(np.ascontiguousarray(a), device=self.dev, dtype=dtype)

    def ngb_sets(self, active, h, kind, mode, g):
        torch = self.torch
        act = self.t(active, torch.int32)
        hh = self.t(h, torch.float64)
        off = torch.empty(len(active) + 1, dtype=torch.int64, device=self.dev)
        total = self.ctx.ngb_search(act, hh, kind, mode, g, off)
        idx = torch.empty(max(total, 1), dtype=torch.int32, device=self.dev)
        total2 = self.ctx.ngb_search(act, hh, kind, mode, g, off, idx, cap=total)
        assert total2 == total
        return off.cpu().numpy(), idx.cpu().numpy()[:total]

    def supersets(self, active, h, kind, g):
        """(group_first, members in key order, group candidate offsets, candidates)."""
        torch = self.torch
        act = self.t(active, torch.int32)
        hh = self.t(h, torch.float64)
        na = len(active)
        goff = torch.empty(na + 1, dtype=torch.int64, device=self.dev)
        gfirst = torch.empty(na + 1, dtype=torch.int32, device=self.dev)
        mem = torch.empty(max(na, 1), dtype=torch.int32, device=self.dev)
        ng, total = self.ctx.group_supersets(act, hh, kind, g, goff)
        cand = torch.empty(max(total, 1), dtype=torch.int32, device=self.dev)
        ng2, total2 = self.ctx.group_supersets(act, hh, kind, g, goff, gfirst, mem, cand, cap=total)
        assert (ng2, total2) == (ng, total)
        return (gfirst.cpu().numpy()[:ng + 1], mem.cpu().numpy()[:na], goff.cpu().numpy()[:ng + 1],
                cand.cpu().numpy()[:total])

    def density(self, active, h, iterate, mode, g):
        torch = self.torch
        n = self.n
        act = self.t(active, torch.int32)
        hh = self.t(np.array(h, dtype=np.float64, copy=True), torch.float64)
        rho = torch.zeros(n, dtype=torch.float32, device=self.dev)
        drho = torch.zeros_like(rho)
        f = torch.zeros_like(rho)
        nn = torch.zeros(n, dtype=torch.int32, device=self.dev)
        it = torch.zeros(n, dtype=torch.int32, device=self.dev)
        self.ctx.density(act, hh, iterate, mode, g, rho, drho, f, nn, it)
        return {"h": hh.cpu().numpy(), "rho": rho.cpu().numpy(), "drhodh": drho.cpu().numpy(),
                "f": f.cpu().numpy(), "nngb": nn.cpu().numpy(), "iters": it.cpu().numpy(),
                "stats": self.ctx.stats()}

    def hydro(self, active, h, rho32, f32, vel32, u32, mode, g):
        torch = self.torch
        n = self.n
        acc = torch.zeros((n, 3), dtype=torch.float32, device=self.dev)
        dudt = torch.zeros(n, dtype=torch.float32, device=self.dev)
        nn = torch.zeros(n, dtype=torch.int32, device=self.dev)
        self.ctx.hydro_force(self.t(active, torch.int32), self.t(h, torch.float64), self.t(rho32),
                             self.t(f32), self.t(vel32), self.t(u32), mode, g, acc, dudt, nn)
        return {"acc": acc.cpu().numpy(), "dudt": dudt.cpu().numpy(), "nngb": nn.cpu().numpy(),
                "stats": self.ctx.stats()}
