"""The decomposition's device steps (sphgrp_key_split, sphgrp_domain_boxes,
sphgrp_halo_select, sphgrp_mask_compact) on the GPU, through the C ABI.

* Each step against its CPU version (test_domain_ranks.CpuOps) on the same inputs:
  owner masks, boxes (fixed-point bounds and the FP32-rounded-up hmax) and halo masks
  equal.
* Two domains, one after the other on this one GPU (the exchange is an array selection
  here; the rank protocol with its collectives is tested on the CPU): every domain's own
  particles plus the halo its boxes select from the other domain are searched with the
  library's grouped density and hydro loops, own particles active; counts must equal the
  single-domain oracle bit for bit, density and accelerations within the usual bars.
"""

import numpy as np
import pytest

import oracle
import sphgen
from gpu_common import Gpu, dataset
from test_domain_ranks import CpuOps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem(cuda_device):
    n = 40000
    d = dataset("clustered", n, 22)
    m = d["m32"].astype(np.float64)
    h, dens = oracle.density_iterate(d["pos"], m, np.full(n, d["h0"]))
    return d, h, dens


def _t(a, dtype=None):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0", dtype=dtype)


def _split(d, world):
    import torch

    from paper_1810_09898_gb300.domain import LibOps

    keys = np.sort(oracle.hilbert_keys(d["pos"]).astype(np.int64))
    split = keys[[len(keys) * j // world for j in range(1, world)]]
    lib = LibOps()
    mask = lib.owner_mask(_t(d["pos"]), torch.as_tensor(split, device="cuda:0")).cpu().numpy()
    cpu = CpuOps(oracle).owner_mask(torch.from_numpy(d["pos"]), torch.from_numpy(split)).numpy()
    assert np.array_equal(mask, cpu)
    owner = sum(w * ((mask >> w) & 1) for w in range(world))   # the set bit's index
    lib.close()
    return owner


@pytest.mark.parametrize("world", [2, 4])
def test_steps_match_their_cpu_versions(problem, world):
    import torch

    from paper_1810_09898_gb300.domain import LibOps

    d, h, _ = problem
    owner = _split(d, world)
    cpu, lib = CpuOps(oracle), LibOps()
    boxes, ranks = [], []
    for r in range(world):
        sel = np.flatnonzero(owner == r)
        pos, m, hh = d["pos"][sel], d["m32"][sel], h[sel]
        b = lib.boxes(_t(pos), _t(m), _t(hh), 3).cpu().numpy()
        bc = cpu.boxes(torch.from_numpy(pos), None, torch.from_numpy(hh), 3).numpy()
        assert np.array_equal(b, bc)
        boxes.append(b)
        ranks.append(np.full(len(b), r, np.int32))
    B, R = np.concatenate(boxes), np.concatenate(ranks)
    for r in range(world):
        sel = np.flatnonzero(owner == r)
        pos, m, hh = d["pos"][sel], d["m32"][sel], h[sel]
        for kind, widen in ((0, 1.0), (1, 1.0), (0, 1.5)):
            mk = lib.halo_mask(_t(pos), _t(m), _t(hh), kind, widen, _t(B), _t(R), r, world).cpu().numpy()
            mc = cpu.halo_mask(torch.from_numpy(pos), None, torch.from_numpy(hh), kind, widen, torch.from_numpy(B),
                               torch.from_numpy(R), r, world).numpy()
            assert np.array_equal(mk, mc), (r, kind, widen, int((mk != mc).sum()))
            for bit in range(world):
                idx = lib.compact(_t(mk), bit).cpu().numpy()
                assert np.array_equal(idx, np.flatnonzero((mc >> bit) & 1))
    lib.close()


def test_two_domains_reproduce_the_single_domain(problem):
    from paper_1810_09898_gb300.domain import LibOps

    d, h, dens = problem
    n = len(h)
    owner = _split(d, 2)
    lib = LibOps()
    parts = []
    for r in range(2):
        sel = np.flatnonzero(owner == r)
        parts.append((sel, lib.boxes(_t(d["pos"][sel]), _t(d["m32"][sel]), _t(h[sel]), 3).cpu().numpy()))
    full_d = oracle.density(d["pos"], d["m32"].astype(np.float64), h)
    rho32, f32 = dens["rho"].astype(np.float32), dens["f"].astype(np.float32)
    full_h = oracle.hydro(d["pos"], d["vel32"].astype(np.float64), d["m32"].astype(np.float64), h,
                          rho32.astype(np.float64), f32.astype(np.float64), d["u32"].astype(np.float64))
    ghosts = {}
    for r in range(2):
        o = 1 - r
        so, bo = parts[o][0], parts[r][1]   # the other domain's particles, this domain's boxes
        for kind in (0, 1):
            mk = lib.halo_mask(_t(d["pos"][so]), _t(d["m32"][so]), _t(h[so]), kind, 1.0, _t(bo),
                               _t(np.full(len(bo), r, np.int32)), o, 2).cpu().numpy()
            ghosts[(r, kind)] = so[(mk >> r) & 1 == 1]
    lib.close()
    for r in range(2):
        own = parts[r][0]
        for kind in (0, 1):
            loc = np.concatenate([own, ghosts[(r, kind)]])
            G = Gpu(d["pos"][loc], d["m32"][loc])
            act = np.arange(len(own), dtype=np.int32)
            if kind == 0:
                out = G.density(act, h[loc], 0, 1, 16)
                assert np.array_equal(out["nngb"][act], full_d["nngb"][own])
                assert np.max(np.abs(out["rho"][act] / full_d["rho"][own] - 1.0)) <= 1e-5
            else:
                out = G.hydro(act, h[loc], rho32[loc], f32[loc], d["vel32"][loc], d["u32"][loc], 1, 16)
                assert np.array_equal(out["nngb"][act], full_h["nngb"][own])
                a, ref = out["acc"][act], full_h["acc"][own]
                assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= 1e-4
            G.ctx.close()
        # the halo is part of the other domain (at this N, h spans a good part of it)
        assert 0 < len(ghosts[(r, 0)]) < n - len(own)


def test_halo_select_rejects_box_ranks_outside_the_world(problem):
    """Box ranks are device data from the caller: a rank outside [0, world) is skipped by
    the kernel (no count or mask bit beyond the world) and the call reports EINVAL."""
    import torch

    import paper_1810_09898_gb300 as sg
    from paper_1810_09898_gb300.domain import LibOps

    d, h, _ = problem
    pos, m = d["pos"][:5000], d["m32"][:5000]
    lib = LibOps()
    B = lib.boxes(_t(pos), _t(m), _t(h[:5000]), 3)
    for bad in (2, -1, 64):
        R = np.zeros(len(B), np.int32)
        R[len(B) // 2:] = 1
        R[0] = bad
        with pytest.raises(sg.SphgrpError, match="EINVAL"):
            lib.halo_mask(_t(pos), _t(m), _t(h[:5000]), 0, 1.0, B.contiguous(), _t(R), 0, 2)
    # valid ranks afterwards: the context still works and matches the CPU version
    R = np.zeros(len(B), np.int32)
    R[len(B) // 2:] = 1
    mk = lib.halo_mask(_t(pos), _t(m), _t(h[:5000]), 0, 1.0, B.contiguous(), _t(R), 0, 2).cpu().numpy()
    mc = CpuOps(oracle).halo_mask(torch.from_numpy(pos), None, torch.from_numpy(h[:5000]), 0, 1.0,
                                  B.cpu(), torch.from_numpy(R), 0, 2).numpy()
    assert np.array_equal(mk, mc)
    lib.close()
