"""The domain decomposition's rank protocol (paper_1810_09898_gb300.domain) with two gloo
ranks on the CPU, against the single-domain oracle.

The particle set starts split at random over the ranks.  ``partition`` must give every
particle to exactly one rank, by contiguous key ranges; ``halo`` must import every
neighbour that a rank's own particles have on the other rank.  The device steps are
replaced here by CPU versions of the same operations (keys from the oracle's curve,
boxes and halo masks in numpy): the protocol, not the kernels, is under test (the
kernels are compared with these CPU versions on the GPU in test_gpu_domain.py).

Each rank then evaluates its own particles over its local set (own + imported) with the
oracle, the local set sorted by global index so that the oracle's sums run in the same
order as over the whole set: neighbour sets, density, hydro accelerations and the
smoothing-length iteration must equal the single-domain results bit for bit.  Hydro
takes rho and f of the imported particles from their own ranks' density, sent along the
hydro halo's plan (``exchange_columns``), not from the single-domain run.
"""

import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 3000
LEVEL = 3


class CpuOps:
    """CPU versions of the per-rank device steps of the decomposition."""

    def __init__(self, oracle):
        self.o = oracle

    def _keys(self, pos):
        return self.o.hilbert_keys(pos.numpy()).astype(np.int64)

    def sorted_keys(self, pos):
        import torch

        return torch.from_numpy(np.sort(self._keys(pos)))

    def owner_mask(self, pos, splitters):
        import torch

        dest = np.searchsorted(splitters.numpy(), self._keys(pos), side="right")
        return torch.from_numpy(np.left_shift(np.int64(1), dest.astype(np.int64)))

    def boxes(self, pos, m, h, level):
        import torch

        p, hh = pos.numpy(), h.numpy()
        cells = self._keys(pos) >> (3 * (21 - level))
        fix = np.floor(p * 2.0 ** 32)
        out = []
        for c in np.unique(cells):
            sel = cells == c
            hm = np.float32(hh[sel].max())
            if float(hm) < hh[sel].max():
                hm = np.nextafter(hm, np.float32(np.inf))
            out.append(np.concatenate([fix[sel].min(0) * 2.0 ** -32, (fix[sel].max(0) + 1.0) * 2.0 ** -32,
                                       [float(hm), sel.sum()]]))
        return torch.from_numpy(np.array(out).reshape(-1, 8))

    def halo_mask(self, pos, m, h, kind, widen, boxes, box_rank, self_rank, world):
        import torch

        p, hh, B, br = pos.numpy(), h.numpy(), boxes.numpy(), box_rank.numpy()
        mask = np.zeros(len(p), np.int64)
        for b in range(len(B)):
            if br[b] == self_rank:
                continue
            gap = np.zeros(len(p))
            for a in range(3):
                best = np.ones(len(p))
                for sh in (-1.0, 0.0, 1.0):
                    q = p[:, a] + sh
                    best = np.minimum(best, np.maximum(0.0, np.maximum(B[b, a] - q, q - B[b, 3 + a])))
                gap += best * best
            reach = np.maximum(widen * B[b, 6], hh) if kind == 1 else np.full(len(p), widen * B[b, 6])
            mask[gap < reach * reach * (1.0 + 1e-12)] |= np.int64(1) << np.int64(br[b])
        return torch.from_numpy(mask)

    def compact(self, mask, bit):
        import torch

        return torch.from_numpy(np.flatnonzero((mask.numpy() >> bit) & 1))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(oracle, sphgen):
    d = sphgen.make("clustered", N, config=21)
    m = d["m"].astype(np.float32).astype(np.float64)
    h, dens = oracle.density_iterate(d["pos"], m, np.full(N, d["h0"]))
    rows = np.column_stack([d["pos"], h, m, d["vel"], d["u"], np.arange(N, dtype=np.float64)])
    return d, rows, dens


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    import sphgen
    from paper_1810_09898_gb300.domain import Decomposition

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d, rows, dens = _problem(oracle, sphgen)
    start = np.random.default_rng(5).integers(0, world, N)
    D = Decomposition(world, rank, ops=CpuOps(oracle), level=LEVEL)
    own = D.partition(torch.from_numpy(rows[start == rank]))
    res = {"own": own[:, 9].numpy().astype(np.int64), "splitters": D.splitters.numpy()}
    own_rf = None   # rho and f of the own particles, in the order of the rows of `own`
    for kind, widen in ((0, 1.0), (1, 1.0), (0, 2.0)):
        ghosts = D.halo(own, kind, widen)
        cat = torch.cat([own, ghosts]).numpy()
        srt = np.argsort(cat[:, 9])
        local = cat[srt]
        gid = local[:, 9].astype(np.int64)
        tgt = np.flatnonzero(np.isin(gid, res["own"])).astype(np.int32)
        pos, h, m = local[:, :3], local[:, 3], local[:, 4]
        key = f"{kind}_{widen}"
        res["ghosts_" + key] = len(ghosts)
        if widen == 1.0:
            off, idx = oracle.ngb_sets(pos, h, tgt, kind)
            res["sets_" + key] = (gid[tgt], off, gid[idx])
        if kind == 0 and widen == 1.0:
            dl = oracle.density(pos, m, h, targets=tgt)
            res["rho"] = dl["rho"]
            # tgt runs in global-index order: back to the order of the rows of `own`
            own_rf = np.empty((len(own), 2))
            own_rf[np.argsort(res["own"])] = np.column_stack([dl["rho"], dl["f"]])
        if kind == 1:
            # rho and f of the imported particles were computed on their own ranks after
            # the hydro halo was sent: they follow its plan
            imp = D.exchange_columns(1, torch.from_numpy(own_rf)).numpy()
            assert imp.shape == (len(ghosts), 2)
            rf = np.concatenate([own_rf, imp])[srt]
            res["acc"] = oracle.hydro(pos, local[:, 5:8], m, h, rf[:, 0], rf[:, 1], local[:, 8], targets=tgt)["acc"]
        if kind == 0 and widen == 2.0:
            # the smoothing-length iteration of the own particles from scattered h
            h0 = h * np.exp(0.05 * np.random.default_rng(9).standard_normal(N))[gid]
            hi, di = oracle.density_iterate(pos, m, h0, targets=tgt)
            res["iter"] = (hi[tgt], di["rho"])
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_the_single_domain():
    sys.path.insert(0, ROOT)
    import oracle
    import sphgen

    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    d, rows, dens = _problem(oracle, sphgen)
    pos, h, m = rows[:, :3], rows[:, 3], rows[:, 4]
    # every particle on exactly one rank, by contiguous key ranges
    owners = np.concatenate([res[0]["own"], res[1]["own"]])
    assert np.array_equal(np.sort(owners), np.arange(N))
    keys = oracle.hilbert_keys(pos).astype(np.int64)
    assert keys[res[0]["own"]].max() < keys[res[1]["own"]].min()
    assert np.array_equal(res[0]["splitters"], res[1]["splitters"])
    assert 0.3 < len(res[0]["own"]) / N < 0.7
    # neighbour sets of both kinds, density and accelerations: as over the whole set
    for kind in (0, 1):
        off, idx = oracle.ngb_sets(pos, h, np.arange(N, dtype=np.int32), kind)
        for r in (0, 1):
            tg, lo, li = res[r][f"sets_{kind}_1.0"]
            for k, g in enumerate(tg):
                assert np.array_equal(li[lo[k]:lo[k + 1]], idx[off[g]:off[g + 1]]), (kind, r, g)
    full_d = oracle.density(pos, m, h)
    full_rho = full_d["rho"]
    full_acc = oracle.hydro(pos, rows[:, 5:8], m, h, full_d["rho"], full_d["f"], rows[:, 8])["acc"]
    h0 = h * np.exp(0.05 * np.random.default_rng(9).standard_normal(N))
    hi_full, di_full = oracle.density_iterate(pos, m, h0)
    for r in (0, 1):
        g = np.sort(res[r]["own"])
        assert np.array_equal(res[r]["rho"], full_rho[g])
        assert np.array_equal(res[r]["acc"], full_acc[g])
        assert np.array_equal(res[r]["iter"][0], hi_full[g])
        assert np.array_equal(res[r]["iter"][1], di_full["rho"][g])
        # the halo is part of the other domain (at this small N, h spans much of it)
        assert 0 < res[r]["ghosts_0_1.0"] < N - len(g)
        assert res[r]["ghosts_0_1.0"] <= res[r]["ghosts_1_1.0"]


def test_single_rank_needs_no_process_group():
    """world = 1: the partition keeps every row, the halo is empty, and later columns
    follow the (empty) plan; exchange_columns before any halo of that kind is an error."""
    import pytest
    import torch

    sys.path.insert(0, ROOT)
    import oracle
    import sphgen
    from paper_1810_09898_gb300.domain import Decomposition

    d, rows, dens = _problem(oracle, sphgen)
    D = Decomposition(1, 0, ops=CpuOps(oracle), level=LEVEL)
    with pytest.raises(RuntimeError):
        D.exchange_columns(1, torch.zeros((len(rows), 2), dtype=torch.float64))
    own = D.partition(torch.from_numpy(rows))
    assert np.array_equal(np.sort(own[:, 9].numpy()), np.arange(N, dtype=np.float64))
    assert D.splitters.numel() == 0
    for kind in (0, 1):
        ghosts = D.halo(own, kind)
        assert ghosts.shape == (0, rows.shape[1])
        cols = D.exchange_columns(kind, torch.ones((own.shape[0], 2), dtype=torch.float64))
        assert cols.shape == (0, 2)
