"""Domain decomposition with halo import: one particle set over several ranks, one GPU
each (torch.distributed; NCCL on GPUs, gloo on CPU).

The paper's code splits the particles along the Hilbert curve into one contiguous key
range per MPI process (Sec. 1.2) and finds the neighbours that lie on other processes by
exporting particles in a second search phase (Sec. 1.1).  Here each rank imports instead:

1. ``partition``: the particles' keys are sampled on every rank and gathered; the
   samples' quantiles split the key order into one contiguous range per rank, and every
   particle is sent to the rank owning its key (one all-to-all).
2. ``halo``: every rank describes its domain by the tight boxes of its particles per
   octree cell of a coarse level, with the largest h in each box, and gathers every
   rank's boxes; each rank then sends every other rank the particles within reach of that
   rank's boxes (one all-to-all): for density within the box's largest h (times a margin
   for the growth of h in a smoothing-length iteration), for hydro within the larger of
   that and the particle's own h.  A rank's local set (its own particles and the
   imported ones) then holds every neighbour of its own particles, and its searches are
   purely local, with its own particles active.
3. ``exchange_columns``: values computed after the halo was sent (rho and f of the
   density loop, which hydro needs for its imported particles too) follow the same
   plan, one all-to-all of the columns.

The device steps (keys, owner masks, boxes, halo masks, compaction) are the library's
kernels (``LibOps``); the exchanges and the row gathers around them are the only host
work.  Records travel as float64 rows of ``FIELDS``; ``gid`` is the particle's global
index (exact in float64 up to 2^53).
"""

from __future__ import annotations

FIELDS = ("x", "y", "z", "h", "m", "vx", "vy", "vz", "u", "gid")
X, H, M, V, U, GID = slice(0, 3), 3, 4, slice(5, 8), 8, 9


class LibOps:
    """The per-rank device steps in the library's kernels (a context per call size)."""

    def __init__(self, **params):
        self._params = params
        self._ctx = None
        self._cap = 0

    def _context(self, n: int):
        from .binding import Context

        if self._ctx is None or n > self._cap:
            if self._ctx is not None:
                self._ctx.close()
            self._cap = max(n, 1)
            self._ctx = Context(self._cap, **self._params)
        return self._ctx

    def _built(self, pos, m):
        c = self._context(pos.shape[0])
        c.sfc_keys_sort(pos)
        c.tree_build(pos, m)
        return c

    def sorted_keys(self, pos):
        import torch

        c = self._context(pos.shape[0])
        keys = torch.empty(pos.shape[0], dtype=torch.int64, device=pos.device)
        c.sfc_keys_sort(pos, keys)
        return keys

    def owner_mask(self, pos, splitters):
        import torch

        c = self._context(pos.shape[0])
        c.sfc_keys_sort(pos)
        mask = torch.empty(pos.shape[0], dtype=torch.int64, device=pos.device)
        c.key_split(splitters, mask)
        return mask

    def boxes(self, pos, m, h, level: int):
        import torch

        c = self._built(pos, m)
        cap = max(1, min(pos.shape[0], 8 ** level))
        out = torch.empty((cap, 8), dtype=torch.float64, device=pos.device)
        nb = c.domain_boxes(h, level, out)
        return out[:nb].clone()

    def halo_mask(self, pos, m, h, kind, widen, boxes, box_rank, self_rank, world):
        import torch

        c = self._built(pos, m)
        mask = torch.empty(pos.shape[0], dtype=torch.int64, device=pos.device)
        counts = torch.empty(world, dtype=torch.int64, device=pos.device)
        c.halo_select(h, kind, widen, boxes, box_rank, self_rank, world, mask, counts)
        return mask

    def compact(self, mask, bit: int):
        import torch

        c = self._context(mask.shape[0])
        idx = torch.empty(max(mask.shape[0], 1), dtype=torch.int32, device=mask.device)
        k = c.mask_compact(mask, bit, idx)
        return idx[:k].long()

    def close(self):
        if self._ctx is not None:
            self._ctx.close()
            self._ctx = None


class Decomposition:
    """One rank's view of the decomposition.  world = 1 needs no process group."""

    def __init__(self, world: int, rank: int, ops=None, group=None, level: int = 3, samples: int = 256):
        self.world, self.rank, self.group = world, rank, group
        self.ops = ops if ops is not None else LibOps()
        self.level = level
        self.samples = samples
        self.splitters = None
        self.plans = {}   # halo kind -> (send index lists, send counts, receive counts)

    # -- collectives
    def _all_gather_rows(self, t):
        """Every rank's rows of t (variable counts), concatenated in rank order, and the
        count of every rank."""
        import torch
        import torch.distributed as dist

        if self.world == 1:
            return t, [t.shape[0]]
        n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
        ns = [torch.zeros_like(n) for _ in range(self.world)]
        dist.all_gather(ns, n, group=self.group)
        counts = [int(x.item()) for x in ns]
        cap = max(max(counts), 1)
        pad = torch.zeros((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[:t.shape[0]] = t
        outs = [torch.zeros_like(pad) for _ in range(self.world)]
        dist.all_gather(outs, pad, group=self.group)
        return torch.cat([o[:k] for o, k in zip(outs, counts)]), counts

    def _exchange(self, rows, mask, plan_key=None):
        """Every rank receives the rows whose mask has its bit, in rank order.  With
        plan_key the send index lists and the counts are kept for exchange_columns."""
        import torch

        idx = [self.ops.compact(mask, r) for r in range(self.world)]
        send_counts = [int(i.shape[0]) for i in idx]
        recv_counts = self._counts(send_counts, rows.device)
        if plan_key is not None:
            self.plans[plan_key] = (idx, send_counts, recv_counts)
        return self._send(rows, idx, send_counts, recv_counts)

    def _counts(self, send_counts, device):
        """Every rank's count for this rank, from every rank's counts (one all-to-all)."""
        import torch
        import torch.distributed as dist

        if self.world == 1:
            return list(send_counts)
        sc = torch.tensor(send_counts, dtype=torch.int64, device=device)
        rc = torch.empty_like(sc)
        dist.all_to_all_single(rc, sc, group=self.group)
        return [int(x) for x in rc.tolist()]

    def _send(self, rows, idx, send_counts, recv_counts):
        import torch
        import torch.distributed as dist

        parts = [rows[i] for i in idx]
        if self.world == 1:
            return parts[0]
        send = torch.cat(parts)
        recv = torch.empty((sum(recv_counts),) + tuple(rows.shape[1:]), dtype=rows.dtype, device=rows.device)
        dist.all_to_all_single(recv, send, output_split_sizes=recv_counts, input_split_sizes=send_counts,
                               group=self.group)
        return recv

    def exchange_columns(self, kind: int, values):
        """Values of the own particles (rows in the order of `own` given to halo(kind))
        sent along the same halo plan: the imported particles' values, in the order of
        the rows halo(kind) returned.  Between density and hydro this carries rho and f
        (and so P and c) of the hydro halo, whose rows were sent before they existed."""
        if kind not in self.plans:
            raise RuntimeError("exchange_columns needs a halo() of the same kind first")
        idx, sc, rc = self.plans[kind]
        return self._send(values, idx, sc, rc)

    # -- steps
    def partition(self, rows):
        """Rows of this rank's particles (the key range it owns), gathered from every rank."""
        import torch

        pos = rows[:, X].contiguous()
        keys = self.ops.sorted_keys(pos)
        step = max(1, keys.shape[0] // self.samples)
        sample, _ = self._all_gather_rows(keys[::step].contiguous())
        # quantiles of the gathered sample split the key order; keys have 63 bits, so
        # their int64 order is their order as unsigned keys
        k = sample.shape[0]
        if self.world > 1 and k > 0:
            srt = torch.sort(sample)[0]
            at = [min(k - 1, (j * k) // self.world) for j in range(1, self.world)]
            self.splitters = srt[torch.tensor(at, device=srt.device)].contiguous()
        else:
            self.splitters = torch.zeros(0, dtype=torch.int64, device=rows.device)
        mask = self.ops.owner_mask(pos, self.splitters)
        return self._exchange(rows, mask)

    def halo(self, own, kind: int, widen: float = 1.0):
        """Rows of the other ranks' particles that this rank's particles can reach (kind:
        0 density, 1 hydro; widen scales the boxes' largest h)."""
        import torch

        pos = own[:, X].contiguous()
        m = own[:, M].to(torch.float32).contiguous()
        h = own[:, H].contiguous()
        boxes = self.ops.boxes(pos, m, h, self.level)
        all_boxes, counts = self._all_gather_rows(boxes)
        box_rank = torch.cat([torch.full((k,), r, dtype=torch.int32, device=own.device)
                              for r, k in enumerate(counts)])
        mask = self.ops.halo_mask(pos, m, h, kind, widen, all_boxes.contiguous(), box_rank, self.rank, self.world)
        return self._exchange(own, mask, plan_key=kind)

