"""torch.autograd.Function over the density + hydro forward and its adjoint.

``sph_forces(ctx, pos, vel, m, u, h, group_size)`` returns ``(acc, rho)``: the hydro
accelerations and the densities of every particle at the smoothing lengths ``h``
(grouped form, one octree over ``pos``).  Its backward is ``sphgrp_backward``: for
incoming gradients ``dL/dacc`` and ``dL/drho`` it returns ``dL/dpos``, ``dL/dvel`` and
``dL/dm`` with the neighbour sets of the forward state held fixed and ``h`` treated
as the function of (pos, m) fixed by (4 pi / 3) h^3 rho = N_ngb m (implicit
function theorem).  ``h`` must therefore satisfy that relation -- for instance the
output of ``Context.density(..., iterate=1)`` with a tight ``nngb_tol`` -- otherwise
the gradient is that of the nearby solution of the relation.  ``u`` and ``h`` get no
gradient.

Everything runs in the CUDA library; this module only orders the calls.
"""

from __future__ import annotations

import torch

from .binding import GROUPED


def _build(ctx, pos, m):
    n = pos.shape[0]
    ctx.sfc_keys_sort(pos)
    ctx.tree_build(pos, m)
    return n


class SPHForces(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos, vel, m, u, h, sph_ctx, group_size):
        pos_d = pos.detach().to(torch.float64).contiguous()
        vel_f = vel.detach().to(torch.float32).contiguous()
        m_f = m.detach().to(torch.float32).contiguous()
        u_f = u.detach().to(torch.float32).contiguous()
        h_d = h.detach().to(torch.float64).contiguous()
        n = _build(sph_ctx, pos_d, m_f)
        dev = pos.device
        active = torch.arange(n, dtype=torch.int32, device=dev)
        rho = torch.empty(n, dtype=torch.float32, device=dev)
        drho = torch.empty_like(rho)
        fgrad = torch.empty_like(rho)
        nngb = torch.empty(n, dtype=torch.int32, device=dev)
        h_work = h_d.clone()
        sph_ctx.density(active, h_work, 0, GROUPED, group_size, rho, drho, fgrad, nngb)
        acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
        dudt = torch.empty(n, dtype=torch.float32, device=dev)
        sph_ctx.hydro_force(active, h_d, rho, fgrad, vel_f, u_f, GROUPED, group_size, acc, dudt)
        fctx.save_for_backward(pos_d, vel_f, m_f, u_f, h_d)
        # an output the loss does not use gives None (not zeros): a loss of rho alone
        # skips the hydro adjoint
        fctx.set_materialize_grads(False)
        fctx.sph_ctx = sph_ctx
        fctx.group_size = group_size
        fctx.dtypes = (pos.dtype, vel.dtype, m.dtype)
        return acc, rho

    @staticmethod
    def backward(fctx, g_acc, g_rho):
        pos_d, vel_f, m_f, u_f, h_d = fctx.saved_tensors
        sph_ctx = fctx.sph_ctx
        n = pos_d.shape[0]
        dev = pos_d.device
        # the context may have served other calls since the forward: rebuild its state
        _build(sph_ctx, pos_d, m_f)
        if g_acc is not None:
            g_acc = g_acc.to(torch.float32).contiguous()
        if g_rho is not None:
            g_rho = g_rho.to(torch.float32).contiguous()
        need_x, need_v, need_m = fctx.needs_input_grad[:3]
        if g_acc is None and g_rho is None:
            return (None,) * 7
        gx = torch.empty((n, 3), dtype=torch.float32, device=dev) if need_x else None
        gv = torch.empty((n, 3), dtype=torch.float32, device=dev) if need_v else None
        gm = torch.empty(n, dtype=torch.float32, device=dev) if need_m else None
        if gx is None and gv is None and gm is None:
            return (None,) * 7
        sph_ctx.backward(h_d, vel_f, u_f, g_acc, g_rho, fctx.group_size, gx, gv, gm)
        tx, tv, tm = fctx.dtypes
        return (gx.to(tx) if gx is not None else None,
                gv.to(tv) if gv is not None else None,
                gm.to(tm) if gm is not None else None,
                None, None, None, None)


def sph_forces(sph_ctx, pos, vel, m, u, h, group_size: int = 16):
    """(acc, rho) of all particles, differentiable in pos, vel and m."""
    return SPHForces.apply(pos, vel, m, u, h, sph_ctx, group_size)
