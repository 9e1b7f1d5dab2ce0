"""torch.autograd.Function over the equilibrium Green's function.

`green_equilibrium(h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps)` takes
real torch tensors h (L x L, symmetric; real hopping), eps (2 x L) and U (L)
and returns (G_gtr, G_les) as complex128 tensors of shape
[n_steps+1, n_orb, n_orb] on the device of h.  The forward runs
kg_green_equilibrium; the backward runs kg_green_equilibrium_vjp (the
library's checkpointed adjoint) with the incoming complex cotangents.  Both
are argument marshalling only.  When h is a CUDA tensor the library works on
torch's current stream of that device (unless `opts` names another stream).

The sector handle built by the forward (device tables and the cached ground
state, which the backward reuses) is owned by a small holder object saved on
the autograd context: the backward frees it, and if the graph is dropped
without a backward the holder frees it when it is garbage-collected.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as K


class _SectorHandle:
    """Owns one kg_sector handle; frees it once (explicitly or on collection)."""

    def __init__(self, handle):
        self.handle = handle

    def free(self):
        h, self.handle = self.handle, None
        if h:
            K.kg_free_sector(h)

    def __del__(self):
        try:
            self.free()
        except Exception:  # interpreter shutdown: the library may be gone
            pass


def _opts_for(device, opts):
    if opts is not None or device.type != "cuda":
        return opts
    o = K.kg_opts_default()
    o.stream = torch.cuda.current_stream(device).cuda_stream
    return o


class GreenEquilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps, opts, checkpoint):
        device = h.device
        opts = _opts_for(device, opts)
        hn = h.detach().cpu().numpy().astype(np.float64)
        en = eps.detach().cpu().numpy().astype(np.float64)
        un = U.detach().cpu().numpy().astype(np.float64)
        holder = _SectorHandle(K.kg_build_sector(L, n_up, n_dn, hn, en, un))
        try:
            Gg, Gl = K.kg_green_equilibrium(holder.handle, orbitals, dt, n_steps, opts)
        except Exception:
            holder.free()
            raise
        ctx.holder = holder
        ctx.args = (L, orbitals, dt, n_steps, opts, checkpoint, device)
        return torch.from_numpy(Gg).to(device), torch.from_numpy(Gl).to(device)

    @staticmethod
    def backward(ctx, dGg, dGl):
        L, orbitals, dt, n_steps, opts, checkpoint, device = ctx.args
        try:
            g_eps, g_hre, _, g_U = K.kg_green_equilibrium_vjp(
                ctx.holder.handle, L, orbitals, dt, n_steps,
                None if dGg is None else dGg.detach().cpu().numpy(),
                None if dGl is None else dGl.detach().cpu().numpy(), opts, checkpoint)
        finally:
            ctx.holder.free()
        # h is passed as a full symmetric matrix: split the tied gradient of
        # each pair (i, j) evenly between h_ij and h_ji
        gh = torch.from_numpy(0.5 * g_hre)
        gh.diagonal().mul_(2.0)
        return (gh.to(device), torch.from_numpy(g_eps).to(device), torch.from_numpy(g_U).to(device),
                None, None, None, None, None, None, None, None)


def green_equilibrium(h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps, opts=None, checkpoint=0):
    return GreenEquilibrium.apply(h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps, opts, checkpoint)
