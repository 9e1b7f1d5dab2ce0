"""torch.autograd.Function over the equilibrium Green's function.

`green_equilibrium(h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps)` takes
real torch tensors h (L x L, symmetric; real hopping), eps (2 x L) and U (L)
and returns (G_gtr, G_les) as complex128 tensors of shape
[n_steps+1, n_orb, n_orb].  The forward runs kg_green_equilibrium; the
backward runs kg_green_equilibrium_vjp (the library's checkpointed adjoint)
with the incoming complex cotangents.  Both are argument marshalling only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as K


class GreenEquilibrium(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps, opts, checkpoint):
        hn = h.detach().cpu().numpy().astype(np.float64)
        en = eps.detach().cpu().numpy().astype(np.float64)
        un = U.detach().cpu().numpy().astype(np.float64)
        handle = K.kg_build_sector(L, n_up, n_dn, hn, en, un)
        try:
            Gg, Gl = K.kg_green_equilibrium(handle, orbitals, dt, n_steps, opts)
        except Exception:
            K.kg_free_sector(handle)
            raise
        ctx.handle = handle
        ctx.args = (L, orbitals, dt, n_steps, opts, checkpoint)
        return torch.from_numpy(Gg), torch.from_numpy(Gl)

    @staticmethod
    def backward(ctx, dGg, dGl):
        L, orbitals, dt, n_steps, opts, checkpoint = ctx.args
        try:
            g_eps, g_hre, _, g_U = K.kg_green_equilibrium_vjp(
                ctx.handle, L, orbitals, dt, n_steps,
                None if dGg is None else dGg.detach().cpu().numpy(),
                None if dGl is None else dGl.detach().cpu().numpy(), opts, checkpoint)
        finally:
            K.kg_free_sector(ctx.handle)
            ctx.handle = None
        # h is passed as a full symmetric matrix: split the tied gradient of
        # each pair (i, j) evenly between h_ij and h_ji
        gh = torch.from_numpy(0.5 * g_hre)
        gh.diagonal().mul_(2.0)
        return gh, torch.from_numpy(g_eps), torch.from_numpy(g_U), None, None, None, None, None, None, None, None


def green_equilibrium(h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps, opts=None, checkpoint=0):
    return GreenEquilibrium.apply(h, eps, U, L, n_up, n_dn, orbitals, dt, n_steps, opts, checkpoint)
