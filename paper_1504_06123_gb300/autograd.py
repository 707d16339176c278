"""torch.autograd.Function over the tangent-linear model of the C library (lbve_create_tangent).

forward(theta) runs the hybrid LB channel for a fixed number of steps with the parameters
theta = (G_inf, tau, gamma_c, g_x) and returns the final velocity and shear-stress profiles; the library
propagates d(state)/d(theta) alongside the state, so backward only contracts the incoming gradients
with the stored derivatives.  Argument marshalling only: every step runs in the CUDA library.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import lbve as L

THETA_NAMES = ("G_inf", "tau", "gamma_c", "g_x")


def _with_params(desc: L.lbve_channel_desc, theta) -> L.lbve_channel_desc:
    d = copy.copy(desc)
    G_inf, tau, gamma_c, g = [float(v) for v in theta]
    d.G_inf, d.tau, d.gamma_c = G_inf, tau, gamma_c
    d.g[0] = g
    return d


def run_profiles(desc: L.lbve_channel_desc, theta, steps: int, rho_init=None, with_tangents: bool = False):
    """(u_x [N], sigma_xy [N]) after `steps` steps, and with_tangents: their derivatives [4, N] each."""
    d = _with_params(desc, theta)
    dim = 2 if d.lattice == L.LBVE_D2Q9 else 3
    N = d.nx * d.ny * d.nz
    mask = L.LBVE_FIELD_U | L.LBVE_FIELD_SIGMA
    ixy = 2 if dim == 2 else 3                   # index of sigma_xy among the packed components
    if not with_tangents:
        h = L.lbve_create(d, rho_init)
        try:
            L.lbve_step(h, steps)
            f = L.lbve_fields(h, mask)
        finally:
            L.lbve_destroy(h)
        return f[:N].copy(), f[dim * N + ixy * N: dim * N + (ixy + 1) * N].copy()
    h = L.lbve_create_tangent(d, rho_init)
    try:
        L.lbve_step(h, steps)
        f = L.lbve_fields(h, mask)
        t = L.lbve_tangent_fields(h, mask)
    finally:
        L.lbve_destroy(h)
    u, s = f[:N].copy(), f[dim * N + ixy * N: dim * N + (ixy + 1) * N].copy()
    du, ds = t[:, :N].copy(), t[:, dim * N + ixy * N: dim * N + (ixy + 1) * N].copy()
    return u, s, du, ds


class LBVEChannel(torch.autograd.Function):
    """theta (float64 tensor [4]) -> (u_x [N], sigma_xy [N]) of the channel after `steps` steps."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, desc: L.lbve_channel_desc, steps: int, rho_init=None):
        u, s, du, ds = run_profiles(desc, theta.detach().cpu().numpy(), steps, rho_init, with_tangents=True)
        ctx.save_for_backward(torch.from_numpy(du), torch.from_numpy(ds))
        return torch.from_numpy(u), torch.from_numpy(s)

    @staticmethod
    def backward(ctx, grad_u, grad_s):
        du, ds = ctx.saved_tensors
        g = torch.zeros(4, dtype=torch.float64)
        if grad_u is not None:
            g = g + du @ grad_u.to(torch.float64)
        if grad_s is not None:
            g = g + ds @ grad_s.to(torch.float64)
        return g, None, None, None


def profile_loss(u, s, u_target, s_target):
    """mean((u - u*)^2)/max|u*|^2 + mean((sigma_xy - sigma*)^2)/max|sigma*|^2 (final step, all nodes)."""
    su = float(np.max(np.abs(np.asarray(u_target)))) ** 2
    ss = float(np.max(np.abs(np.asarray(s_target)))) ** 2
    ut = torch.as_tensor(u_target, dtype=torch.float64)
    st = torch.as_tensor(s_target, dtype=torch.float64)
    return torch.mean((u - ut) ** 2) / su + torch.mean((s - st) ** 2) / ss

