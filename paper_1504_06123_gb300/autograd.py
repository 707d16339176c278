"""torch.autograd.Functions over the differentiated hybrid step of the C library.

Both map theta = (G_inf, tau, gamma_c, g_x) to the final velocity and shear-stress profiles of a channel
run for a fixed number of steps:
  LBVEChannelAdjoint  reverse mode: the forward records a state image every K steps
                      (lbve_create_adjoint); backward replays the segments and runs the adjoint
                      (lbve_backward) -- one backward pass for all four parameters;
  LBVEChannel         forward mode: the library propagates d(state)/d(theta) with the state
                      (lbve_create_tangent); backward contracts the incoming gradients with them.
Argument marshalling only: every step and its derivative run in the CUDA library.
"""
from __future__ import annotations

import copy
import weakref

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


class AdjointRun:
    """Owner of one adjoint handle (its state images and history) between forward and backward.

    The handle is destroyed by release() -- after the backward pass -- or, when no backward ever runs
    (forward under torch.no_grad, outputs unused by any loss, an exception in between), as soon as the
    autograd graph that holds this owner is freed.  `live` counts the handles not yet destroyed."""
    live = 0

    def __init__(self, h):
        self.h = h
        AdjointRun.live += 1
        self._fin = weakref.finalize(self, AdjointRun._destroy, h)

    @staticmethod
    def _destroy(h):
        L.lbve_destroy(h)
        AdjointRun.live -= 1

    @property
    def alive(self) -> bool:
        return self._fin.alive

    def release(self):
        self._fin()          # runs _destroy once; later calls do nothing


class LBVEChannelAdjoint(torch.autograd.Function):
    """theta (float64 tensor [4]) -> (u_x [N], sigma_xy [N]); gradients by the adjoint with checkpoints.

    The forward runs in the precision `desc` asks for -- populations and history LBVE_F64 or LBVE_F32, history
    form P -- and the gradient is that of that model (of its FP32 trajectory for FP32 storage; the adjoint
    itself runs in FP64).  Other storages (the 16-bit history, the factor form) are refused rather than
    silently changed.  One backward pass per forward: the recorded states are freed by the first."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, desc: L.lbve_channel_desc, steps: int, checkpoint_every: int = 64,
                rho_init=None):
        if (desc.pop_precision not in (L.LBVE_F64, L.LBVE_F32) or desc.hist_storage not in (L.LBVE_F64, L.LBVE_F32)
                or desc.hist_form != L.LBVE_FORM_P):
            raise ValueError("LBVEChannelAdjoint differentiates the FP64 or FP32 model with the form-P history: "
                             "desc.pop_precision and desc.hist_storage must be LBVE_F64 or LBVE_F32")
        d = _with_params(desc, theta.detach().cpu().numpy())
        dim = 2 if d.lattice == L.LBVE_D2Q9 else 3
        N = d.nx * d.ny * d.nz
        run = AdjointRun(L.lbve_create_adjoint(d, rho_init, checkpoint_every))
        try:
            L.lbve_step(run.h, steps)
            f = L.lbve_fields(run.h, L.LBVE_FIELD_U | L.LBVE_FIELD_SIGMA)
        except Exception:
            run.release()
            raise
        if not ctx.needs_input_grad[0]:
            run.release()    # theta does not require a gradient: nothing will call backward
        ixy = 2 if dim == 2 else 3
        ctx.run, ctx.dim, ctx.N, ctx.ixy = run, dim, N, ixy
        return (torch.from_numpy(f[:N].copy()),
                torch.from_numpy(f[dim * N + ixy * N: dim * N + (ixy + 1) * N].copy()))

    @staticmethod
    def backward(ctx, grad_u, grad_s):
        if not ctx.run.alive:
            raise RuntimeError("LBVEChannelAdjoint: backward ran a second time; the recorded states are freed "
                               "by the first backward pass (run the forward again)")
        dim, N, ixy = ctx.dim, ctx.N, ctx.ixy
        nsig = 3 if dim == 2 else 6
        du = np.zeros((dim, N))
        ds = np.zeros((nsig, N))
        if grad_u is not None:
            du[0] = grad_u.detach().cpu().numpy()
        if grad_s is not None:
            ds[ixy] = grad_s.detach().cpu().numpy()
        try:
            g = L.lbve_backward(ctx.run.h, du, ds)
        finally:
            ctx.run.release()
        return torch.from_numpy(g), None, None, None, None


def profile_loss(u, s, u_target, s_target):
    """mean((u - u*)^2)/max|u*|^2 + mean((sigma_xy - sigma*)^2)/max|sigma*|^2 (final step, all nodes)."""
    su = float(np.max(np.abs(np.asarray(u_target)))) ** 2
    ss = float(np.max(np.abs(np.asarray(s_target)))) ** 2
    ut = torch.as_tensor(u_target, dtype=torch.float64)
    st = torch.as_tensor(s_target, dtype=torch.float64)
    return torch.mean((u - ut) ** 2) / su + torch.mean((s - st) ** 2) / ss

