"""Startup and cessation of pressure-driven channel flow in the paper's own parameter regime (Sec. IV).

The transients of Figs. Qall, QT and figtau are curves of the velocity, shear stress and normal-stress
difference at the wall distance y/H = d_1/2 = 0.51 of channels whose widths are given by the ratio
t_wall/tau_0 in {0.01, 0.1, 0.5, 1, 2, 4, 8}, for theta = tau/tau_0 = 10 (and 100 for three of them),
normalised by their steady-state values.  This module turns those dimensionless numbers into lattice
channels, runs all of them as one batch (one set of launches per step for every channel), records the
probe values on the device every `every` steps, and returns the series.

Lattice units (dt = dx = 1, rho0 = 1).  With the background viscosity eta_inf = G_inf tau_0 equal to the
BGK viscosity rho0 nu_N, nu_N = (tau_LB - 1/2)/3:
  - t_wall = 4 H^2 rho0 / (pi^2 G_inf tau_0) = 4 H^2 / (pi^2 nu_N)          (Sec. IV, transient dynamics)
  - tau_0 = t_wall / (t_wall/tau_0),  G_inf = rho0 nu_N / tau_0,  tau = theta tau_0
  - the drive: the pressure drop over one channel width equals G_inf (Fig. steadystate: Delta p/(2H) =
    G_inf), i.e. rho0 g = G_inf/(2H); the wall shear stress is G_inf/2, five times the yield stress
    G_inf gamma_c at gamma_c = 1/10 (Sec. II).
  - node j (0 <= j < ny) sits at distance j + 1/2 from the wall at y = -1/2, so y/H = (j + 1/2)/H with
    H = ny/2 (d_0 = 0.5/H and d_1/2 = (H/2 + 1/2)/H, the values printed for 100, 200 and 800 nodes).
    The probe at d is the linear interpolation between the two nodes around it.
"""
from __future__ import annotations

import math
import warnings
from dataclasses import dataclass

import numpy as np

from . import lbve as L

PAPER_T_WALL_OVER_TAU0 = (0.01, 0.1, 0.5, 1.0, 2.0, 4.0, 8.0)   # heavy lines of Fig. Qall
PAPER_THETA = 10.0                                              # Sec. III: "unless stated otherwise"
PAPER_THETA_SLOW = 100.0                                        # Fig. figtau, for t_wall/tau_0 = 0.1, 1, 4
PAPER_GAMMA_C = 0.1                                             # Sec. II
PAPER_TAU_LB = 0.9                                              # Sec. III default
D_HALF = 0.51                                                   # probe position of Figs. Qall, QT, figtau
PAPER_SLOW_POINTS = (0.1, 1.0, 4.0)                             # t_wall/tau_0 of Fig. figtau at theta = 100


def nu_of(tau_lb: float) -> float:
    """BGK kinematic viscosity c_s^2 (tau_LB - 1/2)."""
    return (tau_lb - 0.5) / 3.0


@dataclass(frozen=True)
class RegimeChannel:
    """One channel of the sweep in lattice units."""
    ratio: float      # t_wall / tau_0
    theta: float      # tau / tau_0
    ny: int
    tau_lb: float
    gamma_c: float
    H: float
    nu: float
    t_wall: float
    tau0: float
    G_inf: float
    tau: float
    g: float

    def desc(self, *, nx: int = 1, C: int = 128, B: int, precision=L.LBVE_F64, hist_storage=L.LBVE_F32,
             model=L.LBVE_MODEL_NLM, drive: bool = True) -> L.lbve_channel_desc:
        return L.make_desc(L.LBVE_D2Q9, nx, self.ny, tau_lb=self.tau_lb, G_inf=self.G_inf, tau=self.tau,
                           gamma_c=self.gamma_c, g=(self.g if drive else 0.0, 0.0, 0.0), C=C, B=B,
                           precision=precision, hist_storage=hist_storage, model=model)


def regime_channel(ratio: float, theta: float, ny: int, tau_lb: float = PAPER_TAU_LB,
                   gamma_c: float = PAPER_GAMMA_C, rho0: float = 1.0) -> RegimeChannel:
    """Lattice parameters of a channel of ny nodes with the given t_wall/tau_0 and theta (module doc)."""
    if ratio <= 0 or theta <= 0 or ny < 2 or tau_lb <= 0.5:
        raise ValueError("need ratio > 0, theta > 0, ny >= 2, tau_lb > 1/2")
    nu = nu_of(tau_lb)
    H = ny / 2.0
    t_wall = 4.0 * H * H / (math.pi ** 2 * nu)
    tau0 = t_wall / ratio
    G_inf = rho0 * nu / tau0
    return RegimeChannel(ratio=ratio, theta=theta, ny=ny, tau_lb=tau_lb, gamma_c=gamma_c, H=H, nu=nu,
                         t_wall=t_wall, tau0=tau0, G_inf=G_inf, tau=theta * tau0, g=G_inf / (2.0 * H * rho0))


def width_for(ratio: float, tau0_steps: float, tau_lb: float = PAPER_TAU_LB, ny_min: int = 8) -> int:
    """Even channel width whose tau_0 is closest to tau0_steps at this t_wall/tau_0 (so that the channels
    of one batch need about the same number of steps): H = (pi/2) sqrt(nu_N ratio tau_0)."""
    H = 0.5 * math.pi * math.sqrt(nu_of(tau_lb) * ratio * tau0_steps)
    return max(ny_min, 2 * int(round(H)))


def paper_points(with_slow: bool = True):
    """(t_wall/tau_0, theta) of the paper's transient figures: the seven widths of Fig. Qall at theta = 10,
    and (with_slow) the three of Fig. figtau at theta = 100."""
    pts = [(r, PAPER_THETA) for r in PAPER_T_WALL_OVER_TAU0]
    if with_slow:
        pts += [(r, PAPER_THETA_SLOW) for r in PAPER_SLOW_POINTS]
    return pts


def tau0_for_width(ny: int, ratio: float = 1.0, tau_lb: float = PAPER_TAU_LB) -> float:
    """tau_0 (steps) of a channel of ny nodes at this t_wall/tau_0: 4 H^2 / (pi^2 nu_N ratio)."""
    return 4.0 * (ny / 2.0) ** 2 / (math.pi ** 2 * nu_of(tau_lb) * ratio)


def probe_nodes(ny: int, d: float):
    """(j0, w): the probe at wall distance d (in units of H = ny/2) is (1 - w) v[j0] + w v[j0 + 1]."""
    H = ny / 2.0
    y = d * H - 0.5
    if not (0.0 <= y <= ny - 1):
        raise ValueError("probe position outside the nodes")
    j0 = min(int(math.floor(y)), ny - 2)
    return j0, y - j0


def history_blocks(span_steps: float, C: int = 128) -> int:
    """Smallest number of blocks B whose quasi-logarithmic grid, C (2^B - 1) steps, spans span_steps."""
    B = 1
    while C * (2 ** B - 1) < span_steps:
        B += 1
    return B


def sweep_descs(points, tau0_steps: float = 4000.0, *, ny=None, C: int = 128, span_tau: float = 5.0,
                B: int | None = None, tau_lb: float = PAPER_TAU_LB, gamma_c: float = PAPER_GAMMA_C, nx: int = 1,
                precision=L.LBVE_F64, hist_storage=L.LBVE_F32, ny_min: int = 8):
    """(channels, descs, B) of a batch of paper-regime channels: points = [(t_wall/tau_0, theta)], widths
    from width_for(ratio, tau0_steps) unless `ny` gives them, a history grid of C-point blocks spanning
    span_tau times the largest tau (or B blocks)."""
    points = [(float(r), float(th)) for r, th in points]
    widths = list(ny) if ny is not None else [width_for(r, tau0_steps, tau_lb, ny_min) for r, _ in points]
    channels = [regime_channel(r, th, w, tau_lb, gamma_c) for (r, th), w in zip(points, widths)]
    if B is None:
        B = history_blocks(span_tau * max(c.tau for c in channels), C)
    descs = [c.desc(nx=nx, C=C, B=B, precision=precision, hist_storage=hist_storage) for c in channels]
    return channels, descs, B


def probe_plan(channels, offsets, nx: int, d: float = D_HALF):
    """(node indices, weights): two nodes of column x = 0 around wall distance d in every channel (the
    flow is x-invariant); offsets are the channels' first nodes in the batch."""
    nodes, weights = [], []
    for c, off in zip(channels, offsets):
        j0, w = probe_nodes(c.ny, d)
        nodes += [off + j0 * nx, off + (j0 + 1) * nx]
        weights.append(w)
    return np.array(nodes, dtype=np.int64), weights


class RegimeSweep:
    """A batch of paper-regime channels, driven from rest (startup), then released (cessation).

    points: sequence of (t_wall/tau_0, theta); the other arguments as for sweep_descs.  Every channel is
    probed at wall distance d.
    """

    def __init__(self, points, tau0_steps: float = 4000.0, *, d: float = D_HALF, nx: int = 1, **kw):
        self.channels, self.descs, self.B = sweep_descs(points, tau0_steps, nx=nx, **kw)
        self.C = self.descs[0].hist_C
        self.nx = nx
        self.d = d
        self.batch = L.Channel(self.descs)
        offsets = [L.lbve_channel_nodes(self.batch.h, k)[0] for k in range(len(self.channels))]
        self.nodes, self.weights = probe_plan(self.channels, offsets, nx, d)
        self._records = []

    @property
    def updates_per_step(self) -> int:
        """Node-history updates per step, at most: every node advances all (up to B C) retained points."""
        return sum(desc.nx * desc.ny for desc in self.descs) * self.B * self.C

    def run(self, steps: int, every: int = 1, stream=None):
        """Advance `steps` steps, recording the probes every `every` steps (device-side)."""
        cap = steps // every + 1
        L.lbve_set_probes(self.batch.h, self.nodes, every, cap)
        self.batch.step(steps, stream)
        t, vals, tot = L.lbve_probe_read(self.batch.h, len(self.nodes), 2, cap, stream)
        if tot != len(t):
            raise RuntimeError("probe buffer overflow")
        self._records.append((t, vals))
        return t, vals

    def startup(self, steps: int, every: int = 1, stream=None):
        for k, c in enumerate(self.channels):
            L.lbve_set_force(self.batch.h, (c.g, 0.0, 0.0), k, stream)
        return self.run(steps, every, stream)

    def cessation(self, steps: int, every: int = 1, stream=None):
        L.lbve_set_force(self.batch.h, (0.0, 0.0, 0.0), -1, stream)
        return self.run(steps, every, stream)

    def series(self) -> list:
        """Per channel: {"t", "u", "sxy", "n1", "rho"} at d, over everything run so far.  Values of
        node pairs are interpolated; u is u_x, sxy the shear stress, n1 = sigma_xx - sigma_yy."""
        t = np.concatenate([r[0] for r in self._records])
        v = np.concatenate([r[1] for r in self._records])      # [k, 2 * nchan, 1 + 2 + 3]
        out = []
        for k, w in enumerate(self.weights):
            a, b = v[:, 2 * k], v[:, 2 * k + 1]
            p = (1.0 - w) * a + w * b
            out.append({"t": t, "rho": p[:, 0], "u": p[:, 1], "sxy": p[:, 5], "n1": p[:, 3] - p[:, 4]})
        return out

    def curves(self, n_startup: int) -> list:
        """The normalised transients of Figs. Qall / QT per channel: time on the scales of tau_0 and t_wall
        (t counted from the start of the phase) and u, sigma_xy, N1 at d divided by their values at the end
        of the startup phase (the steady state when that phase was long enough), split at step n_startup
        into {"startup": {...}, "cessation": {...}}."""
        out = []
        for c, ser in zip(self.channels, self.series()):
            t = ser["t"]
            k = int(np.searchsorted(t, n_startup, side="right"))
            if k == 0:
                raise ValueError("no record inside the startup phase")
            ss = {key: ser[key][k - 1] for key in ("u", "sxy", "n1")}
            # a normalising value that vanishes against its own series (a probe on the centreline, a
            # startup too short to build stress) cannot normalise it: that curve is NaN, with a warning
            for key in ("u", "sxy", "n1"):
                scale = float(np.max(np.abs(ser[key]))) if len(ser[key]) else 0.0
                if not (abs(ss[key]) > 1e-9 * scale) or scale == 0.0:
                    warnings.warn(f"channel {c.ny} nodes wide: {key} at the end of startup is {ss[key]!r}, too "
                                  "small to normalise its curve; returning NaN", RuntimeWarning, stacklevel=2)
                    ss[key] = np.nan
            phases = {}
            for name, sl, t0 in (("startup", slice(0, k), 0), ("cessation", slice(k, None), n_startup)):
                tt = (t[sl] - t0).astype(np.float64)
                phases[name] = {"t_over_tau0": tt / c.tau0, "t_over_twall": tt / c.t_wall,
                                **{key: ser[key][sl] / ss[key] for key in ("u", "sxy", "n1")}}
            out.append(phases)
        return out

    def close(self):
        self.batch.close()
