"""The five workloads of the hot path, as channel descriptions (synthetic inputs only).

Shapes follow the paper's setup: pressure-driven planar channel (D2Q9, periodic along the flow,
half-way bounce-back walls) started from rest, and the D3Q19 square duct.  History lengths count
points L = B*C with the paper's block size C = 128 where the workload gives "entries".

Driving force (input recipe): a requested wall Peclet number Pe = gammadot_w tau
gives the wall shear rate; the steady shear stress of the model at that rate,
eta_N gammadot_w + G_inf tau_e gammadot_w with 1/tau_e = 1/tau + gammadot_w/gamma_c, balanced by the
force on half the channel, gives g_Pe = sigma_w / (rho0 H).  Velocities must stay small against the
lattice speed: g is capped at the value for which a channel with only the background viscosity
would reach u_max = 0.1, g_cap = 2 eta_N u_max / (rho0 H^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import inputs
from . import lbve as L

CS2 = 1.0 / 3.0
U_MAX_CAP = 0.1


def force_for_peclet(Pe: float, H: float, tau_lb: float, G_inf: float, tau: float, gamma_c: float,
                     rho0: float = 1.0) -> float:
    eta_N = rho0 * CS2 * (tau_lb - 0.5)
    gd = Pe / tau
    inv_te = 1.0 / tau + (0.0 if math.isinf(gamma_c) else gd / gamma_c)
    sigma_w = eta_N * gd + G_inf * gd / inv_te
    g_pe = sigma_w / (rho0 * H)
    g_cap = 2.0 * eta_N * U_MAX_CAP / (rho0 * H * H)
    return min(g_pe, g_cap)


@dataclass
class Workload:
    name: str
    lattice: int
    nx: int
    ny: int
    nz: int
    tau_lb: float
    G_inf: float
    tau: float
    gamma_c: float
    g: float
    C: int
    B: int
    steps: int
    off_steps: int = 0                  # cessation steps with g = 0 after `steps`
    noise: float = 0.0
    seed: int = 0
    # plain FP32 form: the history (nearly all of the traffic) in FP32; the O(N) populations in FP64,
    # because FP32 populations alone leave ~1e-5 relative error in decaying flows (cessation)
    precision: int = L.LBVE_F64
    hist_storage: int | None = L.LBVE_F32
    model: int = L.LBVE_MODEL_NLM
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def L(self) -> int:
        return self.B * self.C

    def desc(self, **over) -> L.lbve_channel_desc:
        kw = dict(lattice=self.lattice, nx=self.nx, ny=self.ny, nz=self.nz, tau_lb=self.tau_lb, G_inf=self.G_inf,
                  tau=self.tau, gamma_c=self.gamma_c, g=(self.g, 0.0, 0.0), C=self.C, B=self.B,
                  precision=self.precision, hist_storage=self.hist_storage, model=self.model)
        kw.update(over)
        return L.make_desc(**kw)

    def rho_init(self):
        return inputs.initial_density(self.N, self.noise, self.seed)


def plain_channel_small() -> Workload:
    """D2Q9 4 x 32 channel, tau_LB 0.8, G_inf 0.01, tau 200, gamma_c 0.1, 256-step uniform history;
    g = 1e-6 for 2000 steps (startup), then 0 for 1000 (cessation)."""
    return Workload("channel_4x32_L256", L.LBVE_D2Q9, 4, 32, 1, 0.8, 0.01, 200.0, 0.1, 1e-6, 256, 1,
                    steps=2000, off_steps=1000, noise=0.0, seed=1)


def plain_channel_large() -> Workload:
    """D2Q9 1024 x 512 channel, FP32, tau_LB 0.9, G_inf 0.01, tau 1000, gamma_c 0.1, L = 1024 (B 8 x C 128),
    wall Peclet 30 (capped by the Mach limit), 5000 startup steps, density noise 1e-6 (seed 2)."""
    H = 512 / 2
    g = force_for_peclet(30.0, H, 0.9, 0.01, 1000.0, 0.1)
    return Workload("channel_1024x512_L1024", L.LBVE_D2Q9, 1024, 512, 1, 0.9, 0.01, 1000.0, 0.1, g, 128, 8,
                    steps=5000, noise=1e-6, seed=2)


def wm_channel_large() -> Workload:
    """The 1024 x 512 channel of plain_channel_large with the White-Metzner form of Eq. (nlmax)."""
    w = plain_channel_large()
    w.name = "channel_1024x512_L1024_wm"
    w.model = L.LBVE_MODEL_WM
    return w


def inlm_channel_large() -> Workload:
    """The instantaneous nlM of Eq. (inlM) (no history) in a 4096 x 512 channel: the rows of the benchmark
    channel, four times its length, so that the populations (302 MB per copy in FP64) exceed the 129 MB L2
    as the history does in the integral model.  tau = 10 (G_inf tau = 0.1): the explicit instantaneous
    stress is stable up to G_inf tau_M of about 1.7 nu_N (0.23 at tau_LB 0.9) with the density source;
    wall Peclet 30, capped like the others."""
    H = 512 / 2
    g = force_for_peclet(30.0, H, 0.9, 0.01, 10.0, 0.1)
    return Workload("channel_4096x512_inlm", L.LBVE_D2Q9, 4096, 512, 1, 0.9, 0.01, 10.0, 0.1, g, 4, 1,
                    steps=5000, noise=1e-6, seed=2, model=L.LBVE_MODEL_INLM)


def duct_3d() -> Workload:
    """D3Q19 128^3 square duct, G_inf 0.005, tau 500, gamma_c 0.1, L = 512 (B 4 x C 128), Pe 30 capped,
    3000 steps."""
    H = 128 / 2
    g = force_for_peclet(30.0, H, 0.9, 0.005, 500.0, 0.1)
    return Workload("duct_128cubed_L512", L.LBVE_D3Q19, 128, 128, 128, 0.9, 0.005, 500.0, 0.1, g, 128, 4,
                    steps=3000, noise=0.0, seed=3)


def gradient_channel() -> Workload:
    """D2Q9 4 x 128 channel, G_inf 0.01, tau 300, gamma_c 0.1, L = 512 (B 4 x C 128), 4000 steps."""
    H = 128 / 2
    g = force_for_peclet(3.0, H, 0.9, 0.01, 300.0, 0.1)
    return Workload("channel_4x128_L512", L.LBVE_D2Q9, 4, 128, 1, 0.9, 0.01, 300.0, 0.1, g, 128, 4,
                    steps=4000, noise=0.0, seed=5)


def batched_channels(n: int = 64, seed: int = 4) -> list:
    """64 quasi-1D channels (nx 4), widths log-uniform in [8, 512] (even), G_inf in [0.005, 0.02], tau in
    [100, 2000], gamma_c in [0.05, 0.3], Pe in [1, 100]; L = 1024 (B 8 x C 128); 4000 + 2000 steps."""
    widths = inputs.channel_widths(n, 8, 512, seed)
    p = inputs.uniform_params(n, {"G_inf": (0.005, 0.02), "tau": (100.0, 2000.0), "gamma_c": (0.05, 0.3),
                                  "Pe": (1.0, 100.0)}, seed + 1000)
    out = []
    for i in range(n):
        ny = int(widths[i])
        g = force_for_peclet(float(p["Pe"][i]), ny / 2, 0.9, float(p["G_inf"][i]), float(p["tau"][i]),
                             float(p["gamma_c"][i]))
        out.append(Workload(f"batch{i}", L.LBVE_D2Q9, 4, ny, 1, 0.9, float(p["G_inf"][i]), float(p["tau"][i]),
                            float(p["gamma_c"][i]), g, 128, 8, steps=4000, off_steps=2000))
    return out
