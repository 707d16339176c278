"""Write the FP64 oracle's gradient of the differentiation workload to gradient_channel_4x128_L512.json.

Calls only the oracle (and the seeded input generator for the target's perturbation signs).  The workload
is the differentiation config: D2Q9 channel 4 x 128, tau_LB 0.9, G_inf 0.01, tau 300 steps, gamma_c 0.1,
history L = 512 (B 4 x C 128), 4000 startup steps from rest; the body force g is the input recipe's value
for a wall Peclet number 3 (g = min(g_Pe, g_cap), stated below).  Loss (the reading of the config): at the
final step, over all fluid nodes, mean((u_x - u*)^2)/max|u*|^2 + mean((sigma_xy - s*)^2)/max|s*|^2, the
target (u*, s*) from the same oracle run with (G_inf, tau, gamma_c, g) scaled by 1 +- 0.1 (signs seeded 5).
Gradient: central finite differences, relative step h = 1e-4, eight oracle runs.

    python tests/golden/make_gradient_golden.py
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1504_06123_gb300 import inputs  # noqa: E402

NX, NY, TAU_LB, G_INF, TAU, GAMMA_C, C, B, STEPS, SEED, H = 4, 128, 0.9, 0.01, 300.0, 0.1, 128, 4, 4000, 5, 1e-4


def force_for_peclet(Pe, Hw, tau_lb, G_inf, tau, gamma_c, rho0=1.0, u_max=0.1):
    """The input recipe: wall shear rate Pe/tau, steady wall stress eta_N gd + G_inf tau_e gd balanced by the
    force on half the channel; capped where a channel with the background viscosity alone reaches u_max."""
    eta_N = rho0 / 3.0 * (tau_lb - 0.5)
    gd = Pe / tau
    inv_te = 1.0 / tau + gd / gamma_c
    g_pe = (eta_N * gd + G_inf * gd / inv_te) / (rho0 * Hw)
    return min(g_pe, 2.0 * eta_N * u_max / (rho0 * Hw * Hw))


G = force_for_peclet(3.0, NY / 2, TAU_LB, G_INF, TAU, GAMMA_C)


def profiles(theta):
    Gi, tau, gc, g = (float(v) for v in theta)
    ch = oracle.Channel(oracle.D2Q9, NX, NY, tau_lb=TAU_LB, G_inf=Gi, tau=tau, gamma_c=gc, g=(g, 0, 0), C=C, B=B)
    ch.step(STEPS)
    f = ch.fields()
    ch.close()
    return f["u"][:, 0].copy(), f["sigma"][:, 2].copy()


def loss(u, s, ut, st):
    return float(np.mean((u - ut) ** 2) / np.max(np.abs(ut)) ** 2 + np.mean((s - st) ** 2) / np.max(np.abs(st)) ** 2)


def main():
    t0 = time.time()
    theta = np.array([G_INF, TAU, GAMMA_C, G])
    theta_t = inputs.perturbed(theta, seed=SEED)
    ut, st = profiles(theta_t)
    L0 = loss(*profiles(theta), ut, st)
    grad = np.zeros(4)
    for k in range(4):
        tp, tm = theta.copy(), theta.copy()
        tp[k] *= 1 + H
        tm[k] *= 1 - H
        grad[k] = (loss(*profiles(tp), ut, st) - loss(*profiles(tm), ut, st)) / (2 * H * theta[k])
    out = {
        "what": "FP64 oracle, central finite differences of the profile loss of the differentiation workload",
        "workload": {"lattice": "D2Q9", "nx": NX, "ny": NY, "tau_lb": TAU_LB, "C": C, "B": B, "steps": STEPS,
                     "peclet": 3.0, "target_seed": SEED},
        "theta_names": ["G_inf", "tau", "gamma_c", "g_x"],
        "theta": theta.tolist(), "theta_target": theta_t.tolist(), "h_relative": H,
        "loss": L0, "gradient": grad.tolist(),
        "u_target": ut.tolist(), "sigma_xy_target": st.tolist(),
        "oracle_threads": oracle.threads(), "seconds": round(time.time() - t0, 1),
    }
    assert all(math.isfinite(v) for v in out["gradient"])
    with open(os.path.join(HERE, "gradient_channel_4x128_L512.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("gradient", grad, "loss", L0, f"{out['seconds']} s")


if __name__ == "__main__":
    main()
