"""GPU parity at the workloads' stated sizes and lengths, against the FP64 oracle.

The flows start from rest without density noise, so they stay invariant along the periodic flow axis x:
every column of the GPU channel (every x-slice of the duct) must match the oracle's one-column channel
(one-slice duct) of the same width, history grid and parameters, and each comparison below takes the worst
column.  That keeps the oracle affordable at full history length and full run length (its node loops run on
all host cores).  The GPU's columns agree bitwise when every node tile sums its history in the same order;
the balanced ranges of the 16-bit form F cut the tiles at different points, and the columns then differ by
rounding.

  channel 1024 x 512, L = 1024 (B 8 x C 128): 5000 startup steps and 1000 cessation steps (force off),
      plain FP32 history (<= 1e-5) and the 16-bit history (<= 1e-3), each in form P (E - 1 advanced in
      place) and form F (the factor storage)
  duct 32^3 sub-run of the 128^3 duct, L = 512 (B 4 x C 128): 3000 steps, both forms, errors per field
  64-channel batch, L = 1024: 4000 startup + 2000 cessation steps, narrowest, median and widest channel

Per-field errors are normwise max-relative, max|x - x_ref| / max|x_ref|, and are printed for the record.
After cessation the flow decays towards rest (the narrowest batch channel's velocity by four orders of
magnitude in 2000 steps), and a field's magnitude can fall to the level of its storage rounding: there the
denominator is held at 1e-2 of the field's largest magnitude at the checkpoints so far, so that a decayed
field is still compared at one percent of its peak, not at its rounding floor.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import configs
from paper_1504_06123_gb300 import lbve as L

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64, S16 = L.LBVE_F32, L.LBVE_F64, L.LBVE_S16
FP, FF = L.LBVE_FORM_P, L.LBVE_FORM_F
# (population precision, history storage, history form)
PLAIN, RED, PLAIN_F, RED_F = (F64, F32, FP), (F32, S16, FP), (F64, F32, FF), (F32, S16, FF)
FORMS = [PLAIN, RED, PLAIN_F, RED_F]
TOL = {PLAIN: 1e-5, RED: 1e-3, PLAIN_F: 1e-5, RED_F: 1e-3}
NAME = {PLAIN: "plain FP32 history", RED: "16-bit history", PLAIN_F: "form F FP32 history",
        RED_F: "form F 16-bit history"}


def rel(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    num = np.max(np.abs(x - ref))
    return (0.0 if num == 0 else math.inf) if den == 0 else float(num / den)


def run_peaks(refs: list) -> dict:
    """Largest magnitude of each compared field over the oracle checkpoints given."""
    pk = {k: max(float(np.max(np.abs(r[k]))) for r in refs) for k in ("u", "sigma", "kappa", "rho")}
    pk["sigma_xy"] = max(float(np.max(np.abs(r["sigma"][:, -1 if r["sigma"].shape[1] == 3 else 3]))) for r in refs)
    return pk


def field_errors(got: dict, ref: dict, ixy: int, peaks: dict | None = None) -> dict:
    """u, sigma, sigma_xy, N1 (on the sigma scale), kappa and rho of every column / slice against the oracle's
    one (the worst column); with `peaks`, a denominator below 1e-2 of the field's peak is held there (decayed
    flow after cessation)."""
    def cols(key, r):   # got[key] as [slice][x][...] against r as [slice][1][...]
        x = np.asarray(got[key], dtype=np.float64)
        return x.reshape(x.shape[0], x.shape[1], -1), np.asarray(r, dtype=np.float64).reshape(x.shape[0], 1, -1)

    def err(key, x, r):
        den = np.max(np.abs(r))
        if peaks is not None:
            den = max(den, 1e-2 * peaks[key])
        num = np.max(np.abs(x - r))
        return (0.0 if num == 0 else math.inf) if den == 0 else float(num / den)
    e = {k: err(k, *cols(k, ref[k])) for k in ("u", "sigma", "kappa", "rho")}
    gs, rs = cols("sigma", ref["sigma"])
    e["sigma_xy"] = err("sigma_xy", gs[..., ixy], rs[..., ixy])
    sig_den = np.max(np.abs(ref["sigma"]))
    if peaks is not None:
        sig_den = max(sig_den, 1e-2 * peaks["sigma"])
    gn, rn = cols("n1", ref["n1"])
    e["n1_on_sigma_scale"] = float(np.max(np.abs(gn - rn)) / max(sig_den, 1e-300))
    return e


def check(errs: dict, tol: float, what: str):
    print(what, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= tol, f"{what}: {k} error {v:.3e} > {tol:.0e}"


def columns(f: dict, nx: int, ny: int, nz: int = 1) -> dict:
    """The fields as [slice][x][...] (node n = x + nx (y + ny z)); field_errors compares every x."""
    return {k: np.asarray(v).reshape(nz * ny, nx, -1) for k, v in f.items()}


# ---------------------------------------------------------------------------------------------
# The 1024 x 512 channel at L = 1024 through startup and cessation
# ---------------------------------------------------------------------------------------------
CHANNEL_CP = (40, 1000, 5000, 5400, 6000)


@pytest.fixture(scope="module")
def channel_oracle():
    w = configs.plain_channel_large()
    orc = oracle.Channel(oracle.D2Q9, 1, w.ny, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                         g=(w.g, 0, 0), C=w.C, B=w.B)
    out, t = {}, 0
    for cp in CHANNEL_CP:
        orc.step(cp - t)
        t = cp
        out[cp] = orc.fields()
        if t == w.steps:
            orc.set_force((0, 0, 0))
    orc.close()
    return w, out


@pytest.mark.parametrize("prec", FORMS)
def test_channel_1024x512_L1024_startup_cessation_vs_oracle(channel_oracle, prec):
    w, ref = channel_oracle
    ch = L.Channel(w.desc(precision=prec[0], hist_storage=prec[1], hist_form=prec[2]))
    t = 0
    for cp in CHANNEL_CP:
        ch.step(cp - t)
        t = cp
        got = columns(ch.fields(), w.nx, w.ny)
        pk = run_peaks([ref[c] for c in CHANNEL_CP if c <= cp])
        check(field_errors(got, ref[cp], 2, pk), TOL[prec], f"channel 1024x512 L1024 {NAME[prec]} step {cp}:")
        if t == w.steps:
            ch.set_force((0, 0, 0))
    ch.close()


# ---------------------------------------------------------------------------------------------
# The duct's 32^3 sub-run at the duct's history (L = 512) for its 3000 steps
# ---------------------------------------------------------------------------------------------
DUCT_CP = (40, 500, 1500, 3000)


def duct_subrun():
    w = configs.duct_3d()
    n = 32
    g = configs.force_for_peclet(30.0, n / 2, w.tau_lb, w.G_inf, w.tau, w.gamma_c)
    return w, n, g


@pytest.fixture(scope="module")
def duct_oracle():
    w, n, g = duct_subrun()
    orc = oracle.Channel(oracle.D3Q19, 1, n, n, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                         g=(g, 0, 0), C=w.C, B=w.B)
    out, t = {}, 0
    for cp in DUCT_CP:
        orc.step(cp - t)
        t = cp
        out[cp] = orc.fields()
    orc.close()
    return out


@pytest.mark.parametrize("prec", FORMS)
def test_duct_32cubed_L512_3000_steps_vs_oracle(duct_oracle, prec):
    w, n, g = duct_subrun()
    assert (w.C, w.B, w.steps) == (128, 4, 3000)
    ch = L.Channel(L.make_desc(L.LBVE_D3Q19, n, n, n, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                               g=(g, 0, 0), C=w.C, B=w.B, precision=prec[0], hist_storage=prec[1],
                               hist_form=prec[2]))
    t = 0
    for cp in DUCT_CP:
        ch.step(cp - t)
        t = cp
        got = columns(ch.fields(), n, n, n)
        check(field_errors(got, duct_oracle[cp], 3), TOL[prec], f"duct 32^3 L512 {NAME[prec]} step {cp}:")
    ch.close()


# ---------------------------------------------------------------------------------------------
# The 64-channel batch through 4000 startup and 2000 cessation steps
# ---------------------------------------------------------------------------------------------
BATCH_CP = (48, 1000, 4000, 4500, 6000)


def sampled_channels(ws):
    order = sorted(range(len(ws)), key=lambda i: ws[i].ny)
    return order[0], order[len(order) // 2], order[-1]


@pytest.fixture(scope="module")
def batch_oracle():
    ws = configs.batched_channels()
    out = {}
    for i in sampled_channels(ws):
        w = ws[i]
        o = oracle.Channel(oracle.D2Q9, 1, w.ny, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                           g=(w.g, 0, 0), C=w.C, B=w.B)
        t, rec = 0, {}
        for cp in BATCH_CP:
            o.step(cp - t)
            t = cp
            rec[cp] = o.fields()
            if t == w.steps:
                o.set_force((0, 0, 0))
        o.close()
        out[i] = rec
    return ws, out


@pytest.mark.parametrize("prec", FORMS)
def test_batch64_startup_cessation_vs_oracle(batch_oracle, prec):
    ws, ref = batch_oracle
    assert all((w.steps, w.off_steps) == (4000, 2000) for w in ws)
    ch = L.Channel([w.desc(precision=prec[0], hist_storage=prec[1], hist_form=prec[2]) for w in ws])
    t = 0
    for cp in BATCH_CP:
        ch.step(cp - t)
        t = cp
        f = ch.fields()
        for i, r in ref.items():
            w = ws[i]
            got = columns(ch.channel_fields(i, f), w.nx, w.ny)
            pk = run_peaks([r[c] for c in BATCH_CP if c <= cp])
            check(field_errors(got, r[cp], 2, pk), TOL[prec],
                  f"batch channel {i} (ny {w.ny}) {NAME[prec]} step {cp}:")
        if t == ws[0].steps:
            ch.set_force((0, 0, 0))          # cessation in every channel
    ch.close()
