"""GPU parity of the two constitutive variants against the FP64 oracle, through the C ABI.

- LBVE_MODEL_INLM: the instantaneous nlM of Eq. (inlM) (Sec. IV): no history, the series summed in the
  collide kernel in the collision's arithmetic.
- LBVE_MODEL_WM: the White-Metzner form of Eq. (nlmax) (Sec. II): accumulated strain in the second
  exponential, one double per history point.

Tolerances (normwise max-relative per field, as in test_gpu_parity.py): FP64 1e-12; plain FP32 history
with FP64 populations 1e-5; all-FP32 5e-5.  The instantaneous model in FP32 sums its series in float
(resolution 6e-8 of the stress), inside the FP32 bars.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import inputs
from paper_1504_06123_gb300 import lbve as L
from tests.test_gpu_parity import TOL, PLAIN, ALL32, ALL64, compare, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = L.LBVE_F32, L.LBVE_F64
INLM, WM = L.LBVE_MODEL_INLM, L.LBVE_MODEL_WM
ORC_MODEL = {INLM: oracle.INLM, WM: oracle.WM}


def _apply_run(model, prec, lattice, nx, ny, nz, C, B, kseq, G, tau, gc):
    d = 2 if lattice == L.LBVE_D2Q9 else 3
    N = nx * ny * nz
    ch = L.Channel(L.make_desc(lattice, nx, ny, nz, G_inf=G, tau=tau, gamma_c=gc, C=C, B=B, precision=prec[0],
                               hist_storage=prec[1], model=model))
    ns = 3 if d == 2 else 6
    kap_dev = torch.empty((d * d, N), dtype=torch.float64, device="cuda")
    sig_dev = torch.empty((ns, N), dtype=torch.float64, device="cuda")
    out = []
    for t in range(kseq.shape[0]):
        kap_dev.copy_(torch.from_numpy(kseq[t].reshape(N, d * d).T.copy()))
        L.lbve_history_apply(ch.h, kap_dev, sig_dev)
        out.append(sig_dev.cpu().numpy().T.copy())
    ch.close()
    return out


# ---------------------------------------------------------------------------------------------
# The stress law alone on prescribed gradients (lbve_history_apply)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [ALL64, ALL32])
@pytest.mark.parametrize("lattice,nx,ny,nz", [(L.LBVE_D2Q9, 7, 115, 1), (L.LBVE_D3Q19, 3, 7, 11)])
def test_inlm_stress_law_vs_oracle(prec, lattice, nx, ny, nz):
    d = 2 if lattice == L.LBVE_D2Q9 else 3
    N = nx * ny * nz
    G, tau, gc = 0.02, 40.0, 0.1
    # general gradients up to tau_M |kappa| ~ 0.3 (tens of series terms), plus shear-dominated ones
    kseq = inputs.kappa_sequence(6, N, d, 4e-3, seed=21, shear=2e-3)
    ref = oracle.history_run(kseq, 4, 1, G, tau, gc, model=oracle.INLM)
    got = _apply_run(INLM, prec, lattice, nx, ny, nz, 4, 1, kseq, G, tau, gc)
    tol = 1e-12 if prec == ALL64 else 2e-6
    for t in range(kseq.shape[0]):
        assert np.all(np.isfinite(ref[t]))
        assert rel_err(got[t], ref[t]) <= tol, f"step {t}: {rel_err(got[t], ref[t]):.3e}"


def test_inlm_diverging_series_gives_nan_like_the_oracle():
    """Planar extension beyond 2 tau_M eps = 1 (UCM limit): Eq. (inlM) has no sum; both sides give NaN,
    and the converging nodes of the same launch agree."""
    tau = 50.0
    N = 4
    k = np.zeros((1, N, 2, 2))
    for n, x in enumerate([0.5, 0.9, 1.01, 2.0]):   # ratio 2 tau_M eps = x; 0.9 takes ~400 terms
        k[0, n] = np.diag([x / (2 * tau), -x / (2 * tau)])
    ref = oracle.history_run(k, 4, 1, 0.01, tau, math.inf, model=oracle.INLM)[0]
    got = _apply_run(INLM, ALL64, L.LBVE_D2Q9, 1, 4, 1, 4, 1, k, 0.01, tau, math.inf)[0]
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.all(np.isnan(got[2:])) and np.all(np.isfinite(got[:2]))
    np.testing.assert_allclose(got[:2], ref[:2], rtol=1e-11)


@pytest.mark.parametrize("prec", [ALL64, PLAIN])
@pytest.mark.parametrize("lattice,nx,ny,nz,C,B", [
    (L.LBVE_D2Q9, 7, 115, 1, 16, 4),      # 805 nodes: several tiles + ragged tail
    (L.LBVE_D2Q9, 33, 64, 1, 5, 3),       # odd C
    (L.LBVE_D3Q19, 3, 7, 11, 8, 3),       # 3x3 tensors
])
def test_wm_history_vs_oracle(prec, lattice, nx, ny, nz, C, B):
    d = 2 if lattice == L.LBVE_D2Q9 else 3
    N = nx * ny * nz
    T = 150
    G, tau, gc = 0.02, 40.0, 0.1
    kseq = inputs.kappa_sequence(T, N, d, 2e-3, seed=12, shear=1e-3)
    ref = oracle.history_run(kseq, C, B, G, tau, gc, model=oracle.WM)
    got = _apply_run(WM, prec, lattice, nx, ny, nz, C, B, kseq, G, tau, gc)
    tol = TOL[prec[1]]
    for t in list(range(0, T, 7)) + [T - 1]:
        e = rel_err(got[t], ref[t])
        assert e <= tol, f"step {t}: sigma error {e:.3e}"
    # and the variant is not the nlM: the same gradients give a different stress
    nlm = oracle.history_run(kseq, C, B, G, tau, gc, last_only=True)
    assert rel_err(got[-1], nlm) > 100 * tol


# ---------------------------------------------------------------------------------------------
# Full hybrid step: startup and cessation
# ---------------------------------------------------------------------------------------------
def _channel_pair(model, prec, lattice, nx, ny, nz, trace_full=True, **kw):
    desc = L.make_desc(lattice, nx, ny, nz, precision=prec[0], hist_storage=prec[1], model=model,
                       trace_coupling=L.LBVE_TRACE_FULL if trace_full else L.LBVE_TRACE_NONE, **kw)
    ch = L.Channel(desc)
    orc = oracle.Channel(lattice, nx, ny, nz, tau_lb=kw["tau_lb"], G_inf=kw["G_inf"], tau=kw["tau"],
                         gamma_c=kw["gamma_c"], g=kw["g"], C=kw["C"], B=kw["B"], trace_full=trace_full,
                         model=ORC_MODEL[model])
    return ch, orc


def _startup_cessation(ch, orc, on, off, tol, what, run_scale=False):
    """Compare at checkpoints through startup and cessation.  run_scale: after cessation, measure the
    error on the scale of the driven flow (the largest |field| seen up to cessation) instead of the
    decaying current field -- for FP32 populations, whose rounding (about 6e-8 of the peak velocity per
    step) stays fixed in absolute terms while the instantaneous model's flow decays without memory."""
    t = 0
    peak = {}
    for cp in [1, 2, 17, on // 2, on, on + 1, on + off // 3, on + off]:
        ch.step(cp - t)
        orc.step(cp - t)
        t = cp
        g, o = ch.fields(), orc.fields()
        if run_scale and t > on:
            for key in ("u", "sigma", "kappa"):
                e = np.max(np.abs(g[key] - o[key])) / max(np.max(np.abs(o[key])), peak[key])
                assert e <= tol, f"{what} step {t}: {key} error on the run's scale {e:.3e} > {tol:.1e}"
        else:
            compare(g, o, tol, f"{what} step {t}")
            for key in ("u", "sigma", "kappa"):
                peak[key] = max(peak.get(key, 0.0), float(np.max(np.abs(o[key]))))
        if t == on:
            ch.set_force((0, 0, 0))
            orc.set_force((0, 0, 0))


# The instantaneous stress is an explicit viscous stress G_inf tau_M D next to the BGK viscosity nu_N; the
# explicit step is stable for G_inf tau_M up to about 2.5 nu_N with LBVE_TRACE_NONE and about 1.7 nu_N with
# LBVE_TRACE_FULL (where its trace also drives the density source at once): 0.25 and 0.16 at tau_LB = 0.8.
# The coupled runs stay inside: G_inf tau = 0.1 and 0.15.
@pytest.mark.parametrize("prec", [ALL64, PLAIN, ALL32])
@pytest.mark.parametrize("trace_full,tau", [(True, 10.0), (False, 15.0)])
def test_inlm_channel_startup_cessation(prec, trace_full, tau):
    ch, orc = _channel_pair(INLM, prec, L.LBVE_D2Q9, 4, 32, 1, trace_full=trace_full, tau_lb=0.8, G_inf=0.01,
                            tau=tau, gamma_c=0.1, g=(2e-6, 0, 0), C=4, B=1)
    _startup_cessation(ch, orc, 1200, 600, TOL[prec], f"inlM trace_full={trace_full}", run_scale=prec == ALL32)
    ch.close()


def test_inlm_duct_vs_oracle():
    ch, orc = _channel_pair(INLM, ALL64, L.LBVE_D3Q19, 3, 9, 7, tau_lb=0.9, G_inf=0.01, tau=8.0, gamma_c=0.1,
                            g=(1e-5, 0, 0), C=4, B=1)
    _startup_cessation(ch, orc, 120, 60, TOL[ALL64], "inlM duct")
    ch.close()
    ch, orc = _channel_pair(INLM, PLAIN, L.LBVE_D3Q19, 3, 9, 7, tau_lb=0.9, G_inf=0.01, tau=8.0, gamma_c=0.1,
                            g=(1e-5, 0, 0), C=4, B=1)
    _startup_cessation(ch, orc, 120, 60, TOL[PLAIN], "inlM duct f32")
    ch.close()


@pytest.mark.parametrize("prec", [ALL64, PLAIN, ALL32])
@pytest.mark.parametrize("C,B", [(64, 4), (128, 1)])
def test_wm_channel_startup_cessation(prec, C, B):
    ch, orc = _channel_pair(WM, prec, L.LBVE_D2Q9, 4, 32, 1, tau_lb=0.8, G_inf=0.01, tau=200.0, gamma_c=0.1,
                            g=(1e-6, 0, 0), C=C, B=B)
    _startup_cessation(ch, orc, 1500, 700, TOL[prec], f"WM C={C} B={B}")
    ch.close()


def test_wm_duct_vs_oracle():
    ch, orc = _channel_pair(WM, PLAIN, L.LBVE_D3Q19, 3, 8, 6, tau_lb=0.9, G_inf=0.01, tau=40.0, gamma_c=0.1,
                            g=(2e-5, 0, 0), C=8, B=3)
    _startup_cessation(ch, orc, 90, 40, TOL[PLAIN], "WM duct")
    ch.close()


def test_variant_batches_vs_oracle():
    """Channels of different widths and parameters in one batch, for both variants."""
    for model, prec in ((INLM, ALL64), (WM, PLAIN)):
        specs = [(4, 8, 0.01, 10.0, 0.1, 2e-6), (3, 21, 0.005, 12.0, 0.2, 1e-6), (5, 14, 0.02, 5.0, 0.05, 3e-6)]
        descs, orcs = [], []
        for nx, ny, G, tau, gc, g in specs:
            descs.append(L.make_desc(L.LBVE_D2Q9, nx, ny, tau_lb=0.8, G_inf=G, tau=tau, gamma_c=gc, g=(g, 0, 0),
                                     C=16, B=3, precision=prec[0], hist_storage=prec[1], model=model))
            orcs.append(oracle.Channel(oracle.D2Q9, nx, ny, tau_lb=0.8, G_inf=G, tau=tau, gamma_c=gc, g=(g, 0, 0),
                                       C=16, B=3, model=ORC_MODEL[model]))
        ch = L.Channel(descs)
        for n in (5, 60):   # 60: graph replay
            ch.step(n)
            for o in orcs:
                o.step(n)
            f = ch.fields()
            for i, o in enumerate(orcs):
                compare(ch.channel_fields(i, f), o.fields(), TOL[prec], f"model {model} channel {i} t={ch.t}")
        ch.close()


@pytest.mark.parametrize("model", [INLM, WM])
def test_variant_checkpoint_resume_bitwise(model):
    kw = dict(nx=6, ny=14, tau_lb=0.8, G_inf=0.01, tau=10.0, gamma_c=0.1, g=(1e-5, 0, 0), C=8, B=3,
              precision=F64, hist_storage=F32, model=model)
    a = L.Channel(L.make_desc(**kw))
    a.step(37)
    img = L.lbve_checkpoint_save(a.h)
    a.step(50)
    ref = a.fields()
    b = L.Channel(L.make_desc(**kw))
    if model != INLM:   # same summation order of the history sum as a (no history sweep for the instantaneous model)
        S, _, mode = L.lbve_sweep_config(a.h)
        L.lbve_set_sweep_config(b.h, S, mode)
    L.lbve_checkpoint_restore(b.h, img)
    b.step(50)
    for k, v in ref.items():
        assert np.array_equal(b.fields()[k], v), k
    # an image of the other constitutive models is refused (the configuration fingerprint includes it)
    other = L.Channel(L.make_desc(**dict(kw, model=L.LBVE_MODEL_NLM)))
    with pytest.raises(L.LbveError) as e:
        L.lbve_checkpoint_restore(other.h, img)
    assert e.value.status == L.LBVE_EINVAL
    for ch in (a, b, other):
        ch.close()


def test_inlm_keeps_no_history():
    base = dict(nx=8, ny=64, C=128, B=4, precision=F64, hist_storage=F32)
    a = L.Channel(L.make_desc(**base, model=L.LBVE_MODEL_NLM))
    b = L.Channel(L.make_desc(**base, model=INLM))
    c = L.Channel(L.make_desc(**base, model=WM))
    ma, mb, mc = (L.lbve_memory_bytes(x.h) for x in (a, b, c))
    N = 8 * 64   # = Npad (a multiple of 128)
    L_pts = 512
    part = lambda h: 4 * L.lbve_sweep_config(h)[0] * 3 * N   # sweep partial sums (autotuned chunk count)
    # no X, no kappa of the 512 points, no partial sums
    assert mb == ma - 2 * 4 * 4 * L_pts * N - part(a.h)
    # Gamma(t') of every point and Gamma(t) of every node, in double
    assert mc - part(c.h) == ma - part(a.h) + 8 * L_pts * N + 8 * N
    for x in (a, b, c):
        x.close()
