"""GPU parity of the pressure-step boundary along x (Sec. III, the generalised periodic boundary) against
the FP64 oracle, through the C ABI: start-up with a pressure drop per period, cessation by
lbve_set_pressure_step(0), in 2D and 3D, every precision form, both constitutive variants, and batches
that mix pressure-driven and body-force-driven channels.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import lbve as L
from tests.test_gpu_parity import TOL, PLAIN, ALL32, ALL64, RED, compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = L.LBVE_F32, L.LBVE_F64
ORC_MODEL = {L.LBVE_MODEL_NLM: oracle.NLM, L.LBVE_MODEL_INLM: oracle.INLM, L.LBVE_MODEL_WM: oracle.WM}


def _pair(prec, lattice, nx, ny, nz, dp, model=L.LBVE_MODEL_NLM, **kw):
    ch = L.Channel(L.make_desc(lattice, nx, ny, nz, precision=prec[0], hist_storage=prec[1], model=model, dp=dp,
                               **kw))
    orc = oracle.Channel(lattice, nx, ny, nz, tau_lb=kw["tau_lb"], G_inf=kw["G_inf"], tau=kw["tau"],
                         gamma_c=kw["gamma_c"], g=kw.get("g", (0, 0, 0)), C=kw["C"], B=kw["B"],
                         model=ORC_MODEL[model], dp=dp)
    return ch, orc


def _run(ch, orc, on, off, tol, what, run_scale=False):
    """run_scale: after cessation, errors on the scale of the driven flow (largest |field| up to cessation)
    -- for FP32 populations, whose rounding stays fixed in absolute terms while the flow decays."""
    t = 0
    peak = {}
    for cp in [1, 2, 17, on // 2, on, on + 1, on + off // 2, on + off]:
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
        if t == on:   # cessation: no pressure drop (the seam keeps the mean density at rho0)
            ch.set_pressure_step(0.0)
            orc.set_pressure_step(0.0)


@pytest.mark.parametrize("prec", [ALL64, PLAIN, ALL32, RED])
@pytest.mark.parametrize("nx", [1, 5])
def test_pressure_driven_channel_vs_oracle(prec, nx):
    ch, orc = _pair(prec, L.LBVE_D2Q9, nx, 32, 1, 4e-6 * nx, tau_lb=0.8, G_inf=0.01, tau=200.0, gamma_c=0.1,
                    C=64, B=4)
    _run(ch, orc, 1200, 600, TOL[prec], f"nx={nx}", run_scale=prec == ALL32)
    ch.close()


def test_pressure_driven_duct_vs_oracle():
    ch, orc = _pair(PLAIN, L.LBVE_D3Q19, 3, 8, 7, 2e-5, tau_lb=0.9, G_inf=0.01, tau=40.0, gamma_c=0.1, C=8, B=3)
    _run(ch, orc, 80, 40, TOL[PLAIN], "duct")
    ch.close()


@pytest.mark.parametrize("model", [L.LBVE_MODEL_INLM, L.LBVE_MODEL_WM])
def test_pressure_driven_variants_vs_oracle(model):
    ch, orc = _pair(ALL64, L.LBVE_D2Q9, 2, 24, 1, 4e-6, model=model, tau_lb=0.8, G_inf=0.01, tau=10.0,
                    gamma_c=0.1, C=16, B=3)
    _run(ch, orc, 400, 200, TOL[ALL64], f"model {model}")
    ch.close()


def test_batch_mixing_pressure_and_body_force_vs_oracle():
    specs = [dict(nx=1, ny=10, dp=3e-6), dict(nx=4, ny=14, g=(2e-6, 0, 0)), dict(nx=3, ny=22, dp=6e-6)]
    kw = dict(tau_lb=0.8, G_inf=0.01, tau=30.0, gamma_c=0.1, C=16, B=3)
    descs, orcs = [], []
    for sp in specs:
        descs.append(L.make_desc(L.LBVE_D2Q9, sp["nx"], sp["ny"], precision=F64, hist_storage=F32,
                                 dp=sp.get("dp"), g=sp.get("g", (0, 0, 0)), **kw))
        orcs.append(oracle.Channel(oracle.D2Q9, sp["nx"], sp["ny"], g=sp.get("g", (0, 0, 0)), dp=sp.get("dp"),
                                   **kw))
    ch = L.Channel(descs)
    for n in (3, 70):   # 70: graph replay
        ch.step(n)
        for o in orcs:
            o.step(n)
        f = ch.fields()
        for i, o in enumerate(orcs):
            compare(ch.channel_fields(i, f), o.fields(), TOL[PLAIN], f"channel {i} t={ch.t}")
    # a new drop for the pressure-driven channels only
    ch.set_pressure_step(1e-6, channel=2)
    orcs[2].set_pressure_step(1e-6)
    with pytest.raises(L.LbveError) as e:
        ch.set_pressure_step(1e-6, channel=1)      # channel 1 is periodic: no pressure boundary
    assert e.value.status == L.LBVE_ESTATE
    ch.step(40)
    for o in orcs:
        o.step(40)
    f = ch.fields()
    for i, o in enumerate(orcs):
        compare(ch.channel_fields(i, f), o.fields(), TOL[PLAIN], f"channel {i} after the new drop")
    ch.close()


def test_pressure_boundary_density_gradient_and_equivalent_force():
    """The GPU channel carries the pressure drop per period as a linear density profile (3 dp / nx per
    spacing) and reaches the velocity of the equivalent body force g = dp / (rho0 nx)."""
    nx, ny, dp = 6, 16, 6e-6
    kw = dict(tau_lb=0.8, G_inf=0.0, tau=10.0, gamma_c=0.1, C=4, B=1, precision=F64, hist_storage=F64)
    a = L.Channel(L.make_desc(L.LBVE_D2Q9, nx, ny, dp=dp, **kw))
    b = L.Channel(L.make_desc(L.LBVE_D2Q9, nx, ny, g=(dp / nx, 0, 0), **kw))
    a.step(4000)
    b.step(4000)
    fa, fb = a.fields(), b.fields()
    rho = fa["rho"].reshape(ny, nx)
    np.testing.assert_allclose(rho[:, :-1] - rho[:, 1:], 3 * dp / nx, rtol=2e-3)
    err = np.max(np.abs(fa["u"] - fb["u"])) / np.max(np.abs(fb["u"]))
    assert err < 3e-5
    a.close()
    b.close()
