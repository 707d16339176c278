"""Pins of the oracle's two constitutive variants of arXiv:1504.06123 (CPU only).

- The instantaneous nonlinear Maxwell model, Eq. (inlM) of Sec. IV, read as a stress / strain-rate law at
  time t with tau_M = (1/tau + |gammadot|/gamma_c)^-1 (the steady form of Eq. nlmax, Sec. II).
- The White-Metzner variant named in Sec. II: the second exponential of Eq. (nlmax) with the strain
  accumulated between t' and t in place of (t - t') |gammadot(t')|.

Neither test re-types the oracle's arithmetic: they use closed forms (nilpotent shear, planar
extension), the steady upper-convected Maxwell equation solved as a linear system, the defining
Laplace integral evaluated by quadrature with scipy's expm, brute-force per-step sums, the integral
model's own steady state, and the analytic steady channel profile.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle
from tests.refs import closed_schedule

RNG = np.random.default_rng(4242)


def _tau_M(K, tau, gc):
    D = K + K.T
    gd = math.sqrt(0.5 * float(np.sum(D * D)))
    return 1.0 / (1.0 / tau + (0.0 if math.isinf(gc) else gd / gc))


def _unpack(sig, d):
    if d == 2:
        return np.array([[sig[0], sig[2]], [sig[2], sig[1]]])
    return np.array([[sig[0], sig[3], sig[4]], [sig[3], sig[1], sig[5]], [sig[4], sig[5], sig[2]]])


# ---------------------------------------------------------------------------------------------
# Eq. (inlM): closed forms
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("gd", [1e-5, 2e-3, -7e-3, 0.05])
@pytest.mark.parametrize("gc", [0.1, math.inf])
@pytest.mark.parametrize("d,plane", [(2, (0, 1)), (3, (0, 1)), (3, (0, 2)), (3, (1, 2))])
def test_inlm_simple_shear_series_terminates(gd, gc, d, plane):
    """kappa = gd e_ab is nilpotent: d^(1) = D, d^(2) = 2 gd^2 e_aa, d^(n>2) = 0 (Sec. IV, Eq. inlM)."""
    G, tau = 0.01, 40.0
    a, b = plane
    K = np.zeros((d, d))
    K[a, b] = gd
    tM = 1.0 / (1.0 / tau + (0.0 if math.isinf(gc) else abs(gd) / gc))
    ref = np.zeros((d, d))
    ref[a, b] = ref[b, a] = G * tM * gd
    ref[a, a] = 2.0 * G * tM * tM * gd * gd
    S = _unpack(oracle.inlm(K, G, tau, gc), d)
    np.testing.assert_allclose(S, ref, rtol=1e-14, atol=0)
    assert S[b, b] == 0.0


@pytest.mark.parametrize("gc", [math.inf, 0.3])
@pytest.mark.parametrize("x", [0.05, 0.3, 0.6, 0.9])
def test_inlm_planar_extension_geometric_series(gc, x):
    """kappa = eps diag(1, -1): d^(n) = (2 kappa)^n, a geometric series with ratio 2 tau_M eps."""
    G, tau = 0.02, 50.0
    eps = x / (2.0 * tau)
    K = np.diag([eps, -eps])
    tM = _tau_M(K, tau, gc)
    r = 2.0 * tM * eps
    sig = oracle.inlm(K, G, tau, gc)
    np.testing.assert_allclose(sig, [G * r / (1.0 - r), G * (-r) / (1.0 + r), 0.0], rtol=1e-12, atol=1e-300)


def test_inlm_diverging_series_is_nan():
    """Beyond 2 tau_M eps = 1 the series of Eq. (inlM) diverges (no steady extensional stress)."""
    tau = 50.0
    for x in (1.0, 1.2, 3.0):
        K = np.diag([x / (2 * tau), -x / (2 * tau)])
        assert np.all(np.isnan(oracle.inlm(K, 0.01, tau, math.inf)))
    # shear thinning (finite gamma_c) keeps 2 tau_M eps = x / (1 + x tau/gamma_c ...) below 1 here
    K = np.diag([1.2 / (2 * tau), -1.2 / (2 * tau)])
    assert np.all(np.isfinite(oracle.inlm(K, 0.01, tau, 0.1)))


def _random_kappa(d, scale):
    K = RNG.normal(size=(d, d)) * scale
    return K


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("x", [1e-3, 0.05, 0.2])
def test_inlm_equals_steady_ucm_linear_solve(d, x):
    """Summed, Eq. (inlM) is the Neumann series of Z = tau_M (D + kappa Z + Z kappa^T): the steady
    upper-convected Maxwell stress with relaxation time tau_M.  Solved here as a d^2 x d^2 system."""
    G, tau, gc = 0.01, 30.0, 0.1
    for _ in range(4):
        K = _random_kappa(d, 1.0)
        K *= x / (30.0 * np.max(np.abs(np.linalg.eigvals(K + K.T))))
        tM = _tau_M(K, tau, gc)
        I = np.eye(d)
        # vec(kappa Z + Z kappa^T) = (I (x) kappa + kappa (x) I) vec(Z)  (row-major vec)
        Lop = np.kron(K, I) + np.kron(I, K)
        Z = np.linalg.solve(np.eye(d * d) - tM * Lop, tM * (K + K.T).reshape(-1)).reshape(d, d)
        S = _unpack(oracle.inlm(K, G, tau, gc), d)
        np.testing.assert_allclose(S, G * Z, rtol=1e-11, atol=1e-14 * np.max(np.abs(G * Z)))


@pytest.mark.parametrize("d", [2, 3])
def test_inlm_equals_laplace_integral(d):
    """Eq. (inlM) = (G/tau_M) int_0^inf e^{-s/tau_M} exp(kappa s) exp(kappa^T s) ds - G: the Finger tensor
    of a constant gradient, relaxed with the steady rate of Eq. (nlmax) (Sec. II, Sec. IV)."""
    G, tau, gc = 0.01, 20.0, 0.1
    K = _random_kappa(d, 1.0)
    K *= 0.15 / (20.0 * np.max(np.abs(K)))
    tM = _tau_M(K, tau, gc)

    def f(s):
        E = scipy.linalg.expm(K * s)
        return math.exp(-s / tM) * (E @ E.T)

    Y, _err = scipy.integrate.quad_vec(f, 0.0, 60.0 * tM, epsabs=1e-14, epsrel=1e-12)
    ref = G * (Y / tM - np.eye(d))
    S = _unpack(oracle.inlm(K, G, tau, gc), d)
    np.testing.assert_allclose(S, ref, rtol=1e-8, atol=1e-9 * np.max(np.abs(ref)))


@pytest.mark.parametrize("d", [2, 3])
def test_integral_model_relaxes_to_inlm(d):
    """Sec. IV: for a constant gradient the history integral (Eqs. gitt, nlmax) converges to Eq. (inlM).
    Uniform grid of 1000 steps (tau_M about 15): truncation e^{-60} and a trapezoid error O((1/tau_M)^2)."""
    G, tau, gc = 0.01, 20.0, 0.1
    K = _random_kappa(d, 1.0)
    K *= 0.1 / (20.0 * np.max(np.abs(K)))
    T = 1000
    seq = np.broadcast_to(K, (T, 1, d, d)).copy()
    sig = oracle.history_run(seq, T, 1, G, tau, gc, last_only=True)[0]
    ref = oracle.inlm(K, G, tau, gc)
    tM = _tau_M(K, tau, gc)
    err = np.max(np.abs(sig - ref)) / np.max(np.abs(ref))
    assert err < 0.5 / tM ** 2, err


# ---------------------------------------------------------------------------------------------
# Analytic steady channel of the instantaneous model (Sec. IV: "analytical solution" of the steady
# pressure-driven channel): eta_N gd + G tau_M(gd) gd = rho0 g |y|, a quadratic in gd.
# ---------------------------------------------------------------------------------------------
def test_inlm_steady_channel_analytic_profile():
    # G_inf tau = 0.12: inside the stability range of the explicit instantaneous stress (about 1.7 nu_N with
    # the density source, nu_N = 0.1 here)
    ny, tau, G, tau_lb, g, gc = 32, 12.0, 0.01, 0.8, 2e-5, 0.1
    ch = oracle.Channel(oracle.D2Q9, 1, ny, tau_lb=tau_lb, G_inf=G, tau=tau, gamma_c=gc, g=(g, 0, 0),
                        C=4, B=1, model=oracle.INLM)
    ch.step(6000)
    f = ch.fields()
    eta = (tau_lb - 0.5) / 3.0
    H = ny / 2.0

    def gdot(y):   # positive root of eta tau a^2 + (eta gc + G tau gc - S tau) a - S gc = 0
        S = g * abs(y)
        b = eta * gc + G * tau * gc - S * tau
        return (-b + math.sqrt(b * b + 4.0 * eta * tau * S * gc)) / (2.0 * eta * tau)

    y = np.arange(ny) - (ny - 1) / 2.0
    ref = np.array([scipy.integrate.quad(gdot, -H, -abs(yy))[0] for yy in y])   # u(wall) = 0
    u = f["u"][:, 0]
    # LB with the explicit stress: second order, O(1/H^2) of the profile (and the wall slip of BGK)
    assert np.max(np.abs(u - ref)) <= 2e-3 * ref.max()
    # local law at every node: the steady UCM stress of the node's own gradient (linear solve); in the
    # x-invariant channel it is sigma_xy = G tau_M kappa_xy, N1 = 2 G tau_M^2 kappa_xy^2 up to the tiny
    # compressible part of kappa
    I = np.eye(2)
    for n in range(ny):
        K = f["kappa"][n]
        tM = _tau_M(K, tau, gc)
        Lop = np.kron(K, I) + np.kron(I, K)
        Z = np.linalg.solve(np.eye(4) - tM * Lop, tM * (K + K.T).reshape(-1)).reshape(2, 2)
        np.testing.assert_allclose(_unpack(f["sigma"][n], 2), G * Z, rtol=1e-10, atol=1e-13 * G * abs(Z).max())
    kxy = f["kappa"][:, 0, 1]
    tM = 1.0 / (1.0 / tau + np.abs(kxy) / gc)
    np.testing.assert_allclose(f["sigma"][:, 2], G * tM * kxy, rtol=1e-6)
    np.testing.assert_allclose(f["n1"], 2 * G * tM ** 2 * kxy ** 2, rtol=1e-5, atol=1e-6 * f["n1"].max())


# ---------------------------------------------------------------------------------------------
# White-Metzner variant (Sec. II): accumulated strain in the second exponential
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("C", [8, 64])
def test_wm_equals_nlm_for_constant_gradient_on_a_uniform_grid(d, C):
    """With kappa constant from t = 0, the strain since t' >= 0 is (t - t') gammadot: both forms agree
    (points before t = 0 are at rest and contribute nothing)."""
    G, tau, gc = 0.02, 15.0, 0.1
    K = _random_kappa(d, 0.01)
    seq = np.broadcast_to(K, (90, 1, d, d)).copy()
    a = oracle.history_run(seq, C, 1, G, tau, gc, model=oracle.NLM)
    b = oracle.history_run(seq, C, 1, G, tau, gc, model=oracle.WM)
    np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-13 * np.max(np.abs(a)))


def test_wm_equals_nlm_in_the_ucm_limit():
    G, tau = 0.02, 15.0
    seq = RNG.normal(size=(60, 3, 2, 2)) * 0.01
    a = oracle.history_run(seq, 4, 3, G, tau, math.inf, model=oracle.NLM)
    b = oracle.history_run(seq, 4, 3, G, tau, math.inf, model=oracle.WM)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("C,B", [(8, 4), (16, 3), (64, 1)])
def test_wm_constant_shear_closed_form(C, B):
    """kappa = gd e_xy from t = 0 on the merged grid: E = 1 + gd (t - max(t',0)) e_xy exactly, the strain
    of every point is |gd| (t - max(t', 0)) (none before t = 0), kappa as stored (span average)."""
    gd, G, tau, gc, T = 2e-3, 0.01, 40.0, 0.1, 300
    K = np.zeros((T, 1, 2, 2))
    K[:, :, 0, 1] = gd
    sig = oracle.history_run(K, C, B, G, tau, gc, model=oracle.WM)
    for t in [0, 1, 2, 7, 50, 129, 200, T - 1]:
        sxy = sxx = 0.0
        for tp, span, _b, w in closed_schedule(C, B, t):
            m = min(1.0, max(0.0, (tp + span) / span)) if tp < 0 else 1.0
            s = t - tp
            strain = abs(gd) * (t - max(tp, 0))
            gm = G * math.exp(-s / tau - strain / gc)
            sxy += w * gm * m * gd
            sxx += w * gm * 2.0 * m * gd * gd * (t - max(tp, 0))
        assert sig[t, 0, 1] == 0.0
        np.testing.assert_allclose(sig[t, 0, 2], sxy, rtol=1e-13)
        np.testing.assert_allclose(sig[t, 0, 0], sxx, rtol=1e-12, atol=1e-30)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("C,B", [(4, 3), (3, 2), (5, 1), (4, 4)])
def test_wm_history_brute_force(d, C, B):
    """Raw per-step products and sums: E(t,t') = F(t-1)...F(t'), strain = sum_{q=t'}^{t-1} gammadot(q)."""
    T, nn = 40, 3
    G, tau, gc = 0.03, 9.0, 0.2
    kraw = RNG.normal(size=(T, nn, d, d)) * 0.02
    sig = oracle.history_run(kraw, C, B, G, tau, gc, model=oracle.WM)
    F = [[scipy.linalg.expm(kraw[s, n]) for n in range(nn)] for s in range(T)]
    rate = np.sqrt(0.5 * np.sum((kraw + np.swapaxes(kraw, -1, -2)) ** 2, axis=(-1, -2)))   # [T, nn]
    for t in [0, 1, 5, 17, 30, T - 1]:
        for n in range(nn):
            acc = np.zeros((d, d))
            for tp, span, _b, w in closed_schedule(C, B, t):
                s = t - tp
                kap = np.zeros((d, d))
                for q in range(tp, tp + span):
                    if 0 <= q <= t:
                        kap += kraw[q, n]
                kap /= span
                E = np.eye(d)
                strain = 0.0
                for q in range(t - 1, tp - 1, -1):
                    if q >= 0:
                        E = E @ F[q][n]
                        strain += rate[q, n]
                M = E @ kap @ E.T
                acc += w * G * math.exp(-s / tau - strain / gc) * (M + M.T)
            if d == 2:
                ref = [acc[0, 0], acc[1, 1], acc[0, 1]]
            else:
                ref = [acc[0, 0], acc[1, 1], acc[2, 2], acc[0, 1], acc[0, 2], acc[1, 2]]
            np.testing.assert_allclose(sig[t, n], ref, rtol=1e-11, atol=1e-17)


def test_wm_differs_from_nlm_under_oscillation():
    """Oscillatory shear: (t - t')|gammadot(t')| and the accumulated strain differ, so do the stresses."""
    T = 200
    K = np.zeros((T, 1, 2, 2))
    K[:, 0, 0, 1] = 5e-3 * np.sin(2 * np.pi * np.arange(T) / 50.0)
    a = oracle.history_run(K, 64, 4, 0.01, 40.0, 0.1, model=oracle.NLM)
    b = oracle.history_run(K, 64, 4, 0.01, 40.0, 0.1, model=oracle.WM)
    rel = np.max(np.abs(a[-1] - b[-1])) / np.max(np.abs(a[-1]))
    assert rel > 1e-2


def test_wm_steady_channel_equals_nlm():
    """In steady channel flow gammadot is constant in time, so the strain is (t - t') gammadot and the
    White-Metzner fluid settles on the nlM profile (Sec. II); the memory of the start-up is forgotten."""
    ny, tau, G, tau_lb, g, gc, C, B = 16, 30.0, 0.01, 0.8, 2e-5, 0.1, 64, 4
    kw = dict(tau_lb=tau_lb, G_inf=G, tau=tau, gamma_c=gc, g=(g, 0, 0), C=C, B=B)
    a = oracle.Channel(oracle.D2Q9, 1, ny, model=oracle.NLM, **kw)
    b = oracle.Channel(oracle.D2Q9, 1, ny, model=oracle.WM, **kw)
    a.step(4000)
    b.step(4000)
    fa, fb = a.fields(), b.fields()
    for key in ("u", "sigma"):
        err = np.max(np.abs(fa[key] - fb[key])) / np.max(np.abs(fa[key]))
        assert err < 1e-6, (key, err)
    # and during the start-up they differ (the strain then is not (t - t') gammadot(t'))
    a2 = oracle.Channel(oracle.D2Q9, 1, ny, model=oracle.NLM, **kw)
    b2 = oracle.Channel(oracle.D2Q9, 1, ny, model=oracle.WM, **kw)
    a2.step(60)
    b2.step(60)
    ua, ub = a2.fields()["u"], b2.fields()["u"]
    assert np.max(np.abs(ua - ub)) > 1e-6 * np.max(np.abs(ua))


def test_inlm_explicit_coupling_stability_range():
    """The instantaneous stress is an explicit viscous stress G_inf tau_M D on top of the BGK viscosity
    nu_N (Sec. III forcing).  Measured range at tau_LB = 0.8 (nu_N = 0.1), UCM limit: stable for
    G_inf tau = 0.2 and unstable (compressional mode at the walls) for 0.35 without the density source;
    with it, stable at 0.12 and unstable at 0.2.  Documents the limit the GPU tests stay inside."""
    def grows(G_tau, trace_full):
        ch = oracle.Channel(oracle.D2Q9, 1, 32, tau_lb=0.8, G_inf=0.01, tau=G_tau / 0.01, gamma_c=math.inf,
                            g=(1e-6, 0, 0), C=4, B=1, model=oracle.INLM, trace_full=trace_full)
        ch.step(1500)
        a = np.max(np.abs(ch.fields()["kappa"][:, 1, 1]))
        ch.step(1500)
        b = np.max(np.abs(ch.fields()["kappa"][:, 1, 1]))
        return not np.isfinite(b) or (b > 10 * a and b > 1e-12)

    assert not grows(0.2, False) and grows(0.35, False)
    assert not grows(0.12, True) and grows(0.2, True)
