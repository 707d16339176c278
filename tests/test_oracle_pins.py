"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage of arXiv:1504.06123 it pins.  None of them re-types the oracle's own
formulas: they use closed forms, a library routine (scipy's expm), brute force over raw factor
products, an independent enumeration of the history grid, or invariants.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from tests.refs import closed_schedule

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------------------------------------
# Matrix exponential of the stored factors (Eq. eeval): special case of a library routine
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("scale", [1e-6, 1e-3, 0.3, 2.0])
def test_expm_matches_scipy(d, scale):
    for _ in range(20):
        K = RNG.normal(size=(d, d)) * scale
        ref = scipy.linalg.expm(K)
        got = oracle.expm(K)
        # a few ulp of exp(|K|) for the small generators of the method (|kappa| << 1); the 2x2 closed
        # form loses up to ~1e-12 relative to cancellation when |K| is of order 1
        rel = 2e-15 if scale < 1.0 else 1e-12
        assert np.max(np.abs(got - ref)) <= rel * np.exp(np.abs(K).sum()) * d * d


def test_expm_nilpotent_shear_exact():
    # simple shear generator: exp(a e_xy) = 1 + a e_xy exactly
    K = np.array([[0.0, 0.37], [0.0, 0.0]])
    assert np.array_equal(oracle.expm(K), np.array([[1.0, 0.37], [0.0, 1.0]]))


# ---------------------------------------------------------------------------------------------
# History grid (Sec. III quasi-logarithmic layout): oracle's simulated merges vs closed form
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("C,B", [(4, 1), (4, 2), (4, 3), (6, 4), (8, 5), (128, 8), (256, 1), (64, 4)])
def test_schedule_matches_closed_form(C, B):
    ts = list(range(0, 70)) + [255, 256, 257, 1000, 4097, 32767, 32768]
    for t in ts:
        tp, w = oracle.schedule(C, B, t)
        ref = closed_schedule(C, B, t)
        assert np.array_equal(tp, np.array([r[0] for r in ref], dtype=np.int64)), (t, tp)
        assert np.array_equal(w, np.array([r[3] for r in ref])), t


def test_schedule_span_and_count():
    # B blocks of C points: span C (2^B - 1) steps, between B*C-(B-1) and B*C points
    C, B = 16, 5
    for t in range(3 * (1 << B), 3 * (1 << B) + 64):
        tp, w = oracle.schedule(C, B, t)
        assert B * C - (B - 1) <= len(tp) <= B * C
        span = t - tp[-1]
        assert C * ((1 << B) - 1) - (1 << (B - 1)) <= span <= C * ((1 << B) - 1) + (1 << (B - 1))
        # trapezoid weights integrate a constant exactly over the span
        assert math.isclose(w.sum(), span, rel_tol=0, abs_tol=1e-12)


# ---------------------------------------------------------------------------------------------
# P1: E(t,t) = 1, so the point created now contributes -d_t'B = D(t) with weight 1/2
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
def test_first_step_is_half_D(d):
    K = RNG.normal(size=(1, 5, d, d)) * 1e-3
    G = 0.02
    sig = oracle.history_run(K, 8, 3, G, 100.0, 0.1)[0]
    for n in range(5):
        k = K[0, n]
        D = k + k.T
        gd = math.sqrt(0.5 * np.sum(D * D))
        # age 0: the modulus is G_inf regardless of gammadot (t - t' = 0)
        full = 0.5 * G * D
        assert gd > 0
        if d == 2:
            ref = [full[0, 0], full[1, 1], full[0, 1]]
        else:
            ref = [full[0, 0], full[1, 1], full[2, 2], full[0, 1], full[0, 2], full[1, 2]]
        np.testing.assert_allclose(sig[n], ref, rtol=1e-15, atol=0)


# ---------------------------------------------------------------------------------------------
# P2: constant simple shear from t = 0 -- discrete closed form (E = 1 + strain e_xy exactly)
# ---------------------------------------------------------------------------------------------
def shear_closed_form(gd, t, C, B, G, tau, gc):
    """sigma_xy, sigma_xx, sigma_yy of the history integral for kappa = gd e_xy from t = 0.

    For a point of span [t', t'+h) the stored kappa is the time average of kappa over the span,
    i.e. gd times the fraction m of the span at times >= 0; E = 1 + gd (t - max(t',0)) e_xy.
    -d_t'B = m gd (e_xy + e_yx + 2 strain e_xx);  gammadot of the point = m |gd|.
    """
    sxy = sxx = 0.0
    inv_gc = 0.0 if math.isinf(gc) else 1.0 / gc
    for tp, span, _b, w in closed_schedule(C, B, t):
        m = min(1.0, max(0.0, (tp + span) / span)) if tp < 0 else 1.0
        s = t - tp
        strain = gd * (t - max(tp, 0))
        g = G * math.exp(-s / tau - s * m * abs(gd) * inv_gc)
        sxy += w * g * m * gd
        sxx += w * g * 2.0 * m * gd * strain
    return sxy, sxx, 0.0


@pytest.mark.parametrize("C,B", [(64, 1), (8, 4), (16, 3), (128, 2)])
@pytest.mark.parametrize("gc", [0.1, math.inf])
def test_constant_shear_discrete_closed_form(C, B, gc):
    gd, G, tau, T = 2e-3, 0.01, 40.0, 300
    K = np.zeros((T, 1, 2, 2))
    K[:, :, 0, 1] = gd
    sig = oracle.history_run(K, C, B, G, tau, gc)
    for t in [0, 1, 2, 3, 7, 50, 129, 200, T - 1]:
        sxy, sxx, syy = shear_closed_form(gd, t, C, B, G, tau, gc)
        assert sig[t, 0, 1] == 0.0                       # sigma_yy stays exactly 0 (nilpotent kappa)
        np.testing.assert_allclose(sig[t, 0, 2], sxy, rtol=1e-13)
        np.testing.assert_allclose(sig[t, 0, 0], sxx, rtol=1e-12, atol=1e-30)


# ---------------------------------------------------------------------------------------------
# P3: continuum limit -- Maxwell model (Eq. maxwell) and its shear-thinning version
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("gc", [math.inf, 0.1])
def test_startup_shear_continuum_limit(gc):
    gd, G, tau = 1e-3, 0.01, 200.0
    T = 700
    K = np.zeros((T, 1, 2, 2))
    K[:, :, 0, 1] = gd
    sig = oracle.history_run(K, 1024, 1, G, tau, gc)
    inv_te = 1.0 / tau + (0.0 if math.isinf(gc) else gd / gc)
    te = 1.0 / inv_te
    for t in [50, 199, 400, T - 1]:
        ref_xy = G * te * gd * (1.0 - math.exp(-t / te))
        ref_xx = 2.0 * G * gd * gd * (te * te - te * (te + t) * math.exp(-t / te))
        # trapezoid error of a smooth exponential (1/(12 te) relative to te) plus the half-step jump
        # of the integrand at t' = 0 (weight 1 instead of 1/2): |err| <= G gd (e^{-t/te}/2 + 1/(10 te)) te
        tol_xy = G * gd * (0.5 * math.exp(-t / te) + 0.1 / te * te)
        assert abs(sig[t, 0, 2] - ref_xy) <= tol_xy
        assert abs(sig[t, 0, 2] - ref_xy) <= 1e-2 * ref_xy
        assert abs(sig[t, 0, 0] - ref_xx) <= 2e-2 * abs(ref_xx)


# ---------------------------------------------------------------------------------------------
# P4: brute force on tiny grids -- raw per-step factor products and span-averaged kappa
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("C,B", [(4, 3), (3, 2), (5, 1), (4, 4)])
def test_history_brute_force(d, C, B):
    T, nn = 40, 3
    G, tau, gc = 0.03, 9.0, 0.2
    kraw = RNG.normal(size=(T, nn, d, d)) * 0.02
    sig = oracle.history_run(kraw, C, B, G, tau, gc)
    F = [[scipy.linalg.expm(kraw[s, n]) for n in range(nn)] for s in range(T)]
    for t in [0, 1, 5, 17, 30, T - 1]:
        for n in range(nn):
            acc = np.zeros((d, d))
            for tp, span, _b, w in closed_schedule(C, B, t):
                s = t - tp
                # kappa of the point: average of kappa over its span (rest, kappa = 0, before t = 0)
                kap = np.zeros((d, d))
                for q in range(tp, tp + span):
                    if 0 <= q <= t:
                        kap += kraw[q, n]
                kap /= span
                E = np.eye(d)
                for q in range(t - 1, tp - 1, -1):   # E(t,t') = F(t-1) F(t-2) ... F(t')
                    if q >= 0:
                        E = E @ F[q][n]
                M = E @ kap @ E.T
                D = kap + kap.T
                gdk = math.sqrt(0.5 * np.sum(D * D))
                acc += w * G * math.exp(-s / tau - s * gdk / gc) * (M + M.T)
            if d == 2:
                ref = [acc[0, 0], acc[1, 1], acc[0, 1]]
            else:
                ref = [acc[0, 0], acc[1, 1], acc[2, 2], acc[0, 1], acc[0, 2], acc[1, 2]]
            np.testing.assert_allclose(sig[t, n], ref, rtol=1e-11, atol=1e-17)


# ---------------------------------------------------------------------------------------------
# Finite-difference kappa (Sec. III, second order): exact on quadratic fields, wall at half a node
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("ny", [2, 3, 8, 33])
def test_kappa_stencil_exact_on_quadratic(ny):
    nx = 5
    ch = oracle.Channel(oracle.D2Q9, nx, ny, tau_lb=0.8, G_inf=0.0, tau=1.0, gamma_c=1.0, C=4, B=1)
    H = ny / 2.0
    y = np.arange(ny) - (ny - 1) / 2.0
    x = np.arange(nx)
    X, Y = np.meshgrid(x, y)           # [ny, nx], node order x fastest
    a, b = 0.7, -0.3
    ux = a * (H * H - Y * Y)           # vanishes on both walls (y = +-H)
    uy = b * (H * H - Y * Y) * np.cos(2 * np.pi * X / nx)
    u = np.stack([ux.ravel(), uy.ravel()], axis=1)
    k = ch.kappa_of(u)
    dux_dy = (-2 * a * Y).ravel()
    tol = 1e-15 * H * H
    np.testing.assert_allclose(k[:, 0, 1], dux_dy, rtol=0, atol=tol)
    np.testing.assert_allclose(k[:, 0, 0], 0.0, atol=tol)
    np.testing.assert_allclose(k[:, 1, 1], (-2 * b * Y * np.cos(2 * np.pi * X / nx)).ravel(), atol=tol)
    # periodic x: central difference of cos = sin(2 pi/nx)/(2 pi/nx) times the exact derivative
    kx = 2 * np.pi / nx
    ref = (-b * (H * H - Y * Y) * np.sin(kx * X) * np.sin(kx)).ravel()
    np.testing.assert_allclose(k[:, 1, 0], ref, atol=tol)


# ---------------------------------------------------------------------------------------------
# P5: Newtonian Poiseuille (G_inf = 0) -- the steady BGK solution with half-way bounce-back
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("ny", [8, 15, 16])
@pytest.mark.parametrize("tau_lb", [0.8, 0.5 + math.sqrt(3.0) / 4.0, 1.3])
def test_newtonian_poiseuille(ny, tau_lb):
    """u(y) = g/(2 nu) (H^2 - y^2 + (16 L - 3)/12), L = (tau_LB - 1/2)^2: the known steady solution of
    BGK with half-way bounce-back (walls exactly at +-H for L = 3/16).  nu = c_s^2 (tau_LB - 1/2)."""
    g = 1e-6
    ch = oracle.Channel(oracle.D2Q9, 2, ny, tau_lb=tau_lb, G_inf=0.0, tau=10.0, gamma_c=0.1,
                        g=(g, 0, 0), C=4, B=1)
    nu = (tau_lb - 0.5) / 3.0
    H = ny / 2.0
    steps = int(40 * 4 * H * H / (math.pi ** 2 * nu)) + 200
    ch.step(steps)
    u = ch.fields()["u"][:, 0]
    y = np.arange(ny) - (ny - 1) / 2.0
    lam = (tau_lb - 0.5) ** 2
    ref = g / (2 * nu) * (H * H - y * y + (16 * lam - 3) / 12.0)
    u = u.reshape(ny, 2)
    np.testing.assert_allclose(u[:, 0], ref, rtol=1e-9)
    np.testing.assert_array_equal(u[:, 0], u[:, 1])      # x-invariance


def test_newtonian_startup_series():
    """Startup of Poiseuille flow: slowest Fourier mode decays with t_wall = 4 H^2/(pi^2 nu)."""
    g, ny, tau_lb = 1e-6, 32, 0.5 + math.sqrt(3.0) / 4.0
    nu = (tau_lb - 0.5) / 3.0
    H = ny / 2.0
    ch = oracle.Channel(oracle.D2Q9, 1, ny, tau_lb=tau_lb, G_inf=0.0, tau=10.0, gamma_c=0.1,
                        g=(g, 0, 0), C=4, B=1)
    y = np.arange(ny) - (ny - 1) / 2.0
    for t_target in [200, 800, 2000]:
        ch.step(t_target - ch.t)
        u = ch.fields()["u"][:, 0]
        t = ch.t - 0.5       # velocity of step t is the mean of before and after the force impulse
        ref = g / (2 * nu) * (H * H - y * y)
        for k in range(200):
            q = (2 * k + 1) * math.pi / (2 * H)
            ref -= 16 * g * H * H * (-1) ** k / (nu * math.pi ** 3 * (2 * k + 1) ** 3) * np.cos(q * y) * \
                math.exp(-q * q * nu * t)
        umax = g / (2 * nu) * H * H
        assert np.max(np.abs(u - ref)) <= 2e-3 * umax


# ---------------------------------------------------------------------------------------------
# P7: UCM steady state -- parabola with eta_eff = eta_N + G_inf W0 (Eq. nlM with gamma_c -> inf)
# ---------------------------------------------------------------------------------------------
def test_ucm_steady_parabola():
    ny, tau, G, tau_lb, g, C, B = 32, 50.0, 0.01, 0.8, 1e-6, 64, 4
    ch = oracle.Channel(oracle.D2Q9, 1, ny, tau_lb=tau_lb, G_inf=G, tau=tau, gamma_c=math.inf,
                        g=(g, 0, 0), C=C, B=B)
    ch.step(8000)
    f = ch.fields()
    u = f["u"][:, 0]
    tp, w = oracle.schedule(C, B, ch.t - 1)
    s = (ch.t - 1) - tp
    W0 = float(np.sum(w * np.exp(-s / tau)))
    nu_eff = (tau_lb - 0.5) / 3.0 + G * W0
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    # bulk curvature -g/nu_eff (sign and magnitude of the stress coupling, Eq. bodyforce)
    # (the wall stencil disturbs the profile by ~6e-4 next to the wall, decaying geometrically inward)
    np.testing.assert_allclose(d2[11:-11] * nu_eff / g, -1.0, rtol=2e-5)
    H = ny / 2.0
    y = np.arange(ny) - (ny - 1) / 2.0
    ref = g * (H * H - y * y) / (2 * nu_eff)
    assert np.max(np.abs(u - ref)) <= 1e-3 * ref.max()
    # normal stress difference N1 = sigma_xx - sigma_yy >= 0 in channel flow (Sec. IV)
    assert np.all(f["n1"] >= 0)


# ---------------------------------------------------------------------------------------------
# P6: steady nlM channel -- local force balance sigma_xy + eta_N D_xy = -rho0 g y
# ---------------------------------------------------------------------------------------------
def test_nlm_steady_force_balance():
    ny, tau, G, tau_lb, g, gc, C, B = 32, 50.0, 0.01, 0.8, 2e-5, 0.1, 64, 4
    ch = oracle.Channel(oracle.D2Q9, 1, ny, tau_lb=tau_lb, G_inf=G, tau=tau, gamma_c=gc,
                        g=(g, 0, 0), C=C, B=B)
    ch.step(8000)
    f = ch.fields()
    eta_N = (tau_lb - 0.5) / 3.0
    y = np.arange(ny) - (ny - 1) / 2.0
    H = ny / 2.0
    total = f["sigma"][:, 2] + eta_N * (f["kappa"][:, 0, 1] + f["kappa"][:, 1, 0])
    err = (total + g * y) / (g * H)
    assert np.max(np.abs(err)) < 1e-2
    # the stress enters the momentum flux through the second moment of F_i, a discretisation of
    # div sigma that is second order: O(1/H^2) of the local stress in the bulk
    assert np.max(np.abs(err[4:-4])) < 5e-4
    # shear thinning: the structural viscosity sigma_xy/gammadot falls with the local shear rate
    gd = np.abs(f["kappa"][:, 0, 1])
    visc = np.abs(f["sigma"][:, 2]) / np.maximum(gd, 1e-300)
    order = np.argsort(gd[: ny // 2])
    assert np.all(np.diff(visc[: ny // 2][order]) < 0)


# ---------------------------------------------------------------------------------------------
# P9: mass invariant of the density source (Sec. III): sum n(t) - sum delta rho(t-1) is constant
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("lattice,nz", [(oracle.D2Q9, 1), (oracle.D3Q19, 6)])
def test_mass_invariant(lattice, nz):
    nx, ny = 4, 6
    rho0 = 1.0 + RNG.uniform(-1e-3, 1e-3, size=nx * ny * nz)
    ch = oracle.Channel(lattice, nx, ny, nz, tau_lb=0.9, G_inf=0.01, tau=30.0, gamma_c=0.1,
                        g=(1e-4, 0, 0), C=8, B=3, rho_init=rho0)
    m0 = None
    for _ in range(30):
        ch.step(3)
        sn, sd = ch.mass()
        if m0 is None:
            m0 = sn - sd
        assert abs((sn - sd) - m0) <= 1e-13 * abs(m0)
    # without the density source the populations alone conserve mass
    ch2 = oracle.Channel(lattice, nx, ny, nz, tau_lb=0.9, G_inf=0.01, tau=30.0, gamma_c=0.1,
                         g=(1e-4, 0, 0), C=8, B=3, rho_init=rho0, trace_full=False)
    ch2.step(1)
    s0 = ch2.mass()[0]
    ch2.step(40)
    assert abs(ch2.mass()[0] - s0) <= 1e-13 * s0


# ---------------------------------------------------------------------------------------------
# P10: x-invariance without noise (bitwise), symmetric stress; P11 node positions
# ---------------------------------------------------------------------------------------------
def test_translation_invariance_bitwise():
    ch = oracle.Channel(oracle.D2Q9, 4, 10, tau_lb=0.8, G_inf=0.01, tau=50.0, gamma_c=0.1,
                        g=(1e-5, 0, 0), C=8, B=3)
    ch.step(120)
    f = ch.fields()
    u = f["u"].reshape(10, 4, 2)
    s = f["sigma"].reshape(10, 4, 3)
    for x in range(1, 4):
        assert np.array_equal(u[:, x], u[:, 0])
        assert np.array_equal(s[:, x], s[:, 0])
    # channel symmetry y -> -y: u_x even (to rounding), sigma_xy odd
    np.testing.assert_allclose(u[::-1, 0, 0], u[:, 0, 0], rtol=1e-12)
    np.testing.assert_allclose(s[::-1, 0, 2], -s[:, 0, 2], rtol=1e-10, atol=1e-22)


def test_duct_symmetry_3d():
    n = 6
    ch = oracle.Channel(oracle.D3Q19, 2, n, n, tau_lb=0.9, G_inf=0.01, tau=30.0, gamma_c=0.1,
                        g=(1e-5, 0, 0), C=8, B=2)
    ch.step(60)
    f = ch.fields()
    u = f["u"].reshape(n, n, 2, 3)          # [z][y][x][comp]
    # square duct: swapping y and z leaves u_x unchanged
    np.testing.assert_allclose(u[:, :, 0, 0], u[:, :, 0, 0].T, rtol=1e-11)
    assert np.all(u[:, :, 0, 0] > 0)
    # transverse (secondary) velocities map onto each other under the y <-> z swap and are odd under
    # y -> -y, up to the rounding of velocities taken from populations of order 0.05
    atol = 1e-11 * np.max(np.abs(u[..., 0]))
    np.testing.assert_allclose(u[:, :, 0, 1], u[:, :, 0, 2].T, rtol=0, atol=atol)
    np.testing.assert_allclose(u[:, ::-1, 0, 1], -u[:, :, 0, 1], rtol=0, atol=atol)


# ---------------------------------------------------------------------------------------------
# Collision with forcing (Sec. III, Eq. bodyforce and Eq. hydrofields): post-collision moments.
# Lattice isotropy (sum w c_a c_b = c_s^2 delta, fourth moment c_s^4 (dd + dd + dd)) turns the
# forcing into these moment relations; they hold for D2Q9 and D3Q19 alike.
# ---------------------------------------------------------------------------------------------
def _velocities(lattice):
    if lattice == oracle.D2Q9:
        return np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
    c = [[0, 0, 0]]
    for a in range(3):
        for s in (1, -1):
            v = [0, 0, 0]; v[a] = s; c.append(v)
    for a in range(3):
        for b in range(a + 1, 3):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0]; v[a] = sa; v[b] = sb; c.append(v)
    return np.array(c, float)


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q19])
@pytest.mark.parametrize("trace_full", [True, False])
def test_collision_moments(lattice, trace_full):
    d = 2 if lattice == oracle.D2Q9 else 3
    nz = 1 if d == 2 else 3
    tau_lb, rho0 = 0.7, 1.0
    g = np.array([3e-4, -2e-4, 1e-4])[:3]
    ch = oracle.Channel(lattice, 3, 3, nz, tau_lb=tau_lb, G_inf=0.01, tau=10.0, gamma_c=0.1,
                        g=g, C=4, B=1, trace_full=trace_full)
    c = _velocities(lattice)
    cs2 = 1.0 / 3.0
    for _ in range(10):
        n = RNG.uniform(0.02, 0.4, size=lattice)
        nsig = 3 if d == 2 else 6
        sig = RNG.normal(size=nsig) * 1e-3
        tr_prev = RNG.normal() * 1e-3
        post, rho, u = oracle.collide(ch, n, sig, tr_prev)
        S = np.zeros((d, d))
        if d == 2:
            S[0, 0], S[1, 1], S[0, 1] = sig; S[1, 0] = S[0, 1]
        else:
            S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2] = sig
            S[1, 0], S[2, 0], S[2, 1] = S[0, 1], S[0, 2], S[1, 2]
        tr = np.trace(S)
        ddr = -(tr - tr_prev) / (d * cs2) if trace_full else 0.0
        f = rho0 * g[:d]
        rho_raw = n.sum()
        J = c[:, :d].T @ n
        Pi = (c[:, :d].T * n) @ c[:, :d]
        assert rho == pytest.approx(rho_raw + 0.5 * ddr, rel=1e-15)
        np.testing.assert_allclose(u[:d], (J + 0.5 * f) / rho, rtol=1e-13)
        u = u[:d]
        Sb = S - tr / d * np.eye(d)
        # zeroth and first moments
        assert post.sum() == pytest.approx(rho_raw + ddr, rel=1e-14)
        np.testing.assert_allclose(c[:, :d].T @ post, J + f, rtol=1e-13, atol=1e-15)
        # second moment
        Pi_post = (c[:, :d].T * post) @ c[:, :d]
        ref = ((1 - 1 / tau_lb) * Pi + (rho * cs2 * np.eye(d) + rho * np.outer(u, u)) / tau_lb
               - Sb / tau_lb
               + (1 - 0.5 / tau_lb) * (ddr * cs2 * np.eye(d) - ddr * np.outer(u, u)
                                       + np.outer(u, f) + np.outer(f, u)))
        np.testing.assert_allclose(Pi_post, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("gd", [1e-3, 1e-2])
def test_dynamic_yield_stress(gd):
    """Sec. IV: at tau -> infinity the model's shear stress under steady shear tends to G_inf gamma_c at any
    rate (the yield stress of the glass).  On a uniform history grid the trapezoidal sum is a geometric
    series: sigma_xy = G_inf gd sum_k w_k exp(-a k) = G_inf gamma_c (a/2) coth(a/2), a = gd/gamma_c, up to
    the truncation exp(-a T) of the retained span."""
    G, gc = 0.01, 0.1
    a = gd / gc
    T = int(60 / a)
    K = np.zeros((T, 1, 2, 2))
    K[:, 0, 0, 1] = gd
    sig = oracle.history_run(K, T + 8, 1, G, 1e15, gc, last_only=True)[0]
    exact = G * gc * (a / 2) / np.tanh(a / 2)
    assert sig[2] == pytest.approx(exact, rel=1e-10)
    assert abs(sig[2] / (G * gc) - 1.0) < a * a / 12 * 1.01 + 1e-12      # -> the yield stress G_inf gamma_c
    assert sig[1] == 0.0


def _duct_series(ny, nz, g, nu, terms=400):
    """Steady Newtonian flow in a rectangular duct of width 2a (y) and 2b (z) under a body force g: the
    textbook Fourier series u = 16 g a^2 / (nu pi^3) sum_{n odd} (-1)^((n-1)/2) n^-3
    [1 - cosh(n pi z / 2a) / cosh(n pi b / 2a)] cos(n pi y / 2a); nodes at j - (n-1)/2, walls half a node
    outside.  Returns u[z][y]."""
    a, b = ny / 2, nz / 2
    y = np.arange(ny) - (ny - 1) / 2
    z = np.arange(nz) - (nz - 1) / 2
    Y, Z = np.meshgrid(y, z, indexing="ij")
    u = np.zeros_like(Y)
    for n in range(1, 2 * terms, 2):
        x, X = n * np.pi * np.abs(Z) / (2 * a), n * np.pi * b / (2 * a)
        ratio = np.exp(x - X) * (1 + np.exp(-2 * x)) / (1 + np.exp(-2 * X))     # cosh(x) / cosh(X), |x| <= X
        u += (-1) ** ((n - 1) // 2) / n ** 3 * (1 - ratio) * np.cos(n * np.pi * Y / (2 * a))
    return (16 * g * a * a / (nu * np.pi ** 3) * u).T


def test_newtonian_duct_series_second_order():
    """D3Q19 square duct (walls in y and z), G_inf = 0: the steady velocity converges to the duct series at
    second order in the lattice spacing (half-way bounce-back at Lambda = 3/16)."""
    tau_lb = 0.5 + np.sqrt(3.0 / 16.0)
    nu = (tau_lb - 0.5) / 3.0
    g = 1e-6
    err = {}
    for n in (12, 24):
        ch = oracle.Channel(oracle.D3Q19, 1, n, n, tau_lb=tau_lb, G_inf=0.0, tau=10.0, gamma_c=0.1, g=(g, 0, 0),
                            C=4, B=1)
        ch.step(int(16 * n * n / (np.pi ** 2 * nu)))
        u = ch.fields()["u"][:, 0].reshape(n, n)      # node x + nx (y + ny z): [z][y]
        ch.close()
        ex = _duct_series(n, n, g, nu)
        err[n] = np.max(np.abs(u - ex)) / np.max(np.abs(ex))
    assert err[24] < 5e-4
    assert 3.5 < err[12] / err[24] < 4.5                 # second order: (24/12)^2


@pytest.mark.parametrize("a,b", [(0, 1), (0, 2), (1, 2), (2, 0), (1, 0)])
def test_constant_shear_3d_planes(a, b):
    """P2 in 3D: kappa = gd e_ab (velocity component a varying along b) is nilpotent, so E = 1 + strain e_ab
    exactly and the 2D closed form holds in that plane: sigma_ab = the shear value, sigma_aa = the normal
    value, every other packed component (xx, yy, zz, xy, xz, yz) exactly 0."""
    gd, G, tau, gc, T, C, B = 2e-3, 0.01, 40.0, 0.1, 200, 16, 3
    K = np.zeros((T, 1, 3, 3))
    K[:, :, a, b] = gd
    sig = oracle.history_run(K, C, B, G, tau, gc)
    pack = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    for t in (0, 5, 77, T - 1):
        sxy, sxx, _ = shear_closed_form(gd, t, C, B, G, tau, gc)
        for i in range(6):
            if i == pack[(a, b)]:
                np.testing.assert_allclose(sig[t, 0, i], sxy, rtol=1e-13)
            elif i == pack[(a, a)]:
                np.testing.assert_allclose(sig[t, 0, i], sxx, rtol=1e-12, atol=1e-30)
            else:
                assert sig[t, 0, i] == 0.0, (t, i)
