"""Pins of the oracle's pressure-step boundary along x (CPU only).

Sec. III: the paper drives its channels with the generalised periodic boundary of Kim & Pitsch, which fixes a
constant pressure step between the inlet and the outlet of the periodic lattice.  Reading: the periodic
images outside the lattice are ghost nodes carrying the imaged node's non-equilibrium populations on an
equilibrium at the ghost's density; the ghosts sit on the linear pressure profile of the period, so the
pressure drops by dp over nx spacings around the mean rho0.

The pins use the known steady Poiseuille solution of BGK with half-way bounce-back, the linear density
profile the boundary must impose, the equivalence with a uniform body force g = dp / (rho0 nx) (Sec. IV,
Delta p / L = rho0 g), and the reduction to the plain periodic lattice.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("nx", [1, 2, 6])
@pytest.mark.parametrize("tau_lb", [0.8, 0.5 + math.sqrt(3.0) / 4.0])
def test_pressure_driven_newtonian_poiseuille(nx, tau_lb):
    """u(y) = G/(2 nu) (H^2 - y^2 + (16 L - 3)/12) with the pressure gradient G = dp / nx per spacing,
    L = (tau_LB - 1/2)^2 (the BGK bounce-back slip); the density varies along x by O(3 dp), which
    changes u = j / rho by the same relative amount."""
    ny, dp = 16, 1e-6
    ch = oracle.Channel(oracle.D2Q9, nx, ny, tau_lb=tau_lb, G_inf=0.0, tau=10.0, gamma_c=0.1, C=4, B=1, dp=dp)
    nu = (tau_lb - 0.5) / 3.0
    H = ny / 2.0
    ch.step(int(40 * 4 * H * H / (math.pi ** 2 * nu)) + 200)
    f = ch.fields()
    u = f["u"][:, 0].reshape(ny, nx)
    y = np.arange(ny) - (ny - 1) / 2.0
    lam = (tau_lb - 0.5) ** 2
    ref = (dp / nx) / (2 * nu) * (H * H - y * y + (16 * lam - 3) / 12.0)
    for x in range(nx):
        np.testing.assert_allclose(u[:, x], ref, rtol=1e-5)
    assert np.max(np.abs(f["u"][:, 1])) < 1e-5 * ref.max()     # cross flow only at the O(3 dp) compressible level


@pytest.mark.parametrize("nx", [2, 5, 9])
def test_pressure_step_imposes_the_linear_density_profile(nx):
    """Steady state: rho(x) drops by 3 dp / nx per spacing (pressure c_s^2 rho drops by dp per period),
    the same in every row, around the mean rho0."""
    ny, dp = 12, 2e-6
    ch = oracle.Channel(oracle.D2Q9, nx, ny, tau_lb=0.9, G_inf=0.0, tau=10.0, gamma_c=0.1, C=4, B=1, dp=dp)
    ch.step(4000)
    rho = ch.fields()["rho"].reshape(ny, nx)
    slope = rho[:, :-1] - rho[:, 1:]
    np.testing.assert_allclose(slope, 3 * dp / nx, rtol=2e-3)
    assert abs(rho.mean() - 1.0) < 1e-3 * 3 * dp


def test_pressure_step_equals_body_force_for_the_nlm_fluid():
    """Sec. IV: Delta p / L = rho0 g.  The viscoelastic nlM channel driven by a pressure step reaches the
    profile of the same channel driven by g = dp / (rho0 nx), up to the compressible effect of the pressure
    gradient: rho varies along x by 3 dp, so u = j / rho does too, giving kappa_xx ~ 3 dp u / nx, which
    enters the normal stresses (both relative errors are proportional to dp)."""
    nx, ny, dp = 3, 24, 3e-6
    kw = dict(tau_lb=0.8, G_inf=0.01, tau=40.0, gamma_c=0.1, C=32, B=4)
    a = oracle.Channel(oracle.D2Q9, nx, ny, dp=dp, **kw)
    b = oracle.Channel(oracle.D2Q9, nx, ny, g=(dp / nx, 0, 0), **kw)
    a.step(5000)
    b.step(5000)
    fa, fb = a.fields(), b.fields()
    for key, tol in (("u", 1e-4), ("sigma", 3e-4)):
        err = np.max(np.abs(fa[key] - fb[key])) / np.max(np.abs(fb[key]))
        assert err < tol, (key, err)
    # start-up: the pressure gradient is set up by sound waves from the seam, so the pressure-driven flow
    # lags the body-force flow at first (5 % after 20 steps) and joins it as the waves damp out
    errs = []
    c = oracle.Channel(oracle.D2Q9, nx, ny, dp=dp, **kw)
    d = oracle.Channel(oracle.D2Q9, nx, ny, g=(dp / nx, 0, 0), **kw)
    for n in (20, 130, 250):
        c.step(n)
        d.step(n)
        errs.append(np.max(np.abs(c.fields()["u"] - d.fields()["u"])) / np.max(np.abs(d.fields()["u"])))
    assert errs[0] < 0.1 and errs[1] < 1e-2 and errs[2] < 1e-3
    assert errs[0] > errs[1] > errs[2]


def test_pressure_boundary_off_is_the_periodic_lattice_bitwise():
    kw = dict(tau_lb=0.8, G_inf=0.01, tau=40.0, gamma_c=0.1, g=(2e-6, 0, 0), C=8, B=2)
    rho = 1.0 + 1e-6 * np.sin(np.arange(4 * 10))
    a = oracle.Channel(oracle.D2Q9, 4, 10, rho_init=rho, **kw)
    b = oracle.Channel(oracle.D2Q9, 4, 10, rho_init=rho, **kw)
    b.set_pressure_step(1e-5)
    b.set_pressure_step(None)
    a.step(60)
    b.step(60)
    for k, v in a.fields().items():
        assert np.array_equal(v, b.fields()[k]), k


def test_zero_step_pins_the_mean_density():
    """dp = 0 keeps the seam at rho0: a perturbed column relaxes to the mean rho0 (the boundary sets the
    absolute pressure level), while the periodic lattice keeps its initial mass."""
    nx, ny = 3, 8
    rho = np.full(nx * ny, 1.0 + 4e-5)
    a = oracle.Channel(oracle.D2Q9, nx, ny, tau_lb=0.8, G_inf=0.0, tau=10.0, gamma_c=0.1, C=4, B=1,
                       rho_init=rho, dp=0.0)
    b = oracle.Channel(oracle.D2Q9, nx, ny, tau_lb=0.8, G_inf=0.0, tau=10.0, gamma_c=0.1, C=4, B=1,
                       rho_init=rho)
    a.step(3000)
    b.step(3000)
    assert abs(a.fields()["rho"].mean() - 1.0) < 1e-8
    assert abs(b.fields()["rho"].mean() - (1.0 + 4e-5)) < 1e-12


def test_pressure_driven_duct_matches_body_force():
    """D3Q19 square duct: the pressure step along x drives the same flow as the equivalent body force."""
    nx, n, dp = 2, 8, 4e-6
    kw = dict(tau_lb=0.9, G_inf=0.01, tau=20.0, gamma_c=0.1, C=8, B=3)
    a = oracle.Channel(oracle.D3Q19, nx, n, n, dp=dp, **kw)
    b = oracle.Channel(oracle.D3Q19, nx, n, n, g=(dp / nx, 0, 0), **kw)
    a.step(700)
    b.step(700)
    err = np.max(np.abs(a.fields()["u"] - b.fields()["u"])) / np.max(np.abs(b.fields()["u"]))
    assert err < 1e-4
