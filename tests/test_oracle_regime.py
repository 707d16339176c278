"""The oracle against the paper's statements about startup and cessation transients (Sec. IV).

The figures' data are stripped, but the text states properties of the curves; each test below checks one
of them on small oracle channels in the paper's regime (t_wall/tau_0, theta = tau/tau_0, gamma_c = 1/10,
pressure drop over one width equal to G_inf), probed at y/H = 0.51 by linear interpolation:
  - narrow channels (t_wall << tau_0): the startup velocity overshoots its steady value; wide channels
    (t_wall >~ tau_0): it rises monotonically;
  - after cessation the velocity decays through zero (counter-flow), ahead of the shear stress, which
    turns negative too;
  - sigma_xx - sigma_yy > 0 at all times; after cessation it decays monotonically; after startup it
    overshoots in wide channels, much less in narrow ones;
  - Newtonian and linear viscoelastic (UCM) fluids: startup u(t) and cessation u_ss - u(t) coincide; the
    nonlinear model breaks that symmetry;
  - the UCM overshoots and oscillates after startup, shear thinning removes the oscillations (Fig.
    compModels); a larger theta lowers the steady velocity (Fig. figtau).
The lattice parameters are computed here from the paper's definitions, independently of the CUDA
package: eta_inf = G_inf tau_0 = rho0 nu_N (BGK viscosity), t_wall = 4 H^2 rho / (pi^2 G_inf tau_0).
"""
import math

import numpy as np
import pytest

import oracle

TAU_LB = 0.9
NU = (TAU_LB - 0.5) / 3.0


def _params(ratio, theta, ny):
    H = ny / 2.0
    t_wall = 4.0 * H * H / (math.pi ** 2 * NU)       # with G_inf tau_0 = nu (rho0 = 1)
    tau0 = t_wall / ratio
    G = NU / tau0
    return dict(H=H, t_wall=t_wall, tau0=tau0, G=G, tau=theta * tau0, g=G / (2.0 * H))


def _run(ratio, theta, ny, t_start, t_stop, every, *, gamma_c=0.1, newtonian=False, C=32, B=10):
    p = _params(ratio, theta, ny)
    ch = oracle.Channel(oracle.D2Q9, 1, ny, tau_lb=TAU_LB, G_inf=0.0 if newtonian else p["G"], tau=p["tau"],
                        gamma_c=gamma_c, g=(p["g"], 0, 0), C=C, B=B)
    y = 0.51 * p["H"] - 0.5
    j0 = int(math.floor(y))
    w = y - j0
    rows = []
    for phase, n in (("start", t_start), ("stop", t_stop)):
        if phase == "stop":
            ch.set_force((0, 0, 0))
        for _ in range(n // every):
            ch.step(every)
            f = ch.fields()
            pr = lambda a: (1 - w) * a[j0] + w * a[j0 + 1]
            rows.append((ch.t, pr(f["u"][:, 0]), pr(f["sigma"][:, 2]), pr(f["n1"])))
    ch.close()
    r = np.array(rows)
    k = t_start // every
    return p, r[:k], r[k:]


@pytest.fixture(scope="module")
def narrow():      # t_wall/tau_0 = 0.1, theta = 10: 8 nodes across, tau_0 = 486 steps
    p = _params(0.1, 10.0, 8)
    T = int(3 * p["tau"])
    return _run(0.1, 10.0, 8, T, T, T // 300)


@pytest.fixture(scope="module")
def wide():        # t_wall/tau_0 = 8, theta = 10: 24 nodes across, tau_0 = 55 steps
    p = _params(8.0, 10.0, 24)
    T = int(10 * p["tau"])
    return _run(8.0, 10.0, 24, T, T, 8)


def test_startup_overshoot_only_in_narrow_channels(narrow, wide):
    for (p, st, _), overshoot in ((narrow, True), (wide, False)):
        u = st[:, 1] / st[-1, 1]
        # reached the steady state: the last tenth of the startup changes u by < 1e-3
        assert abs(st[-1, 1] - st[int(0.9 * len(st)), 1]) < 1e-3 * st[-1, 1]
        if overshoot:
            # Newtonian-like parabola first, then the slower non-Newtonian steady state
            assert u.max() > 1.1
            assert st[np.argmax(u), 0] < p["tau0"]
        else:
            assert u.max() < 1.0 + 1e-3
            assert np.all(np.diff(st[:, 1]) > -1e-6 * st[-1, 1])   # monotonic rise


def test_cessation_counterflow_velocity_leads_stress(narrow, wide):
    for p, st, sp in (narrow, wide):
        u, s = sp[:, 1], sp[:, 2]
        assert u.min() < -0.01 * st[-1, 1]            # the fluid flows backwards
        assert s.min() < -0.01 * st[-1, 2]            # and the stress turns negative
        tu = sp[np.argmax(u < 0), 0]
        ts = sp[np.argmax(s < 0), 0]
        assert tu < ts                                # velocity first: the phase shift of Fig. QT


def test_normal_stress_difference_positive_and_decays_monotonically(narrow, wide):
    for p, st, sp in (narrow, wide):
        n1 = np.concatenate([st[:, 3], sp[:, 3]])
        assert np.all(n1[1:] > 0)
        n1ss = st[-1, 3]
        # after cessation: monotonic decay (apart from wiggles below 1 % of the steady value once the
        # counter-flow re-shears the fluid)
        d = sp[:, 3] / n1ss
        assert np.max(d - np.minimum.accumulate(d)) < 0.01
        big = d > 0.05
        assert np.all(np.diff(d[big]) < 0)


def test_normal_stress_overshoot_grows_with_width(narrow, wide):
    on = (narrow[1][:, 3] / narrow[1][-1, 3]).max()
    ow = (wide[1][:, 3] / wide[1][-1, 3]).max()
    assert ow > 1.15
    assert on < 1.1
    assert ow > on + 0.1


@pytest.mark.parametrize("kind", ["newtonian", "ucm", "nlm"])
def test_startup_cessation_symmetry(kind):
    theta = 2.0 if kind == "ucm" else 10.0
    p = _params(1.0, theta, 12)
    T = int(12 * p["tau"]) if kind == "ucm" else int(6 * p["tau"])
    gamma_c = math.inf if kind == "ucm" else 0.1
    _, st, sp = _run(1.0, theta, 12, T, T, 8, gamma_c=gamma_c, newtonian=(kind == "newtonian"))
    uss = st[-1, 1]
    amp = np.abs(np.concatenate([st[:, 1], sp[:, 1]])).max()
    err = np.max(np.abs(st[:, 1] + sp[:, 1] - uss)) / amp
    if kind == "newtonian":
        assert err < 1e-12          # linear and x-invariant: exact up to rounding
    elif kind == "ucm":
        assert err < 1e-3           # linear in (u, sigma_xy); only O(u) nonlinearities of the scheme
    else:
        assert err > 0.05           # shear thinning breaks it


@pytest.mark.parametrize("ratio,ny", [(0.1, 8), (1.0, 12)])
def test_ucm_oscillates_and_shear_thinning_damps_it(ratio, ny):
    # Sec. IV (Fig. compModels): the linear-viscoelastic UCM (gamma_c -> infinity) overshoots and
    # oscillates after startup in narrow and intermediate channels; with shear thinning the oscillations
    # disappear (the nlM velocity, once past its maximum, does not dip below its steady value)
    p = _params(ratio, 10.0, ny)
    T = int(3 * p["tau"])
    every = max(1, T // 600)
    _, ucm, _ = _run(ratio, 10.0, ny, T, 8, every, gamma_c=math.inf)
    _, nlm, _ = _run(ratio, 10.0, ny, T, 8, every)
    u, v = ucm[:, 1] / ucm[-1, 1], nlm[:, 1] / nlm[-1, 1]
    assert u.max() > 2.0                                   # strong elastic overshoot
    assert u[np.argmax(u):].min() < 0.9                    # then swings well below the steady value
    assert v.max() < 1.2                                   # the nlM: at most the Newtonian-like overshoot
    assert v[np.argmax(v):].min() > 0.99                   # and no swing below the steady value


def test_slower_structural_relaxation_lowers_the_steady_velocity():
    # Sec. IV (Fig. figtau): at the same width, theta = 100 reaches a lower steady velocity than theta = 10
    # (the slowly relaxing plug is more viscous); velocities on the scale g H^2 / (2 nu)
    vals = {}
    for theta in (10.0, 100.0):
        p = _params(4.0, theta, 8)
        T = int(4 * p["tau"])
        _, st, _ = _run(4.0, theta, 8, T, 8, max(1, T // 400))
        assert abs(st[-1, 1] - st[int(0.9 * len(st)), 1]) < 1e-3 * st[-1, 1]      # steady
        vals[theta] = st[-1, 1] / (p["g"] * p["H"] ** 2 / (2 * NU))
    assert vals[100.0] < vals[10.0]


@pytest.mark.parametrize("trace_full", [True, False])
def test_steady_density_balances_the_normal_stress_difference(trace_full):
    # Sec. IV (steady state): sigma_xx - sigma_yy > 0 in the flowing region pushes the fluid towards the
    # centre, which the density (pressure) increase there balances.  With the trace split of the coupling
    # the lattice momentum flux carries sigma_yy - tr(sigma)/2 = -N1/2, so the steady y-balance is
    # c_s^2 rho(y) + N1(y)/2 = const across the channel.
    p = _params(1.0, 10.0, 16)
    ch = oracle.Channel(oracle.D2Q9, 1, 16, tau_lb=TAU_LB, G_inf=p["G"], tau=p["tau"], gamma_c=0.1,
                        g=(p["g"], 0, 0), C=32, B=8, trace_full=trace_full)
    ch.step(int(6 * p["tau"]))
    f = ch.fields()
    ch.close()
    rho, n1 = f["rho"], f["n1"]
    assert np.all(n1 > 0)
    assert rho[7] > rho[0]                                  # denser in the centre than at the wall
    lhs = (rho - rho[0]) / 3.0                              # c_s^2 (rho(y) - rho(wall node))
    rhs = -(n1 - n1[0]) / 2.0
    assert np.max(np.abs(lhs - rhs)) <= 1e-4 * np.max(np.abs(rhs))     # 1e-6 seen
