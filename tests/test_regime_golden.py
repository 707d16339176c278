"""The paper's printed probe positions and transient-regime parameters (tests/golden/) against the
node convention (walls half a spacing outside the first and last node) and the sweep module's constants.
CPU only: nothing here launches a kernel."""
import os

import numpy as np
import pytest

from paper_1504_06123_gb300 import regime

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_printed_probe_positions_fall_on_nodes():
    # node j sits j + 1/2 from the wall: d = (j + 1/2)/H, H = N/2.  Every printed d is a node (the first
    # node for d_0, node N/4 for d_1/2) -- which fixes the wall half a spacing outside the first node.
    rows = _rows("probe_positions.txt")
    assert len(rows) == 5
    for n_str, d_str in rows:
        N, d = int(n_str), float(d_str)
        H = N / 2
        j = d * H - 0.5
        assert abs(j - round(j)) < 1e-9, (N, d)
        j = int(round(j))
        assert j in (0, N // 4)
        assert (j + 0.5) / H == pytest.approx(d, rel=0, abs=1e-15)
        # the sweep's probe lands on that node with weight 0
        j0, w = regime.probe_nodes(N, d)
        assert j0 == j and abs(w) < 1e-9


def test_probe_interpolation_between_nodes():
    # 20 nodes (H = 10): d = 0.51 lies 4.6 spacings from the first node's position
    j0, w = regime.probe_nodes(20, 0.51)
    assert j0 == 4 and w == pytest.approx(0.6, abs=1e-12)
    with pytest.raises(ValueError):
        regime.probe_nodes(20, 0.01)          # closer to the wall than the first node


def test_regime_constants_match_the_paper():
    kv = {r[0]: [float(x) for x in r[1:]] for r in _rows("regime_points.txt")}
    assert list(regime.PAPER_T_WALL_OVER_TAU0) == kv["t_wall_over_tau0"]
    assert regime.PAPER_THETA == kv["theta"][0]
    assert regime.PAPER_THETA_SLOW == kv["theta_slow"][0]
    assert set(kv["theta_slow_points"]) <= set(regime.PAPER_T_WALL_OVER_TAU0)
    assert regime.PAPER_GAMMA_C == kv["gamma_c"][0]
    assert regime.PAPER_TAU_LB == kv["tau_lb"][0]
    assert regime.D_HALF == kv["d_half"][0]


@pytest.mark.parametrize("ratio,theta,ny", [(0.01, 10, 8), (1.0, 10, 100), (8.0, 100, 40)])
def test_regime_channel_reproduces_its_dimensionless_numbers(ratio, theta, ny):
    c = regime.regime_channel(ratio, theta, ny)
    eta_inf = c.G_inf * c.tau0                      # eta_inf = G_inf tau_0 (Sec. II), rho0 = 1
    assert eta_inf == pytest.approx((0.9 - 0.5) / 3, rel=1e-14)        # = BGK viscosity
    t_wall = 4 * (ny / 2) ** 2 / (np.pi ** 2 * c.G_inf * c.tau0)       # Sec. IV, rho = 1
    assert t_wall / c.tau0 == pytest.approx(ratio, rel=1e-13)
    assert c.tau / c.tau0 == pytest.approx(theta, rel=1e-14)
    assert c.g * ny == pytest.approx(c.G_inf, rel=1e-14)               # Delta p / (2H) = G_inf


def test_width_and_history_span():
    for r in regime.PAPER_T_WALL_OVER_TAU0:
        ny = regime.width_for(r, 4000.0)
        assert ny % 2 == 0 and ny >= 8
    assert regime.width_for(1.0, 7600.0) == 100         # the paper's 100-node channel at t_wall = tau_0
    B = regime.history_blocks(5 * 40000.0, 128)
    assert 128 * (2 ** B - 1) >= 2e5 > 128 * (2 ** (B - 1) - 1)


def test_curves_normalise_by_the_end_of_startup():
    # host-side post-processing only: a sweep object with synthetic records (no device)
    sw = regime.RegimeSweep.__new__(regime.RegimeSweep)
    sw.channels = [regime.regime_channel(1.0, 10.0, 20)]
    sw.weights = [0.25]
    t = np.arange(1, 11) * 10
    vals = np.zeros((10, 2, 6))
    vals[:, 0, 1] = np.linspace(1, 10, 10)          # u at the first node
    vals[:, 1, 1] = np.linspace(1, 10, 10) * 3      # u at the second node
    vals[:, :, 5] = 2.0                             # sigma_xy
    vals[:, :, 3] = 5.0                             # sigma_xx
    vals[:, :, 4] = 1.0                             # sigma_yy
    sw._records = [(t, vals)]
    cur = sw.curves(60)[0]
    st, sp = cur["startup"], cur["cessation"]
    assert len(st["u"]) == 6 and len(sp["u"]) == 4
    u6 = 0.75 * 6 + 0.25 * 18                       # interpolated u at t = 60
    assert st["u"][-1] == pytest.approx(1.0) and sp["u"][0] == pytest.approx((0.75 * 7 + 0.25 * 21) / u6)
    assert np.allclose(st["sxy"], 1.0) and np.allclose(sp["n1"], 1.0)
    c = sw.channels[0]
    assert st["t_over_tau0"][0] == pytest.approx(10 / c.tau0)
    assert sp["t_over_twall"][0] == pytest.approx(10 / c.t_wall)


def test_curves_with_a_vanishing_normaliser_are_nan_with_a_warning():
    # a probe whose shear stress is zero at the end of startup (e.g. on the centreline): its sigma_xy curve
    # cannot be normalised and comes back NaN with a warning; the other curves are unaffected
    sw = regime.RegimeSweep.__new__(regime.RegimeSweep)
    sw.channels = [regime.regime_channel(1.0, 10.0, 20)]
    sw.weights = [0.25]
    t = np.arange(1, 11) * 10
    vals = np.zeros((10, 2, 6))
    vals[:, :, 1] = 1.0                             # u
    vals[:, :, 3] = 5.0                             # sigma_xx
    vals[:, :, 4] = 1.0                             # sigma_yy; sigma_xy stays 0
    sw._records = [(t, vals)]
    with pytest.warns(RuntimeWarning, match="sxy"):
        cur = sw.curves(60)[0]
    assert np.all(np.isnan(cur["startup"]["sxy"])) and np.all(np.isnan(cur["cessation"]["sxy"]))
    assert np.allclose(cur["startup"]["u"], 1.0) and np.allclose(cur["cessation"]["n1"], 1.0)

