"""GPU: the probe recorder (lbve_set_probes / lbve_probe_read) and the paper-regime sweep (Sec. IV).

- the recorder's values are those of lbve_fields at the recorded steps, bitwise, through the 16-step
  graphs and single steps alike; overflow is counted; bad arguments are refused;
- a batch of paper-regime channels through startup and cessation against the FP64 oracle, probe by probe
  (normwise per field over the whole series: <= 1e-12 with an FP64 history, <= 1e-5 for the plain FP32
  form);
- the full sweep of Fig. Qall (seven widths, theta = 10) and Fig. figtau (theta = 100) shows the
  transient features the paper describes (the oracle pins the same features on small channels).
"""
import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import lbve as L
from paper_1504_06123_gb300 import regime

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



def _batch_descs():
    d1 = L.make_desc(L.LBVE_D2Q9, 3, 10, tau_lb=0.8, G_inf=0.01, tau=30.0, gamma_c=0.1, g=(2e-5, 0, 0), C=8, B=3,
                     precision=L.LBVE_F64, hist_storage=L.LBVE_F32)
    d2 = L.make_desc(L.LBVE_D2Q9, 1, 16, tau_lb=0.9, G_inf=0.005, tau=50.0, gamma_c=0.2, g=(1e-5, 0, 0), C=8,
                     B=3, precision=L.LBVE_F64, hist_storage=L.LBVE_F32)
    return [d1, d2]


def test_probe_records_equal_fields_bitwise():
    ch = L.Channel(_batch_descs())
    N = ch.N
    nodes = np.array([0, 7, 29, 30, 45, N - 1], dtype=np.int64)
    ch.step(5)
    img = L.lbve_checkpoint_save(ch.h)
    every, steps = 3, 53            # 3 graphs of 16 steps + 5 single steps, odd parity at the end
    L.lbve_set_probes(ch.h, nodes, every, 100)
    ch.step(steps)
    t, vals, tot = L.lbve_probe_read(ch.h, len(nodes), 2, 100)
    assert list(t) == [s for s in range(6, 5 + steps + 1) if s % every == 0]
    assert tot == len(t)
    # replay from the checkpoint one step at a time and read the fields at every recorded step
    L.lbve_set_probes(ch.h, [], 1, 1)
    L.lbve_checkpoint_restore(ch.h, img)
    ref = []
    for s in range(6, 5 + steps + 1):
        ch.step(1)
        if s % every == 0:
            f = ch.fields()
            ref.append(np.stack([np.concatenate(([f["rho"][n]], f["u"][n], f["sigma"][n])) for n in nodes]))
    ref = np.array(ref)
    assert vals.shape == ref.shape
    assert np.array_equal(vals, ref)
    ch.close()


def test_probe_overflow_reset_and_errors():
    ch = L.Channel(_batch_descs())
    L.lbve_set_probes(ch.h, [3, 4], 1, 4)
    ch.step(10)
    t, vals, tot = L.lbve_probe_read(ch.h, 2, 2, 4)
    assert list(t) == [1, 2, 3, 4] and tot == 10
    L.lbve_set_probes(ch.h, [3], 2, 50)           # clears the records
    ch.step(20)                                     # one graph + 4 steps
    t, vals, tot = L.lbve_probe_read(ch.h, 1, 2, 50)
    assert list(t) == list(range(12, 31, 2)) and tot == 10
    for bad in (dict(nodes=[-1]), dict(nodes=[ch.N]), dict(nodes=[0], every=0), dict(nodes=[0], capacity=0)):
        kw = dict(every=1, capacity=1)
        kw.update(bad)
        with pytest.raises(L.LbveError) as e:
            L.lbve_set_probes(ch.h, kw.pop("nodes"), **kw)
        assert e.value.status == L.LBVE_EINVAL
    L.lbve_set_probes(ch.h, [], 1, 1)
    with pytest.raises(L.LbveError) as e:
        L.lbve_probe_read(ch.h, 1, 2, 1)
    assert e.value.status == L.LBVE_EINVAL
    ch.step(3)                                      # stepping without a recorder still works
    ch.close()
    tg = L.lbve_create_tangent(_batch_descs()[0])
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_probes(tg, [0], 1, 1)
    assert e.value.status == L.LBVE_ENOSUPPORT
    L.lbve_destroy(tg)


def _oracle_series(desc, nodes_local, steps_start, steps_stop, every):
    o = oracle.Channel(oracle.D2Q9, desc.nx, desc.ny, tau_lb=desc.tau_lb, G_inf=desc.G_inf, tau=desc.tau,
                       gamma_c=desc.gamma_c, g=tuple(desc.g), C=desc.hist_C, B=desc.hist_B)
    rows = []
    for n, g in ((steps_start, tuple(desc.g)), (steps_stop, (0.0, 0.0, 0.0))):
        o.set_force(g)
        for _ in range(n // every):
            o.step(every)
            f = o.fields()
            rows.append(np.stack([np.concatenate(([f["rho"][j]], f["u"][j], f["sigma"][j])) for j in nodes_local]))
    o.close()
    return np.array(rows)


@pytest.mark.parametrize("hist,tol", [(L.LBVE_F64, 1e-12), (L.LBVE_F32, 1e-5)])
def test_regime_sweep_vs_oracle(hist, tol):
    # a narrow and a wide channel of the paper's regime at a small tau_0 (300 steps), C = 16 points per block
    sw = regime.RegimeSweep([(0.1, 10.0), (8.0, 10.0)], 300.0, C=16, span_tau=2.0, hist_storage=hist)
    assert [c.ny for c in sw.channels] == [8, 56]
    n_on, n_off, every = 640, 480, 16
    sw.startup(n_on, every)
    sw.cessation(n_off, every)
    t = np.concatenate([r[0] for r in sw._records])
    vals = np.concatenate([r[1] for r in sw._records])
    assert list(t) == list(range(every, n_on + n_off + 1, every))
    for k, desc in enumerate(sw.descs):
        off, _ = L.lbve_channel_nodes(sw.batch.h, k)
        local = [int(n - off) for n in sw.nodes[2 * k:2 * k + 2]]
        ref = _oracle_series(desc, local, n_on, n_off, every)
        got = vals[:, 2 * k:2 * k + 2]
        for name, sl in (("rho", slice(0, 1)), ("u", slice(1, 3)), ("sigma", slice(3, 6))):
            r = ref[..., sl]
            e = np.max(np.abs(got[..., sl] - r)) / np.max(np.abs(r))
            assert e <= tol, (k, name, e)
    # interpolated series: u at d = 0.51 rises, then turns back after cessation
    s = sw.series()
    assert all(np.max(x["u"]) > 0 for x in s)
    sw.close()


def _claims_sweep(points, tau0, startup_tau=3.0, stop_tau=2.0, every=16):
    sw = regime.RegimeSweep(points, tau0)
    tau_max = max(c.tau for c in sw.channels)
    n_on = int(startup_tau * tau_max) // every * every
    n_off = int(stop_tau * tau_max) // every * every
    sw.startup(n_on, every)
    sw.cessation(n_off, every)
    s = sw.series()
    k = n_on // every
    return sw, [({key: v[:k] for key, v in x.items()}, {key: v[k:] for key, v in x.items()}) for x in s]


@pytest.fixture(scope="module")
def paper_sweep():
    """Fig. Qall: the seven widths at theta = 10 (tau_0 about 4000 steps; 8 to 206 nodes across)."""
    pts = [(r, regime.PAPER_THETA) for r in regime.PAPER_T_WALL_OVER_TAU0]
    sw, res = _claims_sweep(pts, 4000.0)
    out = (sw.channels, res)
    sw.close()
    return out


@pytest.fixture(scope="module")
def slow_sweep():
    """Fig. figtau: t_wall/tau_0 = 0.1, 1, 4 at theta = 100 (tau_0 about 400 steps)."""
    pts = [(r, regime.PAPER_THETA_SLOW) for r in (0.1, 1.0, 4.0)]
    sw, res = _claims_sweep(pts, 400.0)
    out = (sw.channels, res)
    sw.close()
    return out


def test_paper_sweep_startup_velocity(paper_sweep):
    chans, res = paper_sweep
    for c, (st, _) in zip(chans, res):
        u = st["u"] / st["u"][-1]
        if c.ratio <= 1.0:     # steady after 3 tau (the widest channels approach it on several t_wall)
            assert abs(st["u"][-1] - st["u"][int(0.9 * len(u))]) < 2e-3 * st["u"][-1], c.ratio
        if c.ratio <= 0.1:
            assert u.max() > 1.05, (c.ratio, u.max())          # overshoot in narrow channels
        if c.ratio >= 2.0:                                      # monotonic rise in wide ones
            assert np.all(np.diff(st["u"]) > -1e-6 * st["u"][-1]), c.ratio
    # the overshoot shrinks as the channel widens
    over = [(st["u"] / st["u"][-1]).max() for st, _ in res]
    assert over[0] > over[1] > over[3]


def test_paper_sweep_cessation(paper_sweep):
    chans, res = paper_sweep
    for c, (st, sp) in zip(chans, res):
        u, s = sp["u"], sp["sxy"]
        assert u.min() < -0.005 * st["u"][-1], c.ratio          # counter-flow
        tu, ts = sp["t"][np.argmax(u < 0)], sp["t"][np.argmax(s < 0)]
        assert np.any(s < 0) and tu < ts, c.ratio               # velocity ahead of the stress
        n1 = np.concatenate([st["n1"], sp["n1"]])
        tt = np.concatenate([st["t"], sp["t"]])
        # sigma_xx - sigma_yy > 0 throughout (zero only before the shear has reached the probe)
        assert np.all(n1 >= 0) and np.all(n1[tt > 0.1 * c.t_wall] > 0), c.ratio
        d = sp["n1"] / st["n1"][-1]
        assert np.max(d - np.minimum.accumulate(d)) < 0.01, c.ratio   # monotonic decay after cessation


def test_paper_sweep_theta_dependence(paper_sweep, slow_sweep):
    # Fig. figtau: at larger theta the steady velocity is lower (higher viscosity of the plug); the
    # narrow channel still overshoots, the wide one does not.  Velocities on the scale g H^2 / (2 nu).
    fast = {c.ratio: (c, st) for c, (st, _) in zip(*paper_sweep)}
    for c, (st, _) in zip(*slow_sweep):
        cf, stf = fast[c.ratio]
        scale = lambda ch: ch.g * ch.H ** 2 / (2 * ch.nu)
        assert st["u"][-1] / scale(c) < stf["u"][-1] / scale(cf), c.ratio
        u = st["u"] / st["u"][-1]
        if c.ratio <= 0.1:
            assert u.max() > 1.05, u.max()
        if c.ratio >= 4.0:     # at most a trace of overshoot left (the rise is monotonic at theta = 10)
            assert u.max() < 1.01, u.max()


def test_regime_bench_batch_vs_oracle():
    """The benchmark's batch (ten channels of Figs. Qall / figtau, nx = 4, L = 1920, launch shape of the
    autotuner) against the oracle: 96 steps of startup with the probes recorded every step; channels of
    10, 100 and 200 nodes across checked node by node (column 0; the flow is x-invariant, so a one-column
    oracle channel is that column) and the probe records of those channels."""
    pts = regime.paper_points()
    chans, descs, B = regime.sweep_descs(pts, regime.tau0_for_width(100), nx=4)
    assert B == 15 and len(descs) == 10
    batch = L.Channel(descs)
    offs = [L.lbve_channel_nodes(batch.h, k)[0] for k in range(len(descs))]
    nodes, _ = regime.probe_plan(chans, offs, 4)
    L.lbve_set_probes(batch.h, nodes, 1, 200)
    steps = 96
    batch.step(steps)
    t, vals, tot = L.lbve_probe_read(batch.h, len(nodes), 2, 200)
    assert list(t) == list(range(1, steps + 1)) and tot == steps
    f = batch.fields()
    for k in (0, 3, 9):
        d = descs[k]
        o = oracle.Channel(oracle.D2Q9, 1, d.ny, tau_lb=d.tau_lb, G_inf=d.G_inf, tau=d.tau, gamma_c=d.gamma_c,
                           g=tuple(d.g), C=d.hist_C, B=d.hist_B)
        ref = []
        for _ in range(steps):
            o.step(1)
            of = o.fields()
            j0 = (nodes[2 * k] - offs[k]) // 4
            ref.append([np.concatenate(([of["rho"][j]], of["u"][j], of["sigma"][j])) for j in (j0, j0 + 1)])
        of = o.fields()
        o.close()
        col = slice(offs[k], offs[k] + 4 * d.ny, 4)           # column x = 0 of channel k
        for key in ("u", "sigma", "kappa"):
            got = f[key][col]
            e = np.max(np.abs(got - of[key])) / np.max(np.abs(of[key]))
            assert e <= 1e-5, (k, key, e)
        ref = np.array(ref)
        got = vals[:, 2 * k:2 * k + 2]
        # on the scale of the channel's field (the shear has not reached the probe of a wide channel yet)
        for sl, key in ((slice(1, 3), "u"), (slice(3, 6), "sigma")):
            e = np.max(np.abs(got[..., sl] - ref[..., sl])) / np.max(np.abs(of[key]))
            assert e <= 1e-5, (k, key, e)
    batch.close()
