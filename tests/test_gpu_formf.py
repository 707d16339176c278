"""GPU parity of history form F -- the paper's factor storage (Sec. III, Eq. eeval) -- against the FP64 oracle.

Form F keeps, per retained point, its factor deviation F - 1 and its rate of strain kappa + kappa^T, written
once, and re-forms E(t, t') every step as the ordered product of the factors (the oracle does the same with
full matrices in FP64).  Storages: FP64 (bar 1e-12, like every FP64 path), FP32 (plain FP32 bar 1e-5) and
16-bit block-scaled (the reduced-precision bar 1e-3).  Every case of the form-P parity tests that applies is
repeated here: the history integral alone on prescribed gradients (ragged node counts, odd block sizes,
3D), the small channel through startup and cessation on both history grids, edge cases, batches, launch
shapes, graph replay and checkpoint / resume.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import configs, inputs
from paper_1504_06123_gb300 import lbve as L
from tests.test_gpu_parity import BATCH, compare, rel_err, same_sweep_shape

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64, S16 = L.LBVE_F32, L.LBVE_F64, L.LBVE_S16
FF = L.LBVE_FORM_F
# (population precision, history storage) -> bar
ALL64, PLAIN, ALL32, RED = (F64, F64), (F64, F32), (F32, F32), (F32, S16)
TOL = {ALL64: 1e-12, PLAIN: 1e-5, ALL32: 5e-5, RED: 1e-3, F64: 1e-12, F32: 1e-5, S16: 1e-3}


@pytest.mark.parametrize("hist", [F64, F32, S16])
@pytest.mark.parametrize("lattice,nx,ny,nz,C,B", [
    (L.LBVE_D2Q9, 7, 115, 1, 16, 4),      # 805 nodes: several tiles + ragged tail
    (L.LBVE_D2Q9, 1, 9, 1, 8, 1),         # uniform ring, tiny
    (L.LBVE_D2Q9, 33, 64, 1, 5, 3),       # odd C
    (L.LBVE_D3Q19, 3, 7, 11, 8, 3),       # 231 nodes, 3x3 tensors
])
def test_formf_history_apply_vs_oracle(hist, lattice, nx, ny, nz, C, B):
    d = 2 if lattice == L.LBVE_D2Q9 else 3
    N = nx * ny * nz
    T = 150
    G, tau, gc = 0.02, 40.0, 0.1
    kseq = inputs.kappa_sequence(T, N, d, 2e-3, seed=11, shear=1e-3)
    ref = oracle.history_run(kseq, C, B, G, tau, gc)
    ch = L.Channel(L.make_desc(lattice, nx, ny, nz, G_inf=G, tau=tau, gamma_c=gc, C=C, B=B, precision=F64,
                               hist_storage=hist, hist_form=FF))
    ns = 3 if d == 2 else 6
    kap_dev = torch.empty((d * d, N), dtype=torch.float64, device="cuda")
    sig_dev = torch.empty((ns, N), dtype=torch.float64, device="cuda")
    worst = 0.0
    for t in range(T):
        kap_dev.copy_(torch.from_numpy(kseq[t].reshape(N, d * d).T.copy()))
        L.lbve_history_apply(ch.h, kap_dev, sig_dev)
        if t % 7 == 0 or t == T - 1:
            e = rel_err(sig_dev.cpu().numpy().T, ref[t])
            worst = max(worst, e)
            assert e <= TOL[hist], f"step {t}: sigma error {e:.3e}"
    print(f"form F history-only {hist} lattice {lattice} C={C} B={B}: worst sigma error {worst:.2e}")
    ch.close()


@pytest.mark.parametrize("prec", [ALL64, PLAIN, ALL32, RED])
@pytest.mark.parametrize("C,B", [(256, 1), (64, 4)])
def test_formf_small_channel_startup_cessation(prec, C, B):
    w = configs.plain_channel_small()
    orc = oracle.Channel(oracle.D2Q9, w.nx, w.ny, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                         g=(w.g, 0, 0), C=C, B=B)
    ch = L.Channel(w.desc(C=C, B=B, precision=prec[0], hist_storage=prec[1], hist_form=FF))
    t = 0
    for cp in [1, 2, 10, 100, 700, w.steps, w.steps + 1, w.steps + 300, w.steps + w.off_steps]:
        ch.step(cp - t)
        orc.step(cp - t)
        t = cp
        compare(ch.fields(), orc.fields(), TOL[prec], f"form F {prec} C={C} B={B} step {t}")
        if t == w.steps:
            ch.set_force((0, 0, 0))
            orc.set_force((0, 0, 0))
    ch.close()


@pytest.mark.parametrize("case", [
    dict(lattice=L.LBVE_D2Q9, nx=1, ny=2, C=4, B=2, G_inf=0.01, tau=20.0, gamma_c=0.1, g=1e-5),
    dict(lattice=L.LBVE_D2Q9, nx=3, ny=7, C=6, B=3, G_inf=0.02, tau=15.0, gamma_c=math.inf, g=2e-5),
    dict(lattice=L.LBVE_D2Q9, nx=6, ny=10, C=8, B=2, G_inf=0.01, tau=30.0, gamma_c=0.2, g=1e-5,
         trace_coupling=L.LBVE_TRACE_NONE),
    dict(lattice=L.LBVE_D2Q9, nx=9, ny=13, C=8, B=3, G_inf=0.01, tau=30.0, gamma_c=0.2, g=1e-5, noise=1e-4),
    dict(lattice=L.LBVE_D3Q19, nx=3, ny=6, nz=5, C=8, B=2, G_inf=0.01, tau=25.0, gamma_c=0.1, g=2e-5),
    dict(lattice=L.LBVE_D3Q19, nx=2, ny=5, nz=4, C=4, B=3, G_inf=0.01, tau=25.0, gamma_c=0.1, g=2e-5,
         wall_z=0, noise=1e-4),
])
@pytest.mark.parametrize("prec", [ALL64, PLAIN, RED])
def test_formf_edge_cases_vs_oracle(case, prec):
    c = dict(case)
    noise = c.pop("noise", 0.0)
    lattice = c.pop("lattice")
    nz = c.pop("nz", 1)
    wall_z = c.pop("wall_z", 1)
    tc = c.pop("trace_coupling", L.LBVE_TRACE_FULL)
    g = c.pop("g")
    N = c["nx"] * c["ny"] * nz
    rho = inputs.initial_density(N, noise, seed=7)
    orc = oracle.Channel(lattice, c["nx"], c["ny"], nz, tau_lb=0.9, G_inf=c["G_inf"], tau=c["tau"],
                         gamma_c=c["gamma_c"], g=(g, 0, 0), C=c["C"], B=c["B"], wall_z=bool(wall_z),
                         trace_full=(tc == L.LBVE_TRACE_FULL), rho_init=rho)
    ch = L.Channel(L.make_desc(lattice, c["nx"], c["ny"], nz, tau_lb=0.9, G_inf=c["G_inf"], tau=c["tau"],
                               gamma_c=c["gamma_c"], g=(g, 0, 0), C=c["C"], B=c["B"], precision=prec[0],
                               hist_storage=prec[1], trace_coupling=tc, wall_z=wall_z, hist_form=FF), rho)
    for n in (1, 5, 60, 200):
        ch.step(n)
        orc.step(n)
        if ch.t == 1 and noise and prec != ALL64:
            continue     # the first step's noise-only gradients are below what FP32 velocities resolve
        compare(ch.fields(), orc.fields(), TOL[prec], f"form F {case} t={ch.t}")
    ch.close()


@pytest.mark.parametrize("prec", [ALL64, PLAIN, RED])
def test_formf_batched_channels_vs_oracle(prec):
    C, B = 16, 4
    descs = [L.make_desc(L.LBVE_D2Q9, c["nx"], c["ny"], tau_lb=c["tau_lb"], G_inf=c["G_inf"], tau=c["tau"],
                         gamma_c=c["gamma_c"], g=(c["g"], 0, 0), C=C, B=B, precision=prec[0], hist_storage=prec[1],
                         hist_form=FF)
             for c in BATCH]
    Ntot = sum(c["nx"] * c["ny"] for c in BATCH)
    rho = inputs.initial_density(Ntot, 1e-5, seed=9)
    ch = L.Channel(descs, rho)
    orcs, off = [], 0
    for c in BATCH:
        n = c["nx"] * c["ny"]
        orcs.append(oracle.Channel(oracle.D2Q9, c["nx"], c["ny"], tau_lb=c["tau_lb"], G_inf=c["G_inf"], tau=c["tau"],
                                   gamma_c=c["gamma_c"], g=(c["g"], 0, 0), C=C, B=B, rho_init=rho[off:off + n]))
        off += n
    t = 0
    for cp in (1, 37, 200, 260, 400):
        ch.step(cp - t)
        for o in orcs:
            o.step(cp - t)
        t = cp
        f = ch.fields()
        for i, o in enumerate(orcs):
            compare(ch.channel_fields(i, f), o.fields(), TOL[prec], f"form F batch channel {i} t={t}")
        if t == 200:
            ch.set_force((0, 0, 0), channel=1)
            orcs[1].set_force((0, 0, 0))
    ch.close()


@pytest.mark.parametrize("hist", [F64, F32, S16])
def test_formf_launch_shapes_agree(hist):
    """Every slot-chunk count gives the same sums up to the order of additions (the chunks' carries are
    composed in the commit); the same shape on two handles gives the same bits; CTA tasks are refused."""
    kw = dict(nx=6, ny=40, G_inf=0.01, tau=40.0, gamma_c=0.1, g=(1e-5, 0, 0), C=16, B=4, precision=F64,
              hist_storage=hist, hist_form=FF)
    Smax = 16 * 4 // 8
    ref = None
    for S in (1, 3, Smax):
        ch = L.Channel(L.make_desc(**kw))
        L.lbve_set_sweep_config(ch.h, S, 0)
        ch.step(70)
        f = ch.fields()
        if ref is None:
            ref = f
        else:
            for key in ("u", "sigma"):
                assert rel_err(f[key], ref[key]) <= {F64: 1e-13, F32: 1e-6, S16: 1e-6}[hist], (S, key)
        ch.close()
    a = L.Channel(L.make_desc(**kw))
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_sweep_config(a.h, 1, 1)
    assert e.value.status == L.LBVE_EINVAL
    b = L.Channel(L.make_desc(**kw))
    same_sweep_shape(a, b)
    a.step(3)
    a.step(45)          # an odd step, then 16-step graphs, then the rest
    for _ in range(48):
        b.step(1)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    a.close()
    b.close()


def test_formf16_balanced_ranges():
    """Task mode 2 of the 16-bit form F (balanced ranges): every warp of the resident grid streams an equal
    run of the tile-major (tile, rank) sequence, a tile is cut into pieces whose chunk records the commit
    composes in rank order.  Against the FP64 oracle at the reduced-precision bar; against chunk tasks to a
    few units of the 16-bit storage's rounding (2^-15 of a vector's scale: a different order of the FP32
    additions can move a stored value across a rounding boundary, and the runs then differ at that level);
    bitwise equal on two handles; refused for another storage and where the pieces of a tile would exceed
    B*C/8."""
    kw = dict(nx=8, ny=320, tau_lb=0.8, G_inf=0.01, tau=200.0, gamma_c=0.1, g=(2e-6, 0, 0), C=128, B=8)
    gkw = dict(kw, precision=F32, hist_storage=S16, hist_form=FF)
    ref = L.Channel(L.make_desc(**gkw))
    L.lbve_set_sweep_config(ref.h, 4, 0)
    bal = [L.Channel(L.make_desc(**gkw)) for _ in range(2)]
    for b in bal:
        L.lbve_set_sweep_config(b.h, 1, 2)
        S, ctas, mode = L.lbve_sweep_config(b.h)
        assert mode == 2 and 1 < S <= 128, (S, ctas, mode)
    ref.step(300)
    bal[0].step(300)
    bal[1].step(7)      # odd steps, then 16-step graphs
    bal[1].step(293)
    fr, f0, f1 = ref.fields(), bal[0].fields(), bal[1].fields()
    orc = oracle.Channel(oracle.D2Q9, kw["nx"], kw["ny"], tau_lb=kw["tau_lb"], G_inf=kw["G_inf"], tau=kw["tau"],
                         gamma_c=kw["gamma_c"], g=kw["g"], C=kw["C"], B=kw["B"])
    orc.step(300)
    compare(f0, orc.fields(), TOL[RED], "balanced ranges, 8 x 320, L = 1024, 300 steps")
    orc.close()
    for key in ("u", "sigma", "kappa"):
        assert rel_err(f0[key], fr[key]) <= 1e-4, key
    for k in f0:
        assert np.array_equal(f0[k], f1[k]), k
    for c in [ref] + bal:
        c.close()
    other = L.Channel(L.make_desc(**dict(gkw, hist_storage=F32)))
    small = L.Channel(L.make_desc(**dict(gkw, ny=40, C=16, B=4)))
    for c in (other, small):
        with pytest.raises(L.LbveError) as e:
            L.lbve_set_sweep_config(c.h, 1, 2)
        assert e.value.status == L.LBVE_EINVAL
        c.close()


def test_formf16_balanced_ranges_duct():
    """Balanced ranges of the 3D sweep (two nodes a lane, 64-node tiles): a 6 x 32 x 32 duct (6144 nodes, 96 tiles,
    each cut into some 26 pieces on 2432 resident warps; L = 4 x 64 allows 32) with the 16-bit form F pinned to
    mode 2, against the FP64 oracle at the reduced-precision bar, and bitwise equal on a second handle."""
    kw = dict(tau_lb=0.9, G_inf=0.005, tau=60.0, gamma_c=0.1, g=(2e-5, 0, 0), C=64, B=4)
    chans = []
    for _ in range(2):
        c = L.Channel(L.make_desc(L.LBVE_D3Q19, 6, 32, 32, precision=F32, hist_storage=S16, hist_form=FF, **kw))
        L.lbve_set_sweep_config(c.h, 1, 2)
        assert L.lbve_sweep_config(c.h)[2] == 2
        chans.append(c)
    chans[0].step(150)
    chans[1].step(3)
    chans[1].step(147)
    f0, f1 = chans[0].fields(), chans[1].fields()
    for k in f0:
        assert np.array_equal(f0[k], f1[k]), k
    orc = oracle.Channel(oracle.D3Q19, 6, 32, 32, **kw)
    orc.step(150)
    compare(f0, orc.fields(), TOL[RED], "balanced ranges, 6 x 32 x 32 duct, L = 256, 150 steps")
    orc.close()
    for c in chans:
        c.close()


@pytest.mark.parametrize("hist", [F32, S16])
def test_formf_empty_trailing_chunks(hist):
    """A history grid where chunk tasks leave the last chunk empty at some steps (B = 3, C = 27: 79 to 81
    points, S = 10 chunks of 9 ranks hold 81 points in nine): the commit composes the chunks up to the one
    that holds the oldest point and reads no product of that one (the 16-bit sweep sums a tile's oldest
    chunk in Horner form and writes none).  Every shape against the FP64 oracle at the storage's bar."""
    kw = dict(nx=4, ny=40, tau_lb=0.8, G_inf=0.01, tau=30.0, gamma_c=0.1, g=(1e-5, 0, 0), C=27, B=3)
    orc = oracle.Channel(oracle.D2Q9, kw["nx"], kw["ny"], tau_lb=kw["tau_lb"], G_inf=kw["G_inf"], tau=kw["tau"],
                         gamma_c=kw["gamma_c"], g=kw["g"], C=kw["C"], B=kw["B"])
    orc.step(90)
    ref = orc.fields()
    orc.close()
    for S in (1, 9, 10):
        ch = L.Channel(L.make_desc(**dict(kw, precision=F32 if hist == S16 else F64, hist_storage=hist,
                                          hist_form=FF)))
        L.lbve_set_sweep_config(ch.h, S, 0)
        ch.step(90)
        compare(ch.fields(), ref, TOL[hist], f"form F {hist} S = {S}")
        ch.close()


@pytest.mark.parametrize("hist", [F32, S16])
def test_formf_checkpoint_resume_bitwise(hist):
    kw = dict(nx=6, ny=14, G_inf=0.01, tau=40.0, gamma_c=0.1, g=(1e-5, 0, 0), C=8, B=3, precision=F32,
              hist_storage=hist, hist_form=FF)
    a = L.Channel(L.make_desc(**kw))
    a.step(37)
    img = L.lbve_checkpoint_save(a.h)
    a.step(50)
    ref = a.fields()
    b = L.Channel(L.make_desc(**kw))
    same_sweep_shape(a, b)
    L.lbve_checkpoint_restore(b.h, img)
    b.step(50)
    for k, v in ref.items():
        assert np.array_equal(b.fields()[k], v), k
    # a form-P handle of the same channel refuses the form-F image
    p = L.Channel(L.make_desc(**dict(kw, hist_form=L.LBVE_FORM_P)))
    with pytest.raises(L.LbveError) as e:
        L.lbve_checkpoint_restore(p.h, img)
    assert e.value.status == L.LBVE_EINVAL
    for ch in (a, b, p):
        ch.close()


def test_formf_reads_less_memory_than_form_p():
    """Form F stores d*d + NS values per point against form P's 2 d*d (2D: 7 against 8, 3D: 15 against 18)."""
    kw = dict(nx=4, ny=64, C=32, B=4)
    sizes = {}
    for form in (L.LBVE_FORM_P, FF):
        for hist in (F32, S16):
            ch = L.Channel(L.make_desc(precision=F32, hist_storage=hist, hist_form=form, **kw))
            sizes[form, hist] = L.lbve_memory_bytes(ch.h)
            ch.close()
    assert sizes[FF, F32] < sizes[L.LBVE_FORM_P, F32]
    assert sizes[FF, S16] < sizes[L.LBVE_FORM_P, S16]
