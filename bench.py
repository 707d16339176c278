#!/usr/bin/env python3
"""Throughput of the hybrid LB step (stress history integral + D2Q9 stream-collide) on one GB300.

Workload: the 1024 x 512 D2Q9 channel with L = 1024 retained history points per node (B = 8 blocks of
C = 128), FP32, synthetic initial density noise 1e-6 (seed 2).  A step is one full hybrid step of every
node.  Metric: node-history updates per second (one retained history point of one node processed in
one step); MLUPS of the full step is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload channel|batched|duct] [--history f32|s16|f64] [--model nlm|wm|inlm]

--impl ours (default): the CUDA library through its C ABI.  Timed region: K steps bracketed by a
barrier and a device synchronisation, CUDA events on the launching stream, max over ranks.  The
history state (17 GB) is far larger than L2, so no flush is needed between steps.
--impl reference: the FP64 CPU oracle (tests' reference implementation) on the host cores, on a
bounded sample of the same workload (2 of the 1024 columns, all 512 rows, full history).
With N > 1 (torchrun) every rank runs an independent replica (the method does not shard across
GPUs here): value = all ranks' updates / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-history updates/s"
UNIT = "node-history updates/s"
METRIC_NODES = "lattice node updates/s"   # the instantaneous model: no history points
BYTES_PER_UPDATE = 48        # FP32 D2Q9: read X (16 B) + write X (16 B) + read kappa (16 B) per point
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-chosen", action="store_true", help="skip the reduced-precision comparison run")
    ap.add_argument("--workload", choices=["channel", "batched", "duct", "regime", "gradient"], default="channel",
                    help="channel: the 1024 x 512 D2Q9 channel (the benchmark line); batched: 64 channels of "
                         "uneven width; duct: the D3Q19 128^3 square duct; regime: the paper's transient sweep "
                         "(ten channels of Figs. Qall and figtau in one batch, probes recorded every step); "
                         "gradient: dL/d(G_inf, tau, gamma_c, g) of the 4 x 128 channel, L = 512, 4000 steps by "
                         "the adjoint with checkpoints every 64 steps (a step of this line = one gradient)")
    ap.add_argument("--history", choices=["f32", "s16", "f64"], default="f32",
                    help="history storage: f32 (plain FP32 form), s16 (16-bit block-scaled precision variant), f64")
    ap.add_argument("--form", choices=["p", "f"], default="p",
                    help="history form: p (E - 1 advanced in place; the benchmark line) or f (the paper's factor "
                         "storage: F - 1 and kappa + kappa^T written once, E re-formed by products every step)")
    ap.add_argument("--lb-steps", type=int, default=None,
                    help="gradient workload: LB steps per gradient (default the workload's 4000); fewer only for "
                         "profiler captures, not a bench line")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-channel batch arms of the channel line (batched chosen form, batched FP32, "
                         "one handle per channel)")
    ap.add_argument("--model", choices=["nlm", "wm", "inlm"], default="nlm",
                    help="constitutive model: nlm (integral nlM, the benchmark line), wm (White-Metzner form), "
                         "inlm (instantaneous nlM of Eq. inlM: no history; metric lattice node updates/s)")
    ap.add_argument("--drive", choices=["force", "pressure"], default="force",
                    help="force: body force g with x periodic (the benchmark line); pressure: the pressure-step "
                         "boundary along x with the equivalent drop dp = rho0 g nx per period")
    ap.add_argument("--nx", type=int, default=None,
                    help="narrower channel (same rows, same history) for profiler captures; not a bench line")
    ap.add_argument("--sweep-shape", default=None,
                    help="S,mode: pin the history sweep's launch shape after the autotuner (slot chunks; mode 0 "
                         "warp tasks, 1 CTA tasks, 2 balanced ranges of the 16-bit form F), e.g. to profile the "
                         "shape a timed run chose")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 7:
                    continue
                try:
                    sm.append(float(f[0]))
                    mx.append(float(f[1]))
                except ValueError:
                    continue
                for name, v in zip(names, f[3:7]):
                    if v.lower() == "active":
                        reasons.add(name)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def points_per_step(C: int, B: int, t0: int, K: int, L) -> list:
    """Retained history points (including the one created) of steps t0 .. t0+K-1 (same at every node)."""
    return [len(L.lbve_schedule(C, B, t)[0]) for t in range(t0, t0 + K)]


def bytes_per_update(D: int, hist: int, form: int, L, wm: bool = False) -> float:
    """Algorithmic history bytes per node-history update of the sweep (what one step must move per retained
    point): form P reads and writes X = E - 1 and reads kappa (d*d values each; the 16-bit frame form reads
    Q - 1 and kappa, int16 mantissas plus an exponent byte each, and rewrites Q every 32nd step); form F only
    reads F - 1 (d*d) and kappa + kappa^T (NS)."""
    DD, NS = D * D, (3 if D == 2 else 6)
    if form == L.LBVE_FORM_F:
        if hist == L.LBVE_S16:
            return 2 * (DD + NS) + 2
        return (DD + NS) * (4 if hist == L.LBVE_F32 else 8)
    if hist == L.LBVE_S16:
        return 2 * (2 * DD + 1) + (2 * DD + 1) / 32
    b = 3 * DD * (4 if hist == L.LBVE_F32 else 8)
    return b + (8 if wm else 0)


FORM_NAMES = {("p", "f32"): "form P, FP32 history (E - 1 and kappa), FP64 populations",
              ("p", "s16"): "form P, 16-bit block-scaled history (kappa, Q in a per-node frame), FP32 populations",
              ("f", "f32"): "form F (factor storage), FP32 history (F - 1, kappa + kappa^T), FP64 populations",
              ("f", "s16"): "form F (factor storage), 16-bit block-scaled F - 1 and kappa + kappa^T, FP32 populations"}
FORM_BAR = {("p", "f32"): 1e-5, ("p", "s16"): 1e-3, ("f", "f32"): 1e-5, ("f", "s16"): 1e-3}


def form_descs(descs, L, form: str, hist: str):
    """Copies of the workload's descriptions in another history form / storage (16-bit: FP32 populations)."""
    import copy as _copy
    out = [_copy.copy(d) for d in descs]
    for d in out:
        d.hist_form = L.LBVE_FORM_F if form == "f" else L.LBVE_FORM_P
        d.hist_storage = L.LBVE_S16 if hist == "s16" else L.LBVE_F32
        d.pop_precision = L.LBVE_F32 if hist == "s16" else L.LBVE_F64
    return out


def time_steps(L, torch, descs, rho, K, W, Kp, stream, sync_ranks):
    """Create a handle, W untimed steps, K steps timed with CUDA events on `stream` (16-step graphs replayed),
    then Kp steps with per-launch events.  Returns (ms of the K steps, max over ranks; ms per sweep launch;
    ms per collide launch; (slot chunks, CTAs, CTA tasks))."""
    ch = L.Channel(descs if len(descs) > 1 else descs[0], rho)
    try:
        ch.step(W, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sync_ranks()
        e0.record(stream)
        ch.step(K, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        L.lbve_profile(ch.h, True)
        ch.step(Kp, stream)
        kms, launches = L.lbve_profile_read(ch.h)
        L.lbve_profile(ch.h, False)
        shape = L.lbve_sweep_config(ch.h)
    finally:
        ch.close()
    return ms, kms[1] / max(launches[1], 1), kms[2] / max(launches[2], 1), shape


def batch_arms(L, torch, configs, chosen: str, K: int, W: int, stream, sync_ranks, max_over_ranks, world: int,
               peak: float) -> dict:
    """The 64-channel batch workload (widths 8-512, L = 1024, 4000 + 2000 steps of which K are timed) in three
    arms: the chosen reduced-precision form batched (one launch sequence for all channels, 16-step graphs
    replayed), the plain FP32 form batched the same way, and the plain FP32 form with one handle per channel
    stepped one launch sequence per channel per step.  Ratios: the chosen batched form against the per-channel
    plain form (the batching variant's comparison) and against the batched plain form (equal launch mode)."""
    ws = configs.batched_channels()
    base = [w.desc() for w in ws]
    N = sum(w.N for w in ws)
    C_, B_ = ws[0].C, ws[0].B
    out = {"workload": f"batch64_channels_L{C_ * B_}", "nodes": N, "widths": [w.ny for w in ws]}
    fm, hs = chosen.split("_")
    arms = {"batched_chosen": form_descs(base, L, fm, hs), "batched_plain_f32": form_descs(base, L, "p", "f32")}
    pts = points_per_step(C_, B_, W, K, L)
    Kp = max(8, min(K, 64))
    pts_p = points_per_step(C_, B_, W + K, Kp, L)
    for name, dc in arms.items():
        ms, sweep_ms, _, shape = time_steps(L, torch, dc, None, K, W, Kp, stream, sync_ranks)
        ms = max_over_ranks(ms)
        bpu = bytes_per_update(2, dc[0].hist_storage, dc[0].hist_form, L)
        out[name] = {"form": FORM_NAMES[(fm, hs) if name == "batched_chosen" else ("p", "f32")],
                     "value": N * sum(pts) * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
                     "sweep_ms_per_launch": sweep_ms,
                     "roofline_frac": bpu * N * (sum(pts_p) - Kp) / Kp / (sweep_ms / 1e3) / 1e9 / peak,
                     "launches_per_step": 3, "sweep": {"slot_chunks": shape[0], "ctas": shape[1],
                                                         "tasks": ("warp", "cta", "balanced")[shape[2]]}}
    # the plain form as separate channels: one handle and one launch sequence per channel per step
    hs_ = [L.Channel(d) for d in arms["batched_plain_f32"]]
    try:
        Kq = max(4, K // 8)
        for h in hs_:
            h.step(2, stream)
        torch.cuda.synchronize()
        sync_ranks()
        t0 = time.perf_counter()
        for _ in range(Kq):
            for h in hs_:
                L.lbve_step(h.h, 1, stream)
        torch.cuda.synchronize()
        dtq = max_over_ranks(time.perf_counter() - t0)
    finally:
        for h in hs_:
            h.close()
    ptsq = points_per_step(C_, B_, 2, Kq, L)
    out["per_channel_plain_f32"] = {"form": FORM_NAMES["p", "f32"], "value": N * sum(ptsq) * world / dtq, "unit": UNIT,
                                    "ms_per_step": 1e3 * dtq / Kq, "launches_per_step": 3 * len(ws)}
    out["chosen_vs_plain_per_channel"] = out["batched_chosen"]["value"] / out["per_channel_plain_f32"]["value"]
    out["chosen_vs_plain_batched"] = out["batched_chosen"]["value"] / out["batched_plain_f32"]["value"]
    return out


def kernel_hash(files=("lbve_kernels.cuh", "lbve_sched.cuh")) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1504_06123_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


PROFILE_OF = {("channel", "nlm"): "sweep_channel_1024x512_L1024.md",
              ("channel", "wm"): "sweep_wm_channel_1024x512_L1024.md",
              ("channel", "inlm"): "collide_inlm_channel_4096x512.md",
              ("regime", "nlm"): "sweep_regime_10_channels_L1920.md"}


# the channel line's other history forms (bench.py's forms entries)
FORM_PROFILE = {"f_s16": "sweep_f16_channel_1024x512_L1024.md", "f_f32": "sweep_f_channel_1024x512_L1024.md",
                "p_s16": "sweep_s16_channel_1024x512_L1024.md"}


def recorded_profile(model: str = "nlm", workload: str = "channel", name: str | None = None) -> dict:
    """Figures of the committed ncu summary of the dominant kernel (dram_bytes_per_launch, and for an
    ALU-bound kernel fp64_thread_inst_per_node), if it was taken on the current source of that kernel (the
    summary names the source files its hash covers); {} otherwise."""
    name = name or PROFILE_OF.get((workload, model))
    p = os.path.join(ROOT, "profiles", name) if name else ""
    if not name or not os.path.exists(p):
        return {}
    kh, files, out = None, ("lbve_kernels.cuh", "lbve_sched.cuh"), {}
    for line in open(p):
        key, _, val = line.partition(":")
        if key == "kernel_source_sha256_16":
            kh = val.strip()
        elif key == "kernel_source_files":
            files = tuple(x.strip() for x in val.split(","))
        elif key in ("dram_bytes_per_launch", "fp64_thread_inst_per_node"):
            out[key] = float(val.strip())
    return out if kh == kernel_hash(files) else {}


def recorded_traffic(model: str = "nlm", workload: str = "channel"):
    return recorded_profile(model, workload).get("dram_bytes_per_launch")


def channel_workload(model: str):
    from paper_1504_06123_gb300 import configs
    return {"nlm": configs.plain_channel_large, "wm": configs.wm_channel_large,
            "inlm": configs.inlm_channel_large}[model]()


def oracle_sample(steps: int | None = None, budget_s: float = 12.0, warmup: int = 1, model: str = "nlm",
                  threads: int = 0):
    """The FP64 oracle on 2 columns x 512 rows of the benchmark channel with its full history: `warmup`
    untimed steps, then `steps` timed ones (or as many as fit in budget_s), its node loops on `threads` host
    threads (0: all cores).  Returns the rate in the workload's unit: node-history updates/s, or node
    updates/s for the instantaneous model, and the thread count used."""
    import oracle
    from paper_1504_06123_gb300 import inputs
    cores = oracle.set_threads(threads)
    w = channel_workload(model)
    nx = 2
    rho = inputs.initial_density(w.N, w.noise, w.seed).reshape(w.ny, w.nx)[:, :nx].ravel()
    ch = oracle.Channel(oracle.D2Q9, nx, w.ny, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                        g=(w.g, 0, 0), C=w.C, B=w.B, rho_init=rho,
                        model={"nlm": oracle.NLM, "wm": oracle.WM, "inlm": oracle.INLM}[model])
    t0 = time.perf_counter()
    ch.step(max(1, warmup))
    one = (time.perf_counter() - t0) / max(1, warmup)
    t_start = ch.t
    n = steps if steps is not None else max(2, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    ch.step(n)
    dt = time.perf_counter() - t0
    if model == "inlm":
        upd = nx * w.ny * n
    else:
        pts = [len(oracle.schedule(w.C, w.B, t)[0]) for t in range(t_start, t_start + n)]
        upd = nx * w.ny * sum(pts)
    ch.close()
    hist = "no history" if model == "inlm" else f"L = {w.L}"
    sample = (f"{nx} of {w.nx} columns x {w.ny} rows, {hist}, steps {t_start}..{t_start + n - 1} ({dt:.1f} s, "
              f"{cores} thread{'s' if cores > 1 else ''})")
    return upd / dt, sample, n, dt, upd, cores


def oracle_sample_batch(descs, steps: int, warmup: int = 1, threads: int = 0):
    """The FP64 oracle on one column (x-invariant flow) of each of the first two channels of a batch or
    duct workload, full width and history: `warmup` untimed steps, then `steps` timed ones, on `threads`
    host threads (0: all cores).  Returns the rate in node-history updates/s, a description of the sample
    and the thread count."""
    import oracle
    cores = oracle.set_threads(threads)
    chans = []
    for d in descs[:2]:
        lat = oracle.D2Q9 if d.lattice == 9 else oracle.D3Q19
        chans.append(oracle.Channel(lat, 1, d.ny, d.nz, tau_lb=d.tau_lb, G_inf=d.G_inf, tau=d.tau,
                                    gamma_c=d.gamma_c, g=tuple(d.g), C=d.hist_C, B=d.hist_B, wall_z=bool(d.wall_z),
                                    model={0: oracle.NLM, 2: oracle.WM}.get(d.model, oracle.NLM)))
    for ch in chans:
        ch.step(max(1, warmup))
    t_start = chans[0].t
    t0 = time.perf_counter()
    for ch in chans:
        ch.step(steps)
    dt = time.perf_counter() - t0
    d0 = descs[0]
    pts = [len(oracle.schedule(d0.hist_C, d0.hist_B, t)[0]) for t in range(t_start, t_start + steps)]
    nodes = sum(d.ny * d.nz for d in descs[:2])
    upd = nodes * sum(pts)
    for ch in chans:
        ch.close()
    sample = (f"one column of channels 0-{len(chans) - 1} ({nodes} nodes), L = {d0.hist_B * d0.hist_C}, "
              f"steps {t_start}..{t_start + steps - 1} ({dt:.1f} s, {cores} thread{'s' if cores > 1 else ''})")
    return upd / dt, sample, steps, dt, upd, cores


def run_reference(args, rank, world):
    if rank != 0:
        return
    metric = METRIC_NODES if args.model == "inlm" else METRIC
    if args.workload == "gradient":
        # the oracle's gradient is central finite differences: 8 forward runs of 4000 steps; timed on a
        # bounded sample (the first steps of one run) and scaled to the 32000 steps
        import oracle
        from paper_1504_06123_gb300 import configs
        cores = oracle.set_threads(0)
        w = configs.gradient_channel()
        ch = oracle.Channel(oracle.D2Q9, w.nx, w.ny, tau_lb=w.tau_lb, G_inf=w.G_inf, tau=w.tau, gamma_c=w.gamma_c,
                            g=(w.g, 0, 0), C=w.C, B=w.B)
        ch.step(max(1, args.warmup))
        n = max(2, args.steps if args.steps != 300 else 20)
        t0 = time.perf_counter()
        ch.step(n)
        dt = time.perf_counter() - t0
        ch.close()
        per_grad = dt / n * 8 * w.steps
        sample = (f"oracle steps {args.warmup}..{args.warmup + n - 1} of one run ({dt:.1f} s, {cores} threads), "
                  f"x 8 runs x {w.steps} steps")
        line = {"metric": "gradient evaluations/s", "value": 1.0 / per_grad, "unit": "gradient evaluations/s",
                "n_gpus": args.gpus, "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * per_grad,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference", "config": {"workload": "gradient_channel_4x128_L512_4000steps", "sample": sample},
                "cpu_baseline": {"value": 1.0 / per_grad, "unit": "gradient evaluations/s", "cores": cores,
                                 "kind": "oracle", "sample": sample},
                "e2e": {"value": 1.0 / per_grad, "unit": "gradient evaluations/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "gpu_launches": 0}
        print(json.dumps(line), flush=True)
        return
    if args.workload != "channel":
        from paper_1504_06123_gb300 import configs
        from paper_1504_06123_gb300 import lbve as L
        name, descs, _, _ = workload_descs(args, L, configs)
        val, sample, n, dt, upd, cores = oracle_sample_batch(descs, steps=args.steps, warmup=args.warmup)
        line = {
            "metric": metric, "value": val, "unit": metric, "n_gpus": args.gpus, "steps": n,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / n, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": name, "sample": sample},
            "cpu_baseline": {"value": val, "unit": metric, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": metric, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0,
        }
        print(json.dumps(line), flush=True)
        return
    # each step: one oracle step of the sample (about 0.1 s on one core), on all host cores
    val, sample, n, dt, upd, cores = oracle_sample(steps=args.steps, warmup=args.warmup, model=args.model)
    line = {
        "metric": metric, "value": val, "unit": metric, "n_gpus": args.gpus, "steps": n, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": channel_workload(args.model).name, "sample": sample},
        "cpu_baseline": {"value": val, "unit": metric, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": metric, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def workload_descs(args, L, configs):
    """(name, descs, rho_init, notes) of the selected workload."""
    if args.model == "inlm" and args.workload != "channel":
        raise SystemExit("--model inlm is measured on the channel workload")
    model = {"nlm": L.LBVE_MODEL_NLM, "wm": L.LBVE_MODEL_WM, "inlm": L.LBVE_MODEL_INLM}[args.model]
    if args.workload == "channel":
        w = channel_workload(args.model)
        if args.nx:
            w.nx = args.nx
        suffix = {"nlm": "", "wm": "_wm"}.get(args.model)
        name = f"channel_{w.nx}x{w.ny}_inlm" if suffix is None else f"channel_{w.nx}x{w.ny}_L{w.L}{suffix}"
        return name, [w.desc()], w.rho_init(), {
            "lattice": "D2Q9", "blocks_B": w.B, "block_C": w.C, "tau_lb": w.tau_lb, "G_inf": w.G_inf, "tau": w.tau,
            "gamma_c": w.gamma_c, "g": w.g}
    if args.workload == "duct":
        w = configs.duct_3d()
        if args.nx:
            w.nx = args.nx
        w.model = model
        return f"duct_{w.nx}x{w.ny}x{w.nz}_L{w.L}" + ("_wm" if args.model == "wm" else ""), [w.desc()], w.rho_init(), {
            "lattice": "D3Q19", "blocks_B": w.B, "block_C": w.C, "tau_lb": w.tau_lb, "G_inf": w.G_inf, "tau": w.tau,
            "gamma_c": w.gamma_c, "g": w.g}
    if args.workload == "regime":
        from paper_1504_06123_gb300 import regime
        pts = regime.paper_points()
        chans, descs, B = regime.sweep_descs(pts, regime.tau0_for_width(100), nx=4)
        for d in descs:
            d.model = model
        return f"paper_regime_{len(descs)}_channels_L{B * descs[0].hist_C}", descs, None, {
            "lattice": "D2Q9", "channels": len(descs), "widths": [c.ny for c in chans], "nx": 4,
            "t_wall_over_tau0": [c.ratio for c in chans], "theta": [c.theta for c in chans],
            "blocks_B": B, "block_C": descs[0].hist_C,
            "probes": "u, rho, sigma at the two nodes around y/H = 0.51 of every channel, recorded every step"}
    ws = configs.batched_channels()
    for w in ws:
        w.model = model
    return f"batch64_channels_L{ws[0].L}" + ("_wm" if args.model == "wm" else ""), [w.desc() for w in ws], None, {
        "lattice": "D2Q9", "channels": len(ws), "widths": [w.ny for w in ws], "blocks_B": ws[0].B,
        "block_C": ws[0].C}


def run_gradient(args, rank, world, local_rank):
    """The differentiation workload: one gradient = the recording forward run (a state image every 64 steps)
    plus lbve_backward, timed end to end with CUDA events on the stream; the tangent-linear model on the
    same workload beside it.  Metric: gradient evaluations per second (and node-history updates/s of the
    forward steps they contain)."""
    import torch
    import numpy as np
    from paper_1504_06123_gb300 import configs, inputs
    from paper_1504_06123_gb300 import lbve as L
    from paper_1504_06123_gb300.autograd import run_profiles
    torch.cuda.set_device(local_rank)
    w = configs.gradient_channel()
    if args.lb_steps:
        w.steps = args.lb_steps
    # the workload's precision is FP32: the plain FP32 form (FP32 history, FP64 populations, as in every FP32
    # workload here: FP32 populations drift by their rounding over 4000 steps); --history f64: the FP64 model
    prec = L.LBVE_F64 if args.history == "f64" else L.LBVE_F32
    desc = w.desc(precision=L.LBVE_F64, hist_storage=prec)
    desc64 = w.desc(precision=L.LBVE_F64, hist_storage=L.LBVE_F64)
    theta = np.array([w.G_inf, w.tau, w.gamma_c, w.g])
    ut, st = run_profiles(desc64, inputs.perturbed(theta, seed=w.seed), w.steps)
    N = w.nx * w.ny
    K = args.steps if args.steps != 300 else 3
    W = args.warmup if args.warmup != 5 else 1
    stream = torch.cuda.current_stream()
    su, ss = float(np.max(np.abs(ut))) ** 2, float(np.max(np.abs(st))) ** 2

    def gradient(desc=desc):
        h = L.lbve_create_adjoint(desc, None, 64)
        try:
            L.lbve_step(h, w.steps, stream)
            f = L.lbve_fields(h, L.LBVE_FIELD_U | L.LBVE_FIELD_SIGMA, None, stream)
            u, sxy = f[:N], f[2 * N + 2 * N: 2 * N + 3 * N]
            du = np.zeros((2, N))
            ds = np.zeros((3, N))
            du[0] = 2.0 * (u - ut) / (N * su)          # d/du of mean((u - u*)^2) / max|u*|^2
            ds[2] = 2.0 * (sxy - st) / (N * ss)
            return L.lbve_backward(h, du, ds, stream)
        finally:
            L.lbve_destroy(h)

    for _ in range(W):
        gradient()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        for _ in range(K):
            g = gradient()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    # the other precision's gradient (one evaluation), the tangent-linear model (FP64, forward mode: all four
    # derivatives in one run) and the plain forward of the same precision, for the ratio backward / forward
    other = desc64 if prec == L.LBVE_F32 else w.desc(precision=L.LBVE_F64, hist_storage=L.LBVE_F32)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    g_other = gradient(other)
    torch.cuda.synchronize()
    dt_other = time.perf_counter() - t3
    t1 = time.perf_counter()
    run_profiles(desc64, theta, w.steps, with_tangents=True)
    torch.cuda.synchronize()
    dt_tan = time.perf_counter() - t1
    run_profiles(desc, theta, w.steps)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    run_profiles(desc, theta, w.steps)
    torch.cuda.synchronize()
    dt_fwd = time.perf_counter() - t2
    pts = points_per_step(desc.hist_C, desc.hist_B, 0, w.steps, L)
    upd = N * sum(pts)
    value = K / dt
    if rank == 0:
        line = {
            "metric": "gradient evaluations/s", "value": value, "unit": "gradient evaluations/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * dt / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == L.LBVE_F64 else "f32", "data": "synthetic",
            "config": {"workload": f"gradient_channel_4x128_L512_{w.steps}steps", "nodes": N,
                       "precision": ("FP64 history" if prec == L.LBVE_F64 else "FP32 history") +
                                    ", FP64 populations (the adjoint itself in FP64)",
                       "history_points": desc.hist_B * desc.hist_C, "lb_steps": w.steps, "checkpoint_every": 64,
                       "loss": "mean((u_x - u*)^2)/max|u*|^2 + mean((sigma_xy - s*)^2)/max|s*|^2, final step",
                       "parallelism": f"replicas{world}", "l2": "state fits in L2 (latency-bound size)"},
            "gradient": [float(x) for x in g],
            "other_precision": {"precision": "FP64" if prec == L.LBVE_F32 else "FP32",
                                "gradient": [float(x) for x in g_other], "gradient_s": dt_other},
            "forward_updates_per_s": upd * K / dt,
            "plain_forward_s": dt_fwd, "gradient_s": dt / K, "gradient_over_forward": (dt / K) / dt_fwd,
            "tangent_s": dt_tan,
            "clocks": clk.summary(), "roofline": None, "cpu_baseline": None, "e2e": None,
        }
        print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1504_06123_gb300 import configs
    from paper_1504_06123_gb300 import lbve as L

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1504_06123_gb300 import ranks

    def max_over_ranks(x: float) -> float:
        return ranks.max_over_ranks(x, dist if world > 1 else None, device="cuda")

    name, descs, rho, notes = workload_descs(args, L, configs)
    if args.drive == "pressure":
        for d in descs:
            d.x_boundary = L.LBVE_X_PRESSURE
            d.dp = d.rho0 * d.g[0] * d.nx
            d.g[0] = 0.0
        name += "_pressure"
        notes = dict(notes, drive="pressure-step boundary along x, dp = rho0 g nx per period")
    hist = {"f32": L.LBVE_F32, "s16": L.LBVE_S16, "f64": L.LBVE_F64}[args.history]
    form = L.LBVE_FORM_F if args.form == "f" else L.LBVE_FORM_P
    for d in descs:
        d.hist_storage = hist
        d.hist_form = form
        if hist == L.LBVE_S16:
            # the reduced-precision form: FP32 populations are well inside its 1e-3 budget
            d.pop_precision = L.LBVE_F32
    inst = args.model == "inlm"
    wm = args.model == "wm"
    if wm and hist == L.LBVE_S16:
        raise SystemExit("the White-Metzner form has no 16-bit history")
    if wm and form == L.LBVE_FORM_F:
        raise SystemExit("the White-Metzner form has no factor-storage history")
    metric = METRIC_NODES if inst else METRIC
    d0 = descs[0]
    N = sum(d.nx * d.ny * d.nz for d in descs)
    D = 2 if d0.lattice == L.LBVE_D2Q9 else 3
    Q = d0.lattice
    bpu = bytes_per_update(D, d0.hist_storage, form, L, wm)
    # the collide kernel, per node: populations in and out, u_raw, sigma, kappa, rho, u out, tr_prev in/out
    pop_bytes = 8 if d0.pop_precision == L.LBVE_F64 else 4
    NS = 3 if D == 2 else 6
    collide_bytes_per_node = 2 * Q * pop_bytes + 8 * (D + NS + D * D + 1 + D + 2)
    stream = torch.cuda.current_stream()
    ch = L.Channel(descs if len(descs) > 1 else descs[0], rho)
    K, W = args.steps, args.warmup
    if args.sweep_shape:
        S_pin, cta_pin = (int(v) for v in args.sweep_shape.split(","))
        L.lbve_set_sweep_config(ch.h, S_pin, cta_pin)
    probes = 0
    if args.workload == "regime":
        from paper_1504_06123_gb300 import regime
        chans = [regime.regime_channel(r, th, d.ny) for (r, th), d in zip(regime.paper_points(), descs)]
        offs = [L.lbve_channel_nodes(ch.h, k)[0] for k in range(len(descs))]
        pnodes, _ = regime.probe_plan(chans, offs, descs[0].nx)
        probes = len(pnodes)
        L.lbve_set_probes(ch.h, pnodes, 1, W + K + max(8, min(K, 64)) + 1)
    ch.step(W, stream)
    torch.cuda.synchronize()
    if inst:
        updates_rank = N * K
    else:
        pts = points_per_step(d0.hist_C, d0.hist_B, W, K, L)
        updates_rank = N * sum(pts)

    # timed region: K steps as a user runs them (16-step graphs replayed)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        ch.step(K, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    value = ranks.job_rate(updates_rank, world, ms_max / 1e3)
    mlups = N * K * world / (ms_max / 1e3) / 1e6

    # per-kernel device time from events around every launch of a further profiled segment
    Kp = max(8, min(K, 64))
    L.lbve_profile(ch.h, True)
    ch.step(Kp, stream)
    kms, launches = L.lbve_profile_read(ch.h)
    L.lbve_profile(ch.h, False)
    hist_ms = kms[1] / max(launches[1], 1)
    coll_ms = kms[2] / max(launches[2], 1)
    peak, peak_kind = peaks()
    roof_extra = {}
    if inst:   # no history: the collide kernel (with the stress series) is the dominant kernel
        alg_bytes = collide_bytes_per_node * N
        achieved = alg_bytes / (coll_ms / 1e3) / 1e9
        roof_kernel = "k_collide_stream"
        state_bytes = 2 * Q * pop_bytes * N
    else:
        pts_p = points_per_step(d0.hist_C, d0.hist_B, W + K, Kp, L)
        alg_bytes = bpu * N * (sum(pts_p) - Kp) / Kp   # the new point is not read from memory
        achieved = alg_bytes / (hist_ms / 1e3) / 1e9
        roof_kernel = {(L.LBVE_FORM_P, True): "k_sweep_s16", (L.LBVE_FORM_P, False): "k_sweep",
                       (L.LBVE_FORM_F, True): "k_sweep_f16", (L.LBVE_FORM_F, False): "k_sweep_f"}[
                           (form, d0.hist_storage == L.LBVE_S16)]
        state_bytes = alg_bytes
    prof = (recorded_profile(args.model, args.workload)
            if not args.nx and args.history == "f32" and args.form == "p" else {})
    traffic = prof.get("dram_bytes_per_launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "kernel": roof_kernel,
                "algorithmic_bytes_per_launch": alg_bytes}
    if inst and d0.pop_precision == L.LBVE_F64 and "fp64_thread_inst_per_node" in prof:
        # bound by the FP64 pipe: 2 FP64 thread instructions per SM per cycle (GB300), 152 SMs, at the
        # sampled SM clock; the instruction count per node is the ncu count of the committed capture
        sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
        inst_s = prof["fp64_thread_inst_per_node"] * N / (coll_ms / 1e3) / 1e9
        roofline = {"bound": "alu", "achieved": inst_s, "peak": None, "unit": "G FP64 thread inst/s",
                    "frac": None, "traffic": traffic, "peak_kind": "derived: 2 FP64 inst / SM / cycle x "
                    f"{sms} SMs x sampled SM clock", "kernel": roof_kernel,
                    "fp64_thread_inst_per_node": prof["fp64_thread_inst_per_node"],
                    "hbm_frac": achieved / peak, "algorithmic_bytes_per_launch": alg_bytes}
    S, ctas, cta_tasks = L.lbve_sweep_config(ch.h) if not inst else (0, 0, 0)
    ch.close()

    extra = {}
    if (args.workload in ("channel", "duct") and args.history == "f32" and args.form == "p" and not args.no_chosen
            and args.model == "nlm"):
        # every other history form on the same workload (the line's own run is form P with the FP32 history);
        # chosen = the fastest of them that meets the reduced-precision bar (1e-3)
        pts_f = sum(pts_p) - Kp
        forms = {"p_f32": {"form": FORM_NAMES["p", "f32"], "value": value, "unit": UNIT, "ms_per_step": ms_max / K,
                           "sweep_ms_per_launch": hist_ms, "bytes_per_update": bpu, "roofline_frac": achieved / peak,
                           "parity_bar": FORM_BAR["p", "f32"]}}
        for fm, hs in (("p", "s16"), ("f", "f32"), ("f", "s16")):
            dc = form_descs(descs, L, fm, hs)
            msc, sweep_c, coll_c, shape_c = time_steps(L, torch, dc, rho, K, W, Kp, stream, barrier)
            msc = max_over_ranks(msc)
            bpu_c = bytes_per_update(D, dc[0].hist_storage, dc[0].hist_form, L)
            traffic_c = (recorded_profile(name=FORM_PROFILE.get(f"{fm}_{hs}")).get("dram_bytes_per_launch")
                         if args.workload == "channel" and not args.nx else None)
            forms[f"{fm}_{hs}"] = {"form": FORM_NAMES[fm, hs], "value": updates_rank * world / (msc / 1e3),
                                   "traffic": traffic_c,
                                   "unit": UNIT, "ms_per_step": msc / K, "sweep_ms_per_launch": sweep_c,
                                   "collide_ms_per_launch": coll_c, "bytes_per_update": bpu_c,
                                   "roofline_frac": bpu_c * N * pts_f / Kp / (sweep_c / 1e3) / 1e9 / peak,
                                   "sweep": {"slot_chunks": shape_c[0], "ctas": shape_c[1],
                                             "tasks": ("warp", "cta", "balanced")[shape_c[2]]},
                                   "parity_bar": FORM_BAR[fm, hs]}
        best = max((k for k in forms if k != "p_f32"), key=lambda k: forms[k]["value"])
        extra = {"forms": forms, "chosen": dict(forms[best], key=best),
                 "chosen_vs_plain": forms[best]["value"] / value}
        if args.workload == "channel" and not args.no_batch and not args.nx:
            extra["batch64"] = batch_arms(L, torch, configs, best, K, W, stream, barrier, max_over_ranks, world, peak)
    if inst and not args.no_chosen:
        # the instantaneous model with FP32 populations (the series summed in float): its collision runs on
        # the FP32 pipe instead of the FP64 one; parity bar of the all-FP32 form 5e-5
        import copy as _copy
        dc = _copy.copy(d0)
        dc.pop_precision = L.LBVE_F32
        chc = L.Channel(dc, rho)
        chc.step(W, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        chc.step(K, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        msc = max_over_ranks(e0.elapsed_time(e1))
        L.lbve_profile(chc.h, True)
        chc.step(Kp, stream)
        kmc, lnc = L.lbve_profile_read(chc.h)
        L.lbve_profile(chc.h, False)
        chc.close()
        coll_c = kmc[2] / max(lnc[2], 1)
        bytes_c = (2 * Q * 4 + 8 * (D + NS + D * D + 1 + D + 2)) * N
        chosen_value = updates_rank * world / (msc / 1e3)
        extra = {"chosen": {"form": "f32 populations, series of Eq. (inlM) summed in float", "value": chosen_value,
                            "unit": metric, "ms_per_step": msc / K, "collide_ms_per_launch": coll_c,
                            "roofline_frac": bytes_c / (coll_c / 1e3) / 1e9 / peak, "parity_bar": 5e-5},
                 "chosen_vs_plain": chosen_value / value}
    if args.workload == "batched":
        # the plain form: one handle per channel, each stepped with its own launches (no batching, no graphs)
        hs = [L.Channel(d) for d in descs]
        Kq = max(4, K // 8)
        for h in hs:
            h.step(2, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Kq):
            for h in hs:
                L.lbve_step(h.h, 1, stream)
        torch.cuda.synchronize()
        dtq = max_over_ranks(time.perf_counter() - t0)
        ptsq = points_per_step(d0.hist_C, d0.hist_B, 2, Kq, L)
        plain = N * sum(ptsq) * world / dtq
        for h in hs:
            h.close()
        extra = {"plain_per_channel": {"value": plain, "unit": UNIT, "ms_per_step": 1e3 * dtq / Kq,
                                       "launches_per_step": 3 * len(descs)},
                 "chosen_vs_plain": value / plain}

    # end to end through the public C ABI, as a user runs the workload: create from the host initial
    # density (H2D), advance K steps, read u and sigma back to pinned host memory (D2H), destroy
    e2e = None
    if not args.no_e2e:
        mask = L.LBVE_FIELD_U | L.LBVE_FIELD_SIGMA
        host = torch.empty((D + (3 if D == 2 else 6)) * N, dtype=torch.float64, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = L.lbve_create_batch(descs, rho) if len(descs) > 1 else L.lbve_create(d0, rho)
        probe_bytes = 0
        if probes:   # the sweep as a user runs it: probes recorded every step, read back at the end
            L.lbve_set_probes(h, pnodes, 1, K)
        L.lbve_step(h, K, stream)
        rc = L.load().lbve_fields(h, mask, host.data_ptr(), 0, int(stream.cuda_stream) or None)
        if probes and rc == 0:
            _, pv, _ = L.lbve_probe_read(h, probes, D, K, stream)
            probe_bytes = 8 * (pv.size + len(pv))
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0)
        L.lbve_destroy(h)
        if rc != 0:
            raise RuntimeError(f"lbve_fields failed: {rc}")
        upd_e = N * K if inst else N * sum(points_per_step(d0.hist_C, d0.hist_B, 0, K, L))
        e2e = {"value": upd_e * world / dt, "unit": metric,
               "h2d_bytes_per_step": (8 * N if rho is not None else 0) / K,
               "d2h_bytes_per_step": (8 * host.numel() + probe_bytes) / K, "steps": K,
               "includes": "create (allocation, autotune, initial density upload), K steps, field read" +
                           (", probe records read" if probes else "") + ", destroy"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "channel":
        # the oracle on all host cores (its node loops split over OpenMP threads), and on one core
        val, sample, _, _, _, cores = oracle_sample(model=args.model, budget_s=8.0, threads=0)
        val1, sample1, _, _, _, _ = oracle_sample(model=args.model, budget_s=8.0, threads=1)
        cpu = {"value": val, "unit": metric, "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": {"value": val1, "unit": metric, "cores": 1, "sample": sample1}}

    clocks = clk.summary()
    if roofline["bound"] == "alu":
        mhz = clocks["sm_mhz"] or clocks["sm_max_mhz"] or 2070.0
        roofline["peak"] = 2 * sms * mhz * 1e6 / 1e9
        roofline["frac"] = roofline["achieved"] / roofline["peak"]
    if rank == 0:
        prec = {L.LBVE_F32: "f32", L.LBVE_F64: "f64", L.LBVE_S16: "s16 (16-bit block-scaled, f32 math)"}
        model_name = {"nlm": "integral nlM, Eqs. (gitt), (nlmax)", "wm": "White-Metzner form of Eq. (nlmax)",
                      "inlm": "instantaneous nlM, Eq. (inlM): no history"}[args.model]
        line = {
            "metric": metric, "value": value, "unit": metric, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {L.LBVE_S16: "s16"}.get(d0.hist_storage, prec.get(d0.hist_storage, "f32")), "data": "synthetic",
            "config": dict({"workload": name, "nodes": N, "history_points": 0 if inst else d0.hist_C * d0.hist_B,
                            "model": model_name,
                            "precision": (f"no history; populations {prec.get(d0.pop_precision)}" if inst else
                                          f"history (E-1, kappa) {prec.get(d0.hist_storage)} storage and arithmetic; "
                                          f"populations {prec.get(d0.pop_precision)}"),
                            "parallelism": f"replicas{world}",
                            "l2": ("no flush: per-step state (" + ("populations" if inst else "history") +
                                   f", {state_bytes / 1e6:.0f} MB) larger than the 129 MB L2")
                                  if state_bytes > 2.5e8 else "state fits in L2 (latency-bound size)",
                            "sweep": {"slot_chunks": S, "ctas": ctas, "tasks": ("warp", "cta", "balanced")[cta_tasks]}},
                           **notes),
            "mlups": mlups,
            "kernel_ms_per_launch": {"moments": kms[0] / max(launches[0], 1), "history": hist_ms,
                                     "collide_stream": kms[2] / max(launches[2], 1)},
            "roofline": roofline,
            "clocks": clocks,
            "gpu_launches": ((2 if inst else 3) + (1 if probes else 0)) * K,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "gradient":
        run_gradient(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
