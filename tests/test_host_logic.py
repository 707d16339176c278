"""Host-side logic on the CPU: argument checks of the newer entry points that must fail before any device
work, and the benchmark's reference arm (the FP64 oracle on a bounded sample) for every workload, whose
JSON line must carry the contract's keys."""
import json
import os
import subprocess
import sys

import pytest

from paper_1504_06123_gb300 import lbve as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_null_handles_are_rejected():
    lib = L.load()
    import ctypes as C
    i64 = C.c_int64
    assert lib.lbve_set_probes(None, 0, None, 1, 1) == L.LBVE_EINVAL
    k, tot = i64(), i64()
    buf = (C.c_double * 4)()
    assert lib.lbve_probe_read(None, buf, C.byref(k), C.byref(tot), None) == L.LBVE_EINVAL
    assert lib.lbve_set_sweep_config(None, 1, 0) == L.LBVE_EINVAL
    s, g, m = C.c_int32(), C.c_int32(), C.c_int32()
    assert lib.lbve_sweep_config(None, C.byref(s), C.byref(g), C.byref(m)) == L.LBVE_EINVAL


def test_allocator_without_free_is_rejected_before_device_work():
    d = L.make_desc(nx=2, ny=4, C=8, B=2)
    half = L.lbve_allocator(L.ALLOC_FN(lambda n, s, c: None), L.FREE_FN(), None)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_ex([d], None, half)
    assert e.value.status == L.LBVE_EINVAL
    bad = L.make_desc(nx=2, ny=1, C=8, B=2)            # invalid description: refused first
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_ex([bad], None, L.make_allocator(lambda n, s: 0, lambda p, s: None))
    assert e.value.status == L.LBVE_EINVAL


@pytest.mark.parametrize("workload", ["channel", "regime", "batched", "gradient"])
def test_reference_arm_prints_one_contract_line(workload):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload,
           "--steps", "2", "--warmup", "1"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]
