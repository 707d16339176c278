"""The C-ABI library on the CPU: it builds, loads, exports every entry point of include/lbve.h, validates
arguments before touching a GPU, and its history grid (the kernel's per-slot roles, run on the host) is
bit-identical to the oracle's merge simulation (Sec. III quasi-logarithmic layout)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1504_06123_gb300 import lbve as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbve_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_header_function():
    lib = L.load()
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTS) == names


def test_strerror():
    assert L.lbve_strerror(0) == "ok"
    assert "invalid" in L.lbve_strerror(L.LBVE_EINVAL)
    assert L.lbve_strerror(12345) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(tau_lb=0.5), dict(ny=1), dict(nx=0), dict(C=3), dict(B=0), dict(B=17), dict(tau=0.0),
    dict(G_inf=-1.0), dict(gamma_c=0.0), dict(G_inf=0.3), dict(nz=2), dict(C=4096, B=2), dict(model=3),
    dict(model=-1),
])
def test_create_rejects_bad_descriptions(bad):
    kw = dict(lattice=L.LBVE_D2Q9, nx=4, ny=8, tau_lb=0.9, G_inf=0.01, tau=100.0, gamma_c=0.1, C=8, B=2)
    kw.update(bad)
    d = L.make_desc(**kw)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(d)
    assert e.value.status == L.LBVE_EINVAL


def test_unsupported_variant_combinations_are_refused_before_any_device_work():
    """White-Metzner with the 16-bit history, and differentiation of the two constitutive variants, are
    valid requests this library does not implement (LBVE_ENOSUPPORT); a batch mixing models is invalid."""
    wm16 = L.make_desc(nx=2, ny=4, C=8, B=2, precision=L.LBVE_F32, hist_storage=L.LBVE_S16, model=L.LBVE_MODEL_WM)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(wm16)
    assert e.value.status == L.LBVE_ENOSUPPORT
    for model in (L.LBVE_MODEL_INLM, L.LBVE_MODEL_WM):
        d = L.make_desc(nx=2, ny=4, C=8, B=2, precision=L.LBVE_F64, model=model)
        with pytest.raises(L.LbveError) as e:
            L.lbve_create_tangent(d)
        assert e.value.status == L.LBVE_ENOSUPPORT
        with pytest.raises(L.LbveError) as e:
            L.lbve_create_adjoint(d)
        assert e.value.status == L.LBVE_ENOSUPPORT
    mixed = [L.make_desc(nx=2, ny=4, C=8, B=2), L.make_desc(nx=2, ny=4, C=8, B=2, model=L.LBVE_MODEL_WM)]
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_batch(mixed)
    assert e.value.status == L.LBVE_EINVAL


def test_pressure_boundary_arguments_are_checked_before_any_device_work():
    import ctypes
    bad = L.make_desc(nx=2, ny=4, C=8, B=2, dp=float("nan"))
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(bad)
    assert e.value.status == L.LBVE_EINVAL
    d = L.make_desc(nx=2, ny=4, C=8, B=2)
    d.x_boundary = 2
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(d)
    assert e.value.status == L.LBVE_EINVAL
    p = L.make_desc(nx=2, ny=4, C=8, B=2, precision=L.LBVE_F64, dp=1e-6)
    for fn in (L.lbve_create_tangent, L.lbve_create_adjoint):
        with pytest.raises(L.LbveError) as e:
            fn(p)
        assert e.value.status == L.LBVE_ENOSUPPORT
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_pressure_step(0, 1e-6)
    assert e.value.status == L.LBVE_EINVAL
    # the C layout: dp follows x_boundary at an 8-byte boundary (the whole layout is compared with the
    # header's struct in test_desc_layout_matches_the_header)
    assert L.lbve_channel_desc.dp.offset % 8 == 0
    assert ctypes.sizeof(L.lbve_channel_desc) % 8 == 0


def test_create_rejects_nonfinite_density():
    d = L.make_desc(nx=2, ny=4, C=8, B=1)
    rho = np.ones(8)
    rho[3] = np.nan
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(d, rho)
    assert e.value.status == L.LBVE_EINVAL


@pytest.mark.parametrize("C,B", [(4, 1), (4, 2), (4, 3), (6, 4), (8, 5), (128, 8), (256, 1), (64, 4), (5, 3),
                                 (128, 4), (7, 16)])
def test_schedule_bit_exact_vs_oracle(C, B):
    ts = list(range(0, 80)) + [127, 128, 129, 255, 1023, 1024, 4097, 32767, 32768, 100000]
    for t in ts:
        tp, w = L.lbve_schedule(C, B, t)
        otp, ow = oracle.schedule(C, B, t)
        assert np.array_equal(tp, otp), (C, B, t)
        assert np.array_equal(w, ow), (C, B, t)


def test_schedule_rejects_bad_args():
    with pytest.raises(L.LbveError):
        L.lbve_schedule(3, 2, 0)
    with pytest.raises(L.LbveError):
        L.lbve_schedule(8, 2, -1)


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d = L.make_desc(nx=2, ny=4, C=8, B=1)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(d)
    assert e.value.status in (L.LBVE_ECUDA, L.LBVE_ENOMEM)


def test_desc_layout_matches_the_header(tmp_path):
    """The binding's ctypes mirror of lbve_channel_desc has the C struct's size and field offsets."""
    import subprocess
    fields = [f[0] for f in L.lbve_channel_desc._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbve.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(lbve_channel_desc));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(lbve_channel_desc, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    import ctypes as C
    assert out[0] == C.sizeof(L.lbve_channel_desc)
    for f, off in zip(fields, out[1:]):
        assert getattr(L.lbve_channel_desc, f).offset == off, f


def test_factor_form_arguments_are_checked_before_any_device_work():
    """hist_form outside {P, F} is invalid; the factor form with the White-Metzner model, and differentiation
    of a factor-form channel, are valid requests this library does not implement."""
    bad = L.make_desc(nx=2, ny=4, C=8, B=2, hist_form=2)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(bad)
    assert e.value.status == L.LBVE_EINVAL
    wm = L.make_desc(nx=2, ny=4, C=8, B=2, model=L.LBVE_MODEL_WM, hist_form=L.LBVE_FORM_F)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(wm)
    assert e.value.status == L.LBVE_ENOSUPPORT
    f64 = L.make_desc(nx=2, ny=4, C=8, B=2, precision=L.LBVE_F64, hist_form=L.LBVE_FORM_F)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_tangent(f64)
    assert e.value.status == L.LBVE_ENOSUPPORT
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_adjoint(f64, None, 8)
    assert e.value.status == L.LBVE_ENOSUPPORT
    mixed = [L.make_desc(nx=2, ny=4, C=8, B=2), L.make_desc(nx=2, ny=4, C=8, B=2, hist_form=L.LBVE_FORM_F)]
    with pytest.raises(L.LbveError) as e:
        L.lbve_create_batch(mixed)
    assert e.value.status == L.LBVE_EINVAL
