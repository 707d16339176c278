"""ctypes binding of the C ABI in ``include/lbve.h`` -- argument marshalling only.

Every step of the method runs in the CUDA library ``_build/liblbve.so``; this module converts Python
values to the C structures and raises :class:`LbveError` on a non-zero status.  Function names are the
C names.  Device pointers may be passed as ints or as torch CUDA tensors (their ``data_ptr()``);
streams as ints, ``torch.cuda.Stream`` objects or ``None`` (the current torch stream when torch is
initialised on CUDA, else the legacy default stream).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

LBVE_OK, LBVE_EINVAL, LBVE_ENOMEM, LBVE_ECUDA, LBVE_ENONFINITE, LBVE_ESTATE, LBVE_ENOSUPPORT = 0, -1, -2, -3, -4, -6, -7
LBVE_ETOOBIG = -8
LBVE_FIXED_STAGING_DOUBLES = 1 << 21
LBVE_D2Q9, LBVE_D3Q19 = 9, 19
LBVE_F32, LBVE_F64, LBVE_BF16, LBVE_S16 = 0, 1, 2, 3
LBVE_TRACE_FULL, LBVE_TRACE_NONE = 0, 1
LBVE_FORM_P, LBVE_FORM_F = 0, 1
LBVE_MODEL_NLM, LBVE_MODEL_INLM, LBVE_MODEL_WM = 0, 1, 2
LBVE_X_PERIODIC, LBVE_X_PRESSURE = 0, 1
LBVE_FIELD_RHO, LBVE_FIELD_U, LBVE_FIELD_SIGMA, LBVE_FIELD_KAPPA, LBVE_FIELD_N1 = 1, 2, 4, 8, 16

# Every entry point declared in include/lbve.h (checked by the tests against the header).
EXPORTS = [
    "lbve_create", "lbve_destroy", "lbve_set_force", "lbve_set_params", "lbve_step", "lbve_get_time",
    "lbve_fields", "lbve_fields_count", "lbve_history_apply", "lbve_mass", "lbve_schedule",
    "lbve_memory_bytes", "lbve_strerror", "lbve_last_cuda_error", "lbve_profile", "lbve_profile_read",
    "lbve_fields_host_fixed", "lbve_create_batch", "lbve_channel_nodes", "lbve_sweep_config",
    "lbve_create_tangent", "lbve_tangent_fields", "lbve_checkpoint_size", "lbve_checkpoint_save",
    "lbve_checkpoint_restore", "lbve_create_adjoint", "lbve_backward", "lbve_set_pressure_step",
    "lbve_set_probes", "lbve_probe_read", "lbve_set_sweep_config", "lbve_create_ex", "lbve_fields_ex",
]


class lbve_channel_desc(C.Structure):
    _fields_ = [
        ("lattice", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("wall_z", C.c_int32),
        ("tau_lb", C.c_double), ("rho0", C.c_double), ("G_inf", C.c_double), ("tau", C.c_double),
        ("gamma_c", C.c_double), ("g", C.c_double * 3), ("hist_C", C.c_int32), ("hist_B", C.c_int32),
        ("hist_storage", C.c_int32), ("pop_precision", C.c_int32), ("trace_coupling", C.c_int32),
        ("model", C.c_int32), ("x_boundary", C.c_int32), ("dp", C.c_double), ("hist_form", C.c_int32),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class lbve_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


def make_allocator(alloc, free) -> lbve_allocator:
    """lbve_allocator calling alloc(bytes, stream) -> device pointer (int, 0/None on failure) and
    free(ptr, stream); stream is the raw cudaStream_t as an int, or None for the legacy default stream.
    Exceptions inside the callbacks count as a failed allocation (alloc) or are dropped (free)."""
    def _alloc(n, stream, ctx):
        try:
            return alloc(int(n), stream) or None
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            free(ptr, stream)
        except Exception:
            pass

    return lbve_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)


def torch_allocator(device: int | None = None) -> lbve_allocator:
    """lbve_allocator on PyTorch's CUDA caching allocator (blocks are 512-byte aligned)."""
    import torch
    dev = torch.cuda.current_device() if device is None else device
    return make_allocator(lambda n, stream: torch.cuda.caching_allocator_alloc(n, dev, stream),
                          lambda ptr, stream: torch.cuda.caching_allocator_delete(ptr))


class LbveError(RuntimeError):
    def __init__(self, status: int, where: str, lib=None):
        msg = f"{where}: {lbve_strerror(status) if lib is not None else status} ({status})"
        if status == LBVE_ECUDA and lib is not None:
            msg += " -- " + lib.lbve_last_cuda_error().decode()
        super().__init__(msg)
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load liblbve.so (building it first if it is missing or stale).  Raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _build.build()
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not found at {p}; run paper_1504_06123_gb300.build.build()")
        lib = C.CDLL(p)
        vp, dp, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64
        lib.lbve_create.argtypes = [C.POINTER(lbve_channel_desc), dp, C.POINTER(vp)]
        lib.lbve_destroy.argtypes = [vp]
        lib.lbve_destroy.restype = None
        lib.lbve_create_batch.argtypes = [C.POINTER(lbve_channel_desc), i32, dp, C.POINTER(vp)]
        lib.lbve_create_ex.argtypes = [C.POINTER(lbve_channel_desc), i32, dp, C.POINTER(lbve_allocator), C.POINTER(vp)]
        lib.lbve_create_tangent.argtypes = [C.POINTER(lbve_channel_desc), dp, C.POINTER(vp)]
        lib.lbve_create_adjoint.argtypes = [C.POINTER(lbve_channel_desc), dp, i32, C.POINTER(vp)]
        lib.lbve_backward.argtypes = [vp, dp, dp, dp, vp]
        lib.lbve_checkpoint_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        lib.lbve_checkpoint_save.argtypes = [vp, vp, i32, vp]
        lib.lbve_checkpoint_restore.argtypes = [vp, vp, i32, vp]
        lib.lbve_tangent_fields.argtypes = [vp, C.c_uint32, vp, vp]
        lib.lbve_channel_nodes.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(i64)]
        lib.lbve_sweep_config.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        lib.lbve_set_sweep_config.argtypes = [vp, i32, i32]
        lib.lbve_set_force.argtypes = [vp, i32, dp, vp]
        lib.lbve_set_params.argtypes = [vp, i32, C.c_double, C.c_double, C.c_double, vp]
        lib.lbve_set_pressure_step.argtypes = [vp, i32, C.c_double, vp]
        lib.lbve_step.argtypes = [vp, i64, vp]
        lib.lbve_get_time.argtypes = [vp, C.POINTER(i64)]
        lib.lbve_fields.argtypes = [vp, C.c_uint32, vp, i32, vp]
        lib.lbve_fields_count.argtypes = [vp, C.c_uint32, C.POINTER(C.c_size_t)]
        lib.lbve_fields_ex.argtypes = [vp, i32, C.c_uint32, vp, i32, i32, vp]
        lib.lbve_history_apply.argtypes = [vp, vp, vp, vp]
        lib.lbve_mass.argtypes = [vp, dp, dp, vp]
        lib.lbve_schedule.argtypes = [i32, i32, i64, C.POINTER(i64), dp, C.POINTER(i32)]
        lib.lbve_memory_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        lib.lbve_strerror.argtypes = [C.c_int]
        lib.lbve_strerror.restype = C.c_char_p
        lib.lbve_fields_host_fixed.argtypes = [vp, C.c_uint32, vp, vp]
        lib.lbve_set_probes.argtypes = [vp, i32, C.POINTER(i64), i32, i64]
        lib.lbve_probe_read.argtypes = [vp, dp, C.POINTER(i64), C.POINTER(i64), vp]
        lib.lbve_profile.argtypes = [vp, i32]
        lib.lbve_profile_read.argtypes = [vp, dp, C.POINTER(i64)]
        lib.lbve_last_cuda_error.argtypes = []
        lib.lbve_last_cuda_error.restype = C.c_char_p
        for name in EXPORTS:       # fail loudly if the library lacks an entry point of the header
            getattr(lib, name)
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != LBVE_OK:
        raise LbveError(rc, where, _lib)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"expected a device pointer or a tensor, got {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return int(torch.cuda.current_stream().cuda_stream) or None
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s or None
    return int(s.cuda_stream) or None


# ---- C ABI, one function each ------------------------------------------------------------------
def lbve_strerror(status: int) -> str:
    return load().lbve_strerror(int(status)).decode()


def lbve_create(desc: lbve_channel_desc, rho_init: np.ndarray | None = None) -> int:
    lib = load()
    h = C.c_void_p()
    ri = None
    if rho_init is not None:
        ri = np.ascontiguousarray(rho_init, dtype=np.float64).ravel()
    rc = lib.lbve_create(C.byref(desc), ri.ctypes.data_as(C.POINTER(C.c_double)) if ri is not None else None,
                         C.byref(h))
    _check(rc, "lbve_create")
    return h.value


def lbve_create_batch(descs, rho_init: np.ndarray | None = None) -> int:
    lib = load()
    arr = (lbve_channel_desc * len(descs))(*descs)
    h = C.c_void_p()
    ri = None
    if rho_init is not None:
        ri = np.ascontiguousarray(rho_init, dtype=np.float64).ravel()
    rc = lib.lbve_create_batch(arr, len(descs), ri.ctypes.data_as(C.POINTER(C.c_double)) if ri is not None else None,
                               C.byref(h))
    _check(rc, "lbve_create_batch")
    return h.value


_ALLOCATORS = {}   # handle -> lbve_allocator kept alive while the handle exists


def lbve_create_ex(descs, rho_init: np.ndarray | None = None, allocator: lbve_allocator | None = None) -> int:
    """lbve_create_batch with the handle's device memory from `allocator` (None: cudaMalloc)."""
    lib = load()
    descs = list(descs) if isinstance(descs, (list, tuple)) else [descs]
    arr = (lbve_channel_desc * len(descs))(*descs)
    h = C.c_void_p()
    ri = None
    if rho_init is not None:
        ri = np.ascontiguousarray(rho_init, dtype=np.float64).ravel()
    rc = lib.lbve_create_ex(arr, len(descs), ri.ctypes.data_as(C.POINTER(C.c_double)) if ri is not None else None,
                            C.byref(allocator) if allocator is not None else None, C.byref(h))
    _check(rc, "lbve_create_ex")
    if allocator is not None:
        _ALLOCATORS[h.value] = allocator
    return h.value


def lbve_create_tangent(desc: lbve_channel_desc, rho_init: np.ndarray | None = None) -> int:
    lib = load()
    h = C.c_void_p()
    ri = None
    if rho_init is not None:
        ri = np.ascontiguousarray(rho_init, dtype=np.float64).ravel()
    rc = lib.lbve_create_tangent(C.byref(desc), ri.ctypes.data_as(C.POINTER(C.c_double)) if ri is not None else None,
                                 C.byref(h))
    _check(rc, "lbve_create_tangent")
    return h.value


def lbve_tangent_fields(h: int, mask: int, stream=None) -> np.ndarray:
    """d(fields)/d(theta_k), theta = (G_inf, tau, gamma_c, g_x): array [4, lbve_fields_count(h, mask)]."""
    cnt = lbve_fields_count(h, mask)
    out = np.empty((4, cnt), dtype=np.float64)
    _check(load().lbve_tangent_fields(h, mask, out.ctypes.data, _stream(stream)), "lbve_tangent_fields")
    return out


def lbve_create_adjoint(desc: lbve_channel_desc, rho_init: np.ndarray | None = None,
                        checkpoint_every: int = 64) -> int:
    lib = load()
    h = C.c_void_p()
    ri = None
    if rho_init is not None:
        ri = np.ascontiguousarray(rho_init, dtype=np.float64).ravel()
    rc = lib.lbve_create_adjoint(C.byref(desc), ri.ctypes.data_as(C.POINTER(C.c_double)) if ri is not None else None,
                                 int(checkpoint_every), C.byref(h))
    _check(rc, "lbve_create_adjoint")
    return h.value


def lbve_backward(h: int, dL_du: np.ndarray, dL_dsigma: np.ndarray, stream=None) -> np.ndarray:
    """dL/d(G_inf, tau, gamma_c, g_x) for seeds dL_du [d, N] and dL_dsigma [nsig, N] of the last step."""
    du = np.ascontiguousarray(dL_du, dtype=np.float64)
    ds = np.ascontiguousarray(dL_dsigma, dtype=np.float64)
    out = np.zeros(4)
    dp = C.POINTER(C.c_double)
    _check(load().lbve_backward(h, du.ctypes.data_as(dp), ds.ctypes.data_as(dp), out.ctypes.data_as(dp),
                                _stream(stream)), "lbve_backward")
    return out


def lbve_checkpoint_size(h: int) -> int:
    n = C.c_size_t()
    _check(load().lbve_checkpoint_size(h, C.byref(n)), "lbve_checkpoint_size")
    return n.value


def lbve_checkpoint_save(h: int, dst=None, stream=None):
    """Save the state; dst None: into a new host bytes buffer (returned); else a device tensor/pointer."""
    if dst is None:
        buf = np.empty(lbve_checkpoint_size(h), dtype=np.uint8)
        _check(load().lbve_checkpoint_save(h, buf.ctypes.data, 0, _stream(stream)), "lbve_checkpoint_save")
        return buf
    _check(load().lbve_checkpoint_save(h, _ptr(dst), 1, _stream(stream)), "lbve_checkpoint_save")
    return dst


def lbve_checkpoint_restore(h: int, src, stream=None) -> None:
    if isinstance(src, np.ndarray):
        _check(load().lbve_checkpoint_restore(h, src.ctypes.data, 0, _stream(stream)), "lbve_checkpoint_restore")
    else:
        _check(load().lbve_checkpoint_restore(h, _ptr(src), 1, _stream(stream)), "lbve_checkpoint_restore")


def lbve_channel_nodes(h: int, channel: int):
    off, cnt = C.c_int64(), C.c_int64()
    _check(load().lbve_channel_nodes(h, channel, C.byref(off), C.byref(cnt)), "lbve_channel_nodes")
    return off.value, cnt.value


def lbve_sweep_config(h: int):
    """(slot chunks, persistent CTAs, task mode: 0 warp tasks / 1 CTA tasks) of the history sweep."""
    s, g, m = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().lbve_sweep_config(h, C.byref(s), C.byref(g), C.byref(m)), "lbve_sweep_config")
    return s.value, g.value, m.value


def lbve_set_sweep_config(h: int, slot_chunks: int, cta_tasks: int) -> None:
    _check(load().lbve_set_sweep_config(h, int(slot_chunks), int(cta_tasks)), "lbve_set_sweep_config")


def lbve_destroy(h: int) -> None:
    load().lbve_destroy(h)
    _ALLOCATORS.pop(h, None)


def lbve_set_force(h: int, g, channel: int = -1, stream=None) -> None:
    gg = (C.c_double * 3)(*[float(v) for v in g])
    _check(load().lbve_set_force(h, channel, gg, _stream(stream)), "lbve_set_force")


def lbve_set_pressure_step(h: int, dp: float, channel: int = -1, stream=None) -> None:
    _check(load().lbve_set_pressure_step(h, channel, float(dp), _stream(stream)), "lbve_set_pressure_step")


def lbve_set_params(h: int, G_inf: float, tau: float, gamma_c: float, channel: int = -1, stream=None) -> None:
    _check(load().lbve_set_params(h, channel, G_inf, tau, gamma_c, _stream(stream)), "lbve_set_params")


def lbve_step(h: int, n_steps: int, stream=None) -> None:
    _check(load().lbve_step(h, int(n_steps), _stream(stream)), "lbve_step")


def lbve_get_time(h: int) -> int:
    t = C.c_int64()
    _check(load().lbve_get_time(h, C.byref(t)), "lbve_get_time")
    return t.value


def lbve_fields_count(h: int, mask: int) -> int:
    n = C.c_size_t()
    _check(load().lbve_fields_count(h, mask, C.byref(n)), "lbve_fields_count")
    return n.value


def lbve_fields_ex(h: int, channel: int, mask: int, dtype: int = LBVE_F64, dst=None, stream=None):
    """Fields of one channel (-1: all nodes) as float64 (LBVE_F64) or float32 (LBVE_F32), one block per field,
    component-major.  dst None: a new numpy array (host copy, synchronising); dst a device tensor / pointer:
    asynchronous device write, returns dst."""
    lib = load()
    if dst is None:
        total = lbve_fields_count(h, mask)
        count = total if channel < 0 else total // _nodes(h) * lbve_channel_nodes(h, channel)[1]
        out = np.empty(count, dtype=np.float64 if dtype == LBVE_F64 else np.float32)
        _check(lib.lbve_fields_ex(h, channel, mask, out.ctypes.data, 0, dtype, _stream(stream)), "lbve_fields_ex")
        return out
    _check(lib.lbve_fields_ex(h, channel, mask, _ptr(dst), 1, dtype, _stream(stream)), "lbve_fields_ex")
    return dst


def _nodes(h: int) -> int:
    """All nodes of the handle (the field count of the density alone)."""
    return lbve_fields_count(h, LBVE_FIELD_RHO)


def lbve_fields(h: int, mask: int, dst=None, stream=None):
    """Fields of the last step.  dst None: returns a new numpy array (host copy, synchronising);
    dst a device tensor / pointer: asynchronous device write, returns dst."""
    lib = load()
    if dst is None:
        out = np.empty(lbve_fields_count(h, mask), dtype=np.float64)
        rc = lib.lbve_fields(h, mask, out.ctypes.data, 0, _stream(stream))
        _check(rc, "lbve_fields")
        return out
    rc = lib.lbve_fields(h, mask, _ptr(dst), 1, _stream(stream))
    _check(rc, "lbve_fields")
    return dst


def lbve_fields_host_fixed(h: int, mask: int, stream=None) -> np.ndarray:
    """lbve_fields into host memory through the library's fixed device staging array (no device
    allocation).  Returns a new numpy array; raises LbveError (LBVE_ETOOBIG) past the array's size."""
    out = np.empty(lbve_fields_count(h, mask), dtype=np.float64)
    _check(load().lbve_fields_host_fixed(h, mask, out.ctypes.data, _stream(stream)), "lbve_fields_host_fixed")
    return out


def lbve_set_probes(h: int, nodes, every: int = 1, capacity: int = 1) -> None:
    """Record [t, per node: rho, u[d], sigma[nsig]] after every step whose count t is a multiple of
    `every` (device-side, inside the step graphs); `nodes` are node indices (empty: remove the recorder)."""
    nn = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64).ravel())
    ptr = nn.ctypes.data_as(C.POINTER(C.c_int64)) if nn.size else None
    _check(load().lbve_set_probes(h, int(nn.size), ptr, int(every), int(capacity)), "lbve_set_probes")


def lbve_probe_read(h: int, n_probes: int, d: int, capacity: int, stream=None):
    """(t [k], values [k, n_probes, 1 + d + nsig], n_total) of the stored probe records (k <= capacity;
    n_total > k means records were dropped).  Synchronising."""
    nsig = 3 if d == 2 else 6
    rec = 1 + n_probes * (1 + d + nsig)
    out = np.empty((capacity, rec), dtype=np.float64)
    k, tot = C.c_int64(), C.c_int64()
    _check(load().lbve_probe_read(h, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(k), C.byref(tot),
                                  _stream(stream)), "lbve_probe_read")
    out = out[: k.value]
    return out[:, 0].astype(np.int64), out[:, 1:].reshape(k.value, n_probes, 1 + d + nsig).copy(), tot.value


def lbve_history_apply(h: int, kappa_dev, sigma_dev, stream=None) -> None:
    _check(load().lbve_history_apply(h, _ptr(kappa_dev), _ptr(sigma_dev), _stream(stream)), "lbve_history_apply")


def lbve_mass(h: int, stream=None):
    a, b = C.c_double(), C.c_double()
    _check(load().lbve_mass(h, C.byref(a), C.byref(b), _stream(stream)), "lbve_mass")
    return a.value, b.value


def lbve_schedule(C_: int, B: int, t: int):
    """Host-only: (t' newest first, trapezoidal weights) of the retained history points after step t."""
    tp = np.zeros(C_ * B, dtype=np.int64)
    w = np.zeros(C_ * B)
    n = C.c_int32()
    rc = load().lbve_schedule(C_, B, t, tp.ctypes.data_as(C.POINTER(C.c_int64)),
                              w.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n))
    _check(rc, "lbve_schedule")
    return tp[: n.value].copy(), w[: n.value].copy()


def lbve_memory_bytes(h: int) -> int:
    n = C.c_size_t()
    _check(load().lbve_memory_bytes(h, C.byref(n)), "lbve_memory_bytes")
    return n.value


def lbve_profile(h: int, enable: bool) -> None:
    _check(load().lbve_profile(h, int(bool(enable))), "lbve_profile")


def lbve_profile_read(h: int):
    """(ms[3], launches[3]) summed over the recorded lbve_step launches: moments, history, collide-stream."""
    ms = (C.c_double * 3)()
    n = (C.c_int64 * 3)()
    _check(load().lbve_profile_read(h, ms, n), "lbve_profile_read")
    return list(ms), list(n)


# ---- convenience wrapper ---------------------------------------------------------------------------
def make_desc(lattice=LBVE_D2Q9, nx=4, ny=32, nz=1, *, tau_lb=0.9, rho0=1.0, G_inf=0.01, tau=200.0,
              gamma_c=0.1, g=(0.0, 0.0, 0.0), C=128, B=1, precision=LBVE_F32, hist_storage=None,
              trace_coupling=LBVE_TRACE_FULL, wall_z=1, model=LBVE_MODEL_NLM, dp=None,
              hist_form=None) -> lbve_channel_desc:
    """dp = None: x periodic, driven by g; a number: the pressure-step boundary with drop dp per period.
    hist_form: LBVE_FORM_P (default) or LBVE_FORM_F (the factor storage of Sec. III)."""
    d = lbve_channel_desc()
    d.lattice, d.nx, d.ny, d.nz, d.wall_z = lattice, nx, ny, nz, wall_z
    d.tau_lb, d.rho0, d.G_inf, d.tau = tau_lb, rho0, G_inf, tau
    d.gamma_c = math.inf if gamma_c is None else gamma_c
    d.g[0], d.g[1], d.g[2] = [float(v) for v in g]
    d.hist_C, d.hist_B = C, B
    d.pop_precision = precision
    d.hist_storage = precision if hist_storage is None else hist_storage
    d.trace_coupling = trace_coupling
    d.model = model
    d.x_boundary = LBVE_X_PERIODIC if dp is None else LBVE_X_PRESSURE
    d.dp = 0.0 if dp is None else float(dp)
    d.hist_form = LBVE_FORM_P if hist_form is None else hist_form
    return d


class Channel:
    """Owns one lbve handle (one channel, or a batch when given a list of descriptions).  fields() returns
    host arrays in the oracle's [node][component] layout; channel_fields(c) slices one channel."""

    def __init__(self, desc, rho_init=None, allocator: lbve_allocator | None = None):
        if isinstance(desc, (list, tuple)):
            self.descs = list(desc)
            self.desc = self.descs[0]
        else:
            self.descs = [desc]
            self.desc = desc
        if allocator is not None:
            self.h = lbve_create_ex(self.descs, rho_init, allocator)
        elif len(self.descs) > 1:
            self.h = lbve_create_batch(self.descs, rho_init)
        else:
            self.h = lbve_create(desc, rho_init)
        self.d = 2 if self.desc.lattice == LBVE_D2Q9 else 3
        self.N = sum(d.nx * d.ny * d.nz for d in self.descs)

    def close(self):
        if getattr(self, "h", None):
            lbve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self) -> int:
        return lbve_get_time(self.h)

    def step(self, n: int = 1, stream=None):
        lbve_step(self.h, n, stream)

    def set_force(self, g, channel: int = -1, stream=None):
        lbve_set_force(self.h, g, channel, stream)

    def set_pressure_step(self, dp, channel: int = -1, stream=None):
        lbve_set_pressure_step(self.h, dp, channel, stream)

    def set_params(self, G_inf, tau, gamma_c, channel: int = -1, stream=None):
        lbve_set_params(self.h, G_inf, tau, gamma_c, channel, stream)

    def channel_fields(self, c: int, fields: dict | None = None) -> dict:
        f = self.fields() if fields is None else fields
        off, cnt = lbve_channel_nodes(self.h, c)
        return {k: v[off:off + cnt] for k, v in f.items()}

    def fields(self, stream=None) -> dict:
        d, N = self.d, self.N
        ns = 3 if d == 2 else 6
        mask = LBVE_FIELD_RHO | LBVE_FIELD_U | LBVE_FIELD_SIGMA | LBVE_FIELD_KAPPA | LBVE_FIELD_N1
        a = lbve_fields(self.h, mask, None, stream)
        o = 0
        rho = a[o:o + N]; o += N
        u = a[o:o + d * N].reshape(d, N).T.copy(); o += d * N
        sig = a[o:o + ns * N].reshape(ns, N).T.copy(); o += ns * N
        kap = a[o:o + d * d * N].reshape(d * d, N).T.reshape(N, d, d).copy(); o += d * d * N
        n1 = a[o:o + N]
        return {"rho": rho.copy(), "u": u, "sigma": sig, "kappa": kap, "n1": n1.copy()}

    def mass(self, stream=None):
        return lbve_mass(self.h, stream)

    def memory_bytes(self) -> int:
        return lbve_memory_bytes(self.h)
