"""FP64 CPU oracle of the hybrid LB scheme of arXiv:1504.06123 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference leg may import
this package.  The product (``paper_1504_06123_gb300``) never imports, links or runs it, and the two
share no code: this wrapper loads ``lbve_oracle.c`` (plain C, FP64, the paper's factor storage),
compiled with gcc into ``oracle/_build/``.

Each function names the passage it follows; the C source states the readings of the paper it takes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbve_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbve_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19 = 9, 19
# constitutive model of sigma_struc: integral nlM (Eqs. gitt, nlmax), instantaneous nlM (Eq. inlM),
# White-Metzner form of Eq. (nlmax) (accumulated strain in the second exponential, Sec. II)
NLM, INLM, WM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it must build the same on x86 and Arm).

    LBVE_ORACLE_LIB names a prebuilt oracle library to load instead (the planted-mistake tests compile a
    copy of the source with one deliberate error and check that the pins reject it)."""
    alt = os.environ.get("LBVE_ORACLE_LIB")
    if alt:
        return alt
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP splits the node loops over host threads (bitwise the same results); without it the
        # oracle builds serial
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        lib.orc_history_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_int, dp, dp, C.c_int, C.c_int]
        lib.orc_history_run.restype = C.c_int
        lib.orc_schedule.argtypes = [C.c_int, C.c_int, C.c_int64, C.POINTER(C.c_int64), dp]
        lib.orc_schedule.restype = C.c_int
        lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_double, dp, C.c_int, C.c_int, C.c_int, dp]
        lib.orc_create.restype = C.c_void_p
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_set_force.argtypes = [C.c_void_p, dp]
        lib.orc_set_params.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double]
        lib.orc_set_pressure.argtypes = [C.c_void_p, C.c_int, C.c_double]
        lib.orc_set_model.argtypes = [C.c_void_p, C.c_int]
        lib.orc_set_model.restype = C.c_int
        lib.orc_inlm.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, dp]
        lib.orc_inlm.restype = C.c_int
        lib.orc_time.argtypes = [C.c_void_p]
        lib.orc_time.restype = C.c_int64
        lib.orc_step.argtypes = [C.c_void_p, C.c_int64]
        lib.orc_step.restype = C.c_int
        lib.orc_fields.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        lib.orc_populations.argtypes = [C.c_void_p, dp]
        lib.orc_mass.argtypes = [C.c_void_p, dp, dp]
        lib.orc_kappa_of.argtypes = [C.c_void_p, dp, dp]
        lib.orc_expm.argtypes = [C.c_int, dp, dp]
        lib.orc_set_threads.argtypes = [C.c_int]
        lib.orc_set_threads.restype = C.c_int
        lib.orc_get_threads.restype = C.c_int
        # all host cores unless LBVE_ORACLE_THREADS says otherwise (results do not depend on the count)
        lib.orc_set_threads(int(os.environ.get("LBVE_ORACLE_THREADS", "0")))
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's node loops (n < 1: all cores); returns the count in use (1 when the
    oracle was built without OpenMP).  Every node's arithmetic is the same whatever the count, so results
    are bitwise independent of it."""
    return int(_load().orc_set_threads(int(n)))


def threads() -> int:
    """Host threads the oracle's node loops use now."""
    return int(_load().orc_get_threads())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def expm(K: np.ndarray) -> np.ndarray:
    """exp of a 2x2 (closed form) or 3x3 (scaled Taylor) matrix -- the factor exp(kappa dt), Eq. (eeval)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    d = K.shape[0]
    out = np.zeros((d, d))
    _load().orc_expm(d, _dp(K), _dp(out))
    return out


def history_run(kappa_seq: np.ndarray, C_: int, B: int, G_inf: float, tau: float, gamma_c: float,
                last_only: bool = False, model: int = NLM) -> np.ndarray:
    """Stress history integral with a prescribed velocity gradient at every node and step.

    kappa_seq: [T, nnodes, d, d] (or [T, nnodes, d*d]) -- kappa(t) of each node, row-major
    kappa[a, b] = d v_a / d x_b.  Returns sigma_struc [T, nnodes, nsig] (or [nnodes, nsig] with
    last_only), components xx, yy, xy (2D) or xx, yy, zz, xy, xz, yz (3D).
    Follows Eq. (gitt) with the modulus of Eq. (nlmax) on the quasi-logarithmic grid and factor
    storage of Sec. III / Eq. (eeval).  model = WM takes the accumulated strain in the modulus;
    model = INLM evaluates Eq. (inlM) on kappa(t) alone (C_ and B are then unused).
    """
    k = np.ascontiguousarray(kappa_seq, dtype=np.float64)
    T, nn = k.shape[0], k.shape[1]
    dd = int(np.prod(k.shape[2:]))
    d = int(round(math.sqrt(dd)))
    nsig = 3 if d == 2 else 6
    out = np.zeros((nn, nsig) if last_only else (T, nn, nsig))
    rc = _load().orc_history_run(d, nn, C_, B, G_inf, tau, gamma_c, T, _dp(k), _dp(out), int(last_only),
                                 int(model))
    if rc != 0:
        raise ValueError("orc_history_run rejected its arguments")
    return out


def inlm(K: np.ndarray, G_inf: float, tau: float, gamma_c: float) -> np.ndarray:
    """sigma_struc of the instantaneous nlM, Eq. (inlM), for one gradient K [d, d] (series as printed).

    Returns the packed components (xx, yy, xy or xx, yy, zz, xy, xz, yz); NaN where the series diverges.
    """
    K = np.ascontiguousarray(K, dtype=np.float64)
    d = K.shape[0]
    out = np.zeros(3 if d == 2 else 6)
    if _load().orc_inlm(d, _dp(K), G_inf, tau, gamma_c, _dp(out)) != 0:
        raise ValueError("orc_inlm rejected its arguments")
    return out


def schedule(C_: int, B: int, t: int):
    """Retained history points after step t: (t' newest first, trapezoidal weights). Sec. III layout."""
    tp = np.zeros(B * C_, dtype=np.int64)
    w = np.zeros(B * C_)
    n = _load().orc_schedule(C_, B, t, tp.ctypes.data_as(C.POINTER(C.c_int64)), _dp(w))
    if n < 0:
        raise ValueError("orc_schedule rejected its arguments")
    return tp[:n].copy(), w[:n].copy()


class Channel:
    """One LB channel (D2Q9 planar channel or D3Q19 duct) with the nlM stress history, in FP64.

    Sec. III: BGK collision, forcing Eq. (bodyforce), fields Eq. (hydrofields), history of Eq. (gitt)
    with Eq. (nlmax).  x is periodic; walls (half-way bounce-back) at y = -1/2 and ny - 1/2, and at
    z = -1/2, nz - 1/2 for a duct.
    """

    def __init__(self, lattice: int, nx: int, ny: int, nz: int = 1, *, tau_lb: float, G_inf: float,
                 tau: float, gamma_c: float, g=(0.0, 0.0, 0.0), C: int, B: int, rho0: float = 1.0,
                 trace_full: bool = True, wall_z: bool = True, rho_init: np.ndarray | None = None,
                 model: int = NLM, dp: float | None = None):
        self.lib = _load()
        self.lattice, self.nx, self.ny, self.nz = lattice, nx, ny, nz
        self.d = 2 if lattice == D2Q9 else 3
        self.Q = lattice
        self.N = nx * ny * nz
        gg = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(3))
        ri = None
        if rho_init is not None:
            ri = np.ascontiguousarray(np.asarray(rho_init, dtype=np.float64).reshape(self.N))
        self._h = self.lib.orc_create(lattice, nx, ny, nz, int(wall_z), tau_lb, rho0, G_inf, tau, gamma_c,
                                      _dp(gg), C, B, int(trace_full), _dp(ri) if ri is not None else None)
        if not self._h:
            raise ValueError("orc_create rejected its arguments")
        if self.lib.orc_set_model(self._h, int(model)) != 0:
            self.close()
            raise ValueError("unknown constitutive model")
        if dp is not None:
            self.set_pressure_step(dp)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.orc_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def t(self) -> int:
        return int(self.lib.orc_time(self._h))

    def step(self, n: int = 1):
        self.lib.orc_step(self._h, int(n))

    def set_force(self, g):
        gg = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(3))
        self.lib.orc_set_force(self._h, _dp(gg))

    def set_pressure_step(self, dp: float | None):
        """Pressure-step boundary along x (Sec. III, generalised periodic boundary): pressure drop dp over one
        period (nx spacings), mean density rho0; None restores the plain periodic boundary."""
        if dp is None:
            self.lib.orc_set_pressure(self._h, 0, 0.0)
        else:
            self.lib.orc_set_pressure(self._h, 1, float(dp))

    def set_params(self, G_inf: float, tau: float, gamma_c: float):
        self.lib.orc_set_params(self._h, G_inf, tau, gamma_c)

    def fields(self) -> dict:
        """rho [N], u [N,d], sigma [N,nsig], kappa [N,d,d], n1 [N] of the last completed step."""
        N, d = self.N, self.d
        nsig = 3 if d == 2 else 6
        rho, u, sig = np.zeros(N), np.zeros((N, d)), np.zeros((N, nsig))
        kap, n1 = np.zeros((N, d, d)), np.zeros(N)
        self.lib.orc_fields(self._h, _dp(rho), _dp(u), _dp(sig), _dp(kap), _dp(n1))
        return {"rho": rho, "u": u, "sigma": sig, "kappa": kap, "n1": n1}

    def populations(self) -> np.ndarray:
        out = np.zeros((self.N, self.Q))
        self.lib.orc_populations(self._h, _dp(out))
        return out

    def mass(self):
        """(sum of populations, sum of delta rho(t-1) = -tr sigma(t-1)/(d c_s^2)) -- the density source."""
        a, b = C.c_double(), C.c_double()
        self.lib.orc_mass(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def kappa_of(self, u: np.ndarray) -> np.ndarray:
        """kappa [N,d,d] of a prescribed velocity field u [N,d] by the finite-difference stencil."""
        uu = np.zeros((self.N, 3))
        uu[:, : self.d] = np.asarray(u).reshape(self.N, self.d)
        uu = np.ascontiguousarray(uu)
        out = np.zeros((self.N, self.d, self.d))
        self.lib.orc_kappa_of(self._h, _dp(uu), _dp(out))
        return out


def collide(ch: "Channel", n: np.ndarray, sigma: np.ndarray, tr_prev: float):
    """Post-collision populations of one node (BGK + Eq. (bodyforce)) with the channel's parameters.

    Returns (post [Q], rho, u [3]) where rho, u are the hydrodynamic fields of Eq. (hydrofields).
    """
    lib = _load()
    if not getattr(lib, "_collide_typed", False):
        lib.orc_collide.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double,
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib._collide_typed = True
    nn = np.ascontiguousarray(n, dtype=np.float64)
    sg = np.zeros(6)
    sg[: len(sigma)] = sigma
    post = np.zeros(ch.Q)
    rho = C.c_double()
    u = np.zeros(3)
    lib.orc_collide(ch._h, _dp(nn), _dp(sg), float(tr_prev), _dp(post), C.byref(rho), _dp(u))
    return post, rho.value, u
