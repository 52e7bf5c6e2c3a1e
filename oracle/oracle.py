"""FP64 CPU oracle of the isothermal MHD step (arXiv:2012.08758, Sec. 4).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the
benchmark's CPU-baseline leg are the only users.  The product library never
imports, links or runs anything here, and nothing here imports the product.

Thin ctypes wrapper around ``mhd_oracle.c`` (plain C, built with gcc into
``liboracle.so`` next to this file).  Arrays are numpy float64 of shape
(7, nz, ny, nx) -- x fastest -- in the field order
ln rho, u_x, u_y, u_z, A_x, A_y, A_z.

``ORACLE_LIB_OVERRIDE`` names another build of the same source to load
instead (the mutation test uses it to run the pins against planted bugs).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mhd_oracle.c")
LIB = os.environ.get("ORACLE_LIB_OVERRIDE") or os.path.join(HERE, "liboracle.so")

# Index of each quantity in the vector written by orc_diagnostics.
DIAG_NAMES = ("urms", "brms", "umax", "bmax", "ekin", "emag", "divb_max", "mass", "vmax")


# gcc flags of every build of the oracle (ISO C11: no contraction of a*b+c
# into fused multiply-adds, so every build rounds the same operations).
CFLAGS = ("-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11")
# The timed CPU baseline's build: the same source and rounding, tuned for the
# host it runs on (built there, next to nothing else, on first use).
CFLAGS_NATIVE = ("-O3", "-march=native", "-fopenmp", "-fPIC", "-shared", "-std=c11")


def compile_oracle(src: str, out: str, flags=CFLAGS) -> str:
    """gcc `src` into the shared library `out` with `flags`."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *flags, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP over z-planes of the RHS)."""
    if os.environ.get("ORACLE_LIB_OVERRIDE"):
        return LIB
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        compile_oracle(SRC, LIB)
    return LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("cs", C.c_double), ("nu", C.c_double), ("eta", C.c_double),
        ("f0", C.c_double), ("kmin", C.c_double), ("kmax", C.c_double), ("sigma", C.c_double),
        ("seed", C.c_uint64),
        ("cfl", C.c_double), ("cfl_visc", C.c_double), ("dt_fixed", C.c_double),
        ("forcing_mode", C.c_int), ("upwind", C.c_int),
    ]


class OrcForcing(C.Structure):
    _fields_ = [
        ("k", C.c_int * 3), ("kp", C.c_double * 3), ("phi", C.c_double),
        ("e", C.c_double * 3), ("a", C.c_double * 3), ("b", C.c_double * 3),
        ("amp", C.c_double),
    ]


@dataclass
class Params:
    """Physical and numerical parameters (defaults: Sec. 4 units, L = 2 pi)."""
    nx: int = 32
    ny: int = 32
    nz: int = 32
    lx: float = 2 * math.pi
    ly: float = 2 * math.pi
    lz: float = 2 * math.pi
    cs: float = 1.0
    nu: float = 5e-3
    eta: float = 5e-3
    f0: float = 0.0
    kmin: float = 2.5
    kmax: float = 3.5
    sigma: float = 0.0
    seed: int = 1
    cfl: float = 0.4
    cfl_visc: float = 0.08
    dt_fixed: float = 0.0
    forcing_mode: int = 0
    upwind: int = 0

    def c(self) -> OrcParams:
        return OrcParams(self.nx, self.ny, self.nz, self.lx, self.ly, self.lz, self.cs,
                         self.nu, self.eta, self.f0, self.kmin, self.kmax, self.sigma,
                         self.seed & 0xFFFFFFFFFFFFFFFF, self.cfl, self.cfl_visc,
                         self.dt_fixed, self.forcing_mode, self.upwind)

    @property
    def shape(self):
        return (7, self.nz, self.ny, self.nx)


def host_tag() -> str:
    """Short hash of this host's CPU model and flags (a -march=native build
    is only valid on a CPU like the one it was built on)."""
    import hashlib
    try:
        with open("/proc/cpuinfo") as f:
            info = [l for l in f if l.startswith(("model name", "flags"))][:2]
    except OSError:
        info = []
    return hashlib.sha256("".join(info).encode()).hexdigest()[:12]


def use_native() -> str:
    """Switch this process to the host-tuned build (CFLAGS_NATIVE), compiled
    on first use for this host's CPU; same source, same rounding.  Used by
    the timed CPU baseline only."""
    global LIB, _lib
    path = os.path.join(HERE, f"liboracle_native_{host_tag()}.so")
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(SRC):
        compile_oracle(SRC, path, CFLAGS_NATIVE)
    if LIB != path:
        LIB, _lib = path, None
    return path


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.basename(LIB).startswith("liboracle_native_"):
            build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(OrcParams)
        fp = C.POINTER(OrcForcing)
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        for name in ("orc_stencil_d1", "orc_stencil_d2"):
            getattr(L, name).argtypes = [dp, C.c_double]
            getattr(L, name).restype = C.c_double
        L.orc_stencil_up.argtypes = [dp, C.c_double, C.c_int]
        L.orc_stencil_up.restype = C.c_double
        L.orc_dup.argtypes = [pp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_dup.restype = C.c_double
        L.orc_stencil_dmix.argtypes = [dp, C.c_double, C.c_double]
        L.orc_stencil_dmix.restype = C.c_double
        L.orc_d1.argtypes = [pp, dp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_d1.restype = C.c_double
        L.orc_d2.argtypes = [pp, dp, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_d2.restype = C.c_double
        L.orc_dmix.argtypes = [pp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_dmix.restype = C.c_double
        L.orc_kshell.argtypes = [C.c_double, C.c_double, C.POINTER(C.c_int), C.c_int]
        L.orc_kshell.restype = C.c_int
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_forcing_draw.argtypes = [pp, C.c_int64, fp]
        L.orc_forcing_draw.restype = None
        L.orc_forcing_amplitude.argtypes = [pp, C.c_double, fp]
        L.orc_forcing_amplitude.restype = None
        L.orc_forcing_at.argtypes = [pp, fp, C.c_int, C.c_int, C.c_int, dp]
        L.orc_forcing_at.restype = None
        L.orc_rhs_at.argtypes = [pp, dp, fp, C.c_int, C.c_int, C.c_int, dp]
        L.orc_rhs_at.restype = None
        L.orc_rhs.argtypes = [pp, dp, fp, dp]
        L.orc_rhs.restype = None
        L.orc_max_speed.argtypes = [pp, dp]
        L.orc_max_speed.restype = C.c_double
        L.orc_dt.argtypes = [pp, dp]
        L.orc_dt.restype = C.c_double
        L.orc_step.argtypes = [pp, dp, C.c_int64, dp, dp, fp]
        L.orc_step.restype = C.c_double
        L.orc_run.argtypes = [pp, dp, C.c_int64, C.c_int, C.c_double, dp]
        L.orc_run.restype = C.c_double
        L.orc_curl.argtypes = [pp, dp, dp]
        L.orc_curl.restype = None
        L.orc_diagnostics.argtypes = [pp, dp, dp]
        L.orc_diagnostics.restype = None
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n: int) -> int:
    """Threads for the RHS loop; returns the count in effect."""
    return lib().orc_set_threads(int(n))


# ---- stencils -------------------------------------------------------------
def stencil_d1(line7, h):
    a = np.ascontiguousarray(line7, dtype=np.float64)
    return lib().orc_stencil_d1(_dp(a), float(h))


def stencil_d2(line7, h):
    a = np.ascontiguousarray(line7, dtype=np.float64)
    return lib().orc_stencil_d2(_dp(a), float(h))


def stencil_up(line7, h, direction):
    """Upwind-biased first derivative (R8): direction >= 0 for a flow
    towards +axis (uses f(-3..2)), < 0 for the mirror (f(-2..3))."""
    a = np.ascontiguousarray(line7, dtype=np.float64)
    return lib().orc_stencil_up(_dp(a), float(h), int(direction))


def dup(p: Params, f, axis, direction):
    """Periodic upwind-biased first derivative of one field along axis."""
    return _field_op(p, f, lib().orc_dup, axis, direction)


def stencil_dmix(patch7x7, ha, hb):
    """patch[sb+3, sa+3] = f(a + sa*ha, b + sb*hb)."""
    a = np.ascontiguousarray(patch7x7, dtype=np.float64)
    return lib().orc_stencil_dmix(_dp(a), float(ha), float(hb))


def _field_op(p: Params, f: np.ndarray, fn, *axes):
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (p.nz, p.ny, p.nx)
    pc = p.c()
    out = np.empty_like(f)
    for k in range(p.nz):
        for j in range(p.ny):
            for i in range(p.nx):
                out[k, j, i] = fn(C.byref(pc), _dp(f), i, j, k, *axes)
    return out


def d1(p: Params, f, axis):
    """Periodic first derivative of one field along axis (0=x,1=y,2=z)."""
    return _field_op(p, f, lib().orc_d1, axis)


def d2(p: Params, f, axis):
    return _field_op(p, f, lib().orc_d2, axis)


def dmix(p: Params, f, a, b):
    return _field_op(p, f, lib().orc_dmix, a, b)


# ---- forcing ---------------------------------------------------------------
def kshell(kmin, kmax) -> np.ndarray:
    n = lib().orc_kshell(kmin, kmax, None, 0)
    buf = (C.c_int * (3 * max(n, 1)))()
    lib().orc_kshell(kmin, kmax, buf, n)
    return np.array(buf[: 3 * n], dtype=np.int64).reshape(n, 3)


def splitmix64(seed: int, counter: int) -> int:
    return int(lib().orc_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, counter & 0xFFFFFFFFFFFFFFFF))


@dataclass
class Forcing:
    k: tuple
    kp: tuple
    phi: float
    e: tuple
    a: tuple
    b: tuple
    amp: float
    _c: OrcForcing = field(repr=False, default=None)


def _wrap_forcing(F: OrcForcing) -> Forcing:
    return Forcing(tuple(F.k), tuple(F.kp), F.phi, tuple(F.e), tuple(F.a), tuple(F.b), F.amp, F)


def forcing_draw(p: Params, step: int, dt: float | None = None) -> Forcing:
    F = OrcForcing()
    pc = p.c()
    lib().orc_forcing_draw(C.byref(pc), int(step), C.byref(F))
    if dt is not None:
        lib().orc_forcing_amplitude(C.byref(pc), float(dt), C.byref(F))
    return _wrap_forcing(F)


def forcing_field(p: Params, F: Forcing) -> np.ndarray:
    """f(x) on the grid, shape (3, nz, ny, nx)."""
    out = np.empty((3, p.nz, p.ny, p.nx))
    pc = p.c()
    v = (C.c_double * 3)()
    for k in range(p.nz):
        for j in range(p.ny):
            for i in range(p.nx):
                lib().orc_forcing_at(C.byref(pc), C.byref(F._c), i, j, k, v)
                out[:, k, j, i] = v[:]
    return out


# ---- RHS, dt, step, diagnostics --------------------------------------------
def rhs(p: Params, q: np.ndarray, F: Forcing | None = None) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.shape == p.shape
    out = np.empty_like(q)
    pc = p.c()
    lib().orc_rhs(C.byref(pc), _dp(q), C.byref(F._c) if F is not None else None, _dp(out))
    return out


def rhs_at(p: Params, q: np.ndarray, points, F: Forcing | None = None) -> np.ndarray:
    """dq/dt at the listed (i, j, k) points only; returns (len(points), 7)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.shape == p.shape
    pc = p.c()
    out = np.empty((len(points), 7))
    v = (C.c_double * 7)()
    Fc = C.byref(F._c) if F is not None else None
    for n, (i, j, k) in enumerate(points):
        lib().orc_rhs_at(C.byref(pc), _dp(q), Fc, int(i), int(j), int(k), v)
        out[n] = v[:]
    return out


def max_speed(p: Params, q) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().orc_max_speed(C.byref(p.c()), _dp(q))


def dt(p: Params, q) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().orc_dt(C.byref(p.c()), _dp(q))


def step(p: Params, q: np.ndarray, step_index: int, w: np.ndarray | None = None):
    """One RK3-2N step in place; returns (dt, Forcing)."""
    assert q.dtype == np.float64 and q.flags["C_CONTIGUOUS"] and q.shape == p.shape
    w = np.zeros_like(q) if w is None else w
    r = np.empty_like(q)
    F = OrcForcing()
    d = lib().orc_step(C.byref(p.c()), _dp(q), int(step_index), _dp(w), _dp(r), C.byref(F))
    return d, _wrap_forcing(F)


def run(p: Params, q: np.ndarray, nsteps: int, step0: int = 0, t0: float = 0.0):
    """nsteps steps in place; returns (t, dts)."""
    assert q.dtype == np.float64 and q.flags["C_CONTIGUOUS"] and q.shape == p.shape
    dts = np.zeros(max(nsteps, 1))
    t = lib().orc_run(C.byref(p.c()), _dp(q), int(step0), int(nsteps), float(t0), _dp(dts))
    return t, dts[:nsteps]


def diagnostics(p: Params, q) -> dict:
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(len(DIAG_NAMES))
    lib().orc_diagnostics(C.byref(p.c()), _dp(q), _dp(out))
    return dict(zip(DIAG_NAMES, out.tolist()))


def curl(p: Params, q) -> np.ndarray:
    """B = curl A with the first-derivative stencil, shape (3, nz, ny, nx)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.shape == p.shape
    B = np.empty((3, p.nz, p.ny, p.nx))
    lib().orc_curl(C.byref(p.c()), _dp(q), _dp(B))
    return B


def spectrum(p: Params, q) -> np.ndarray:
    """Magnetic energy spectrum of Sec. 5 (power spectra), per unit volume:
    E_B(m) = 1/2 sum over integer wave vectors k with m - 1/2 <= |k| < m + 1/2
    of |B^(k)|^2, B^ = N^-3 * (discrete Fourier transform of B); the sum over
    m is <B^2>/2.  The library FFT is the primitive; shells m = 0 .. M with
    M = floor(sqrt((nx//2)^2 + (ny//2)^2 + (nz//2)^2) + 1/2).  Cubic box."""
    B = curl(p, q)
    n = p.nx * p.ny * p.nz
    power = sum(np.abs(np.fft.fftn(B[c])) ** 2 for c in range(3)) / float(n) ** 2
    kz = np.fft.fftfreq(p.nz, 1.0 / p.nz)
    ky = np.fft.fftfreq(p.ny, 1.0 / p.ny)
    kx = np.fft.fftfreq(p.nx, 1.0 / p.nx)
    K2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    m = np.floor(np.sqrt(K2) + 0.5).astype(np.int64)
    mmax = int(math.floor(math.sqrt((p.nx // 2) ** 2 + (p.ny // 2) ** 2 + (p.nz // 2) ** 2) + 0.5))
    return 0.5 * np.bincount(m.ravel(), weights=power.ravel(), minlength=mmax + 1)


def growth_rate(t, brms) -> float:
    """Least-squares slope of ln B_rms against t (Sec. 4, growth-rate fit
    B_rms ~ exp(lambda t)); a library polynomial fit is the primitive."""
    t = np.asarray(t, dtype=np.float64)
    y = np.log(np.asarray(brms, dtype=np.float64))
    return float(np.polyfit(t, y, 1)[0])
