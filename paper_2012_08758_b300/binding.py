"""ctypes binding of the C ABI in include/mhd.h: same names, argument
marshalling only.  Every call goes to libmhd_b300.so; there is no fallback."""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhd_b300.so")

MHD_F32, MHD_F64 = 0, 1
MHD_OK, MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_ETIMEOUT, MHD_ENONFINITE, MHD_ESTATE = 0, -1, -2, -3, -4, -5, -6
(MHD_URMS, MHD_BRMS, MHD_UMAX, MHD_BMAX, MHD_EKIN, MHD_EMAG, MHD_DIVB_MAX, MHD_MASS, MHD_VMAX,
 MHD_NREDUCE) = range(10)
REDUCE_NAMES = ("urms", "brms", "umax", "bmax", "ekin", "emag", "divb_max", "mass", "vmax")
MHD_KERNEL_AUTO, MHD_KERNEL_SMEM, MHD_KERNEL_TMA = 0, 1, 2

_CODES = {MHD_EINVAL: "EINVAL", MHD_ENOMEM: "ENOMEM", MHD_ECUDA: "ECUDA", MHD_ETIMEOUT: "ETIMEOUT",
          MHD_ENONFINITE: "ENONFINITE", MHD_ESTATE: "ESTATE"}


class MhdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class MhdParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("cs", C.c_double), ("nu", C.c_double), ("eta", C.c_double),
        ("f0", C.c_double), ("kmin", C.c_double), ("kmax", C.c_double), ("sigma", C.c_double),
        ("seed", C.c_uint64),
        ("cfl", C.c_double), ("cfl_visc", C.c_double), ("dt_fixed", C.c_double),
        ("forcing_mode", C.c_int), ("dtype", C.c_int), ("kernel", C.c_int), ("tile", C.c_int),
        ("upwind", C.c_int),
    ]


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: build it with "
                "`python -m paper_2012_08758_b300.build` (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        vp, sz, i64 = C.c_void_p, C.c_size_t, C.c_int64
        pp = C.POINTER(MhdParams)
        dp = C.POINTER(C.c_double)
        sig = {
            "mhd_default_params": (None, [pp]),
            "mhd_resolve_params": (C.c_int, [pp, pp]),
            "mhd_workspace_bytes": (C.c_int, [pp, C.POINTER(sz)]),
            "mhd_create": (C.c_int, [pp, vp, vp, sz, C.POINTER(vp)]),
            "mhd_destroy": (None, [vp]),
            "mhd_set_state": (C.c_int, [vp, vp, C.c_int, C.c_double, i64]),
            "mhd_get_state": (C.c_int, [vp, vp, C.c_int, dp, C.POINTER(i64)]),
            "mhd_step": (C.c_int, [vp, C.c_int]),
            "mhd_step_timed": (C.c_int, [vp, C.c_int, dp, dp]),
            "mhd_reduce": (C.c_int, [vp, C.c_int, dp]),
            "mhd_diagnostics": (C.c_int, [vp, dp]),
            "mhd_time": (C.c_int, [vp, dp, dp, C.POINTER(i64)]),
            "mhd_sync": (C.c_int, [vp]),
            "mhd_forcing_draw": (C.c_int, [vp, i64, dp]),
            "mhd_eval_rhs": (C.c_int, [vp, i64, C.c_double, vp, C.c_int]),
            "mhd_eval_rhs_at": (C.c_int, [vp, i64, C.c_double, C.c_int, vp, vp]),
            "mhd_last_error": (C.c_char_p, [vp]),
            "mhd_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(vp)]),
            "mhd_batch_step": (C.c_int, [vp, C.c_int]),
            "mhd_batch_destroy": (None, [vp]),
            "mhd_diagnostics_noalloc": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                                  C.c_double, C.c_double, C.c_double, vp, vp]),
            "mhd_alu_peak": (C.c_int, [C.c_int, vp, dp, dp]),
            "mhd_spectrum_shells": (C.c_int, [pp, C.POINTER(C.c_int)]),
            "mhd_set_seed_field": (C.c_int, [vp, C.c_uint64, C.c_double]),
            "mhd_padding_check": (C.c_int, [vp, C.POINTER(C.c_longlong)]),
            "mhd_wait_selftest": (C.c_int, [vp, dp, dp]),
            "mhd_substep_plan": (C.c_int, [pp, C.c_int, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int),
                                           C.POINTER(C.c_int)]),
            "mhd_spectrum": (C.c_int, [vp, dp, C.c_int, C.POINTER(C.c_int)]),
            "mhd_slabs_create": (C.c_int, [pp, C.c_int, C.c_int, vp, C.POINTER(vp)]),
            "mhd_slabs_extent": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "mhd_slabs_set_state": (C.c_int, [vp, vp, C.c_int, C.c_double, i64]),
            "mhd_slabs_get_state": (C.c_int, [vp, vp, C.c_int, dp, C.POINTER(i64)]),
            "mhd_slabs_step": (C.c_int, [vp, C.c_int]),
            "mhd_slabs_diagnostics": (C.c_int, [vp, dp]),
            "mhd_slabs_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != MHD_OK:
        msg = lib().mhd_last_error(ctx)
        raise MhdError(rc, msg.decode() if msg else "")
    return rc


def mhd_default_params(**overrides) -> MhdParams:
    p = MhdParams()
    lib().mhd_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"mhd_params has no field {k}")
        setattr(p, k, v)
    return p


def mhd_resolve_params(p: MhdParams) -> MhdParams:
    """p with the automatic kernel and tile choices made."""
    out = MhdParams()
    _check(lib().mhd_resolve_params(C.byref(p), C.byref(out)))
    return out


def mhd_workspace_bytes(p: MhdParams) -> int:
    n = C.c_size_t()
    _check(lib().mhd_workspace_bytes(C.byref(p), C.byref(n)))
    return n.value


def mhd_create(p: MhdParams, stream: int = 0, workspace: int = 0, workspace_bytes: int = 0) -> int:
    """Returns the context handle (an int).  stream: cudaStream_t as int;
    workspace: device pointer as int (0: the library allocates)."""
    out = C.c_void_p()
    _check(lib().mhd_create(C.byref(p), C.c_void_p(stream or None), C.c_void_p(workspace or None),
                            workspace_bytes, C.byref(out)))
    return out.value


def mhd_destroy(ctx: int) -> None:
    lib().mhd_destroy(C.c_void_p(ctx))


def _host(a: np.ndarray):
    if a.dtype == np.float64:
        return MHD_F64
    if a.dtype == np.float32:
        return MHD_F32
    raise TypeError("host arrays must be float32 or float64")


def mhd_set_state(ctx: int, q: np.ndarray, t: float = 0.0, step: int = 0) -> None:
    q = np.ascontiguousarray(q)
    _check(lib().mhd_set_state(C.c_void_p(ctx), q.ctypes.data_as(C.c_void_p), _host(q), float(t),
                               int(step)), C.c_void_p(ctx))


def mhd_get_state(ctx: int, out: np.ndarray | None = None, shape=None, dtype=np.float64):
    """Returns (state, t, step); state has shape (7, nz, ny, nx)."""
    t = C.c_double()
    st = C.c_int64()
    if out is None:
        out = np.empty(shape, dtype=dtype)
    assert out.flags["C_CONTIGUOUS"]
    _check(lib().mhd_get_state(C.c_void_p(ctx), out.ctypes.data_as(C.c_void_p), _host(out),
                               C.byref(t), C.byref(st)), C.c_void_p(ctx))
    return out, t.value, st.value


def mhd_step(ctx: int, nsteps: int) -> None:
    _check(lib().mhd_step(C.c_void_p(ctx), int(nsteps)), C.c_void_p(ctx))


def mhd_step_timed(ctx: int, nsteps: int):
    """Returns (stage_ms[4], total_ms): device time of the step prologue and
    of substeps 1-3, summed over nsteps steps, and the total elapsed time."""
    st = (C.c_double * 4)()
    tot = C.c_double()
    _check(lib().mhd_step_timed(C.c_void_p(ctx), int(nsteps), st, C.byref(tot)), C.c_void_p(ctx))
    return list(st), tot.value


def mhd_reduce(ctx: int, kind: int) -> float:
    v = C.c_double()
    _check(lib().mhd_reduce(C.c_void_p(ctx), int(kind), C.byref(v)), C.c_void_p(ctx))
    return v.value


def mhd_diagnostics(ctx: int) -> dict:
    out = (C.c_double * MHD_NREDUCE)()
    _check(lib().mhd_diagnostics(C.c_void_p(ctx), out), C.c_void_p(ctx))
    return dict(zip(REDUCE_NAMES, list(out)))


def mhd_time(ctx: int):
    t, dt = C.c_double(), C.c_double()
    st = C.c_int64()
    _check(lib().mhd_time(C.c_void_p(ctx), C.byref(t), C.byref(dt), C.byref(st)), C.c_void_p(ctx))
    return t.value, dt.value, st.value


def mhd_sync(ctx: int) -> None:
    _check(lib().mhd_sync(C.c_void_p(ctx)), C.c_void_p(ctx))


def mhd_forcing_draw(ctx: int, step: int) -> dict:
    out = (C.c_double * 13)()
    _check(lib().mhd_forcing_draw(C.c_void_p(ctx), int(step), out), C.c_void_p(ctx))
    v = list(out)
    return dict(k=tuple(int(round(x)) for x in v[0:3]), phi=v[3], e=tuple(v[4:7]),
                a=tuple(v[7:10]), b=tuple(v[10:13]))


def mhd_eval_rhs(ctx: int, shape, step: int = 0, dt_forcing: float = 0.0, dtype=np.float64):
    out = np.empty(shape, dtype=dtype)
    _check(lib().mhd_eval_rhs(C.c_void_p(ctx), int(step), float(dt_forcing),
                              out.ctypes.data_as(C.c_void_p), _host(out)), C.c_void_p(ctx))
    return out


def mhd_eval_rhs_at(ctx: int, points, step: int = 0, dt_forcing: float = 0.0) -> np.ndarray:
    """dq/dt at the listed (i, j, k) points: array (len(points), 7)."""
    ijk = np.ascontiguousarray(np.asarray(points, dtype=np.int32).reshape(-1, 3))
    out = np.empty((len(ijk), 7))
    _check(lib().mhd_eval_rhs_at(C.c_void_p(ctx), int(step), float(dt_forcing), len(ijk),
                                 ijk.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p)),
           C.c_void_p(ctx))
    return out


def mhd_last_error(ctx: int | None = None) -> str:
    m = lib().mhd_last_error(C.c_void_p(ctx) if ctx else None)
    return m.decode() if m else ""


def mhd_batch_create(ctxs) -> int:
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    out = C.c_void_p()
    _check(lib().mhd_batch_create(arr, len(ctxs), C.byref(out)))
    return out.value


def mhd_batch_step(batch: int, nsteps: int) -> None:
    _check(lib().mhd_batch_step(C.c_void_p(batch), int(nsteps)))


def mhd_batch_destroy(batch: int) -> None:
    lib().mhd_batch_destroy(C.c_void_p(batch))


def mhd_slabs_create(p: MhdParams, nslabs: int, overlap: int = 1, stream: int = 0) -> int:
    """The grid of p decomposed into nslabs z-slabs on the current device."""
    out = C.c_void_p()
    _check(lib().mhd_slabs_create(C.byref(p), int(nslabs), int(overlap), C.c_void_p(stream or None),
                                  C.byref(out)))
    return out.value


def mhd_slabs_extent(slabs: int, slab: int) -> tuple[int, int]:
    z0, nz = C.c_int(), C.c_int()
    _check(lib().mhd_slabs_extent(C.c_void_p(slabs), int(slab), C.byref(z0), C.byref(nz)))
    return z0.value, nz.value


def mhd_slabs_set_state(slabs: int, q: np.ndarray, t: float = 0.0, step: int = 0) -> None:
    q = np.ascontiguousarray(q)
    dt = MHD_F32 if q.dtype == np.float32 else MHD_F64
    q = q if q.dtype in (np.float32, np.float64) else q.astype(np.float64)
    _check(lib().mhd_slabs_set_state(C.c_void_p(slabs), q.ctypes.data_as(C.c_void_p), dt, float(t), int(step)))


def mhd_slabs_get_state(slabs: int, shape, dtype=np.float64):
    out = np.empty(shape, dtype=dtype)
    t, st = C.c_double(), C.c_int64()
    _check(lib().mhd_slabs_get_state(C.c_void_p(slabs), out.ctypes.data_as(C.c_void_p),
                                     MHD_F32 if out.dtype == np.float32 else MHD_F64, C.byref(t), C.byref(st)))
    return out, t.value, st.value


def mhd_slabs_step(slabs: int, nsteps: int) -> None:
    _check(lib().mhd_slabs_step(C.c_void_p(slabs), int(nsteps)))


def mhd_slabs_diagnostics(slabs: int) -> dict:
    out = (C.c_double * MHD_NREDUCE)()
    _check(lib().mhd_slabs_diagnostics(C.c_void_p(slabs), out))
    return dict(zip(REDUCE_NAMES, list(out)))


def mhd_slabs_destroy(slabs: int) -> None:
    lib().mhd_slabs_destroy(C.c_void_p(slabs))


MHD_NOALLOC_MAX_POINTS = 1 << 24


def mhd_diagnostics_noalloc(state_dev: int, dtype: int, nx: int, ny: int, nz: int, lx: float,
                            ly: float, lz: float, cs: float, out_dev: int, stream: int = 0) -> None:
    """Diagnostics of a dense device state into out_dev (9 device doubles)
    without any device allocation; pointers and stream are ints."""
    _check(lib().mhd_diagnostics_noalloc(C.c_void_p(state_dev), int(dtype), int(nx), int(ny), int(nz),
                                         float(lx), float(ly), float(lz), float(cs),
                                         C.c_void_p(out_dev), C.c_void_p(stream or None)))


def mhd_set_seed_field(ctx: int, seed: int, amp: float) -> None:
    """The paper's initial state generated on the device (t = 0, step 0)."""
    _check(lib().mhd_set_seed_field(C.c_void_p(ctx), int(seed) & 0xFFFFFFFFFFFFFFFF, float(amp)), ctx)


def mhd_substep_plan(p: MhdParams, grid_ctas: int):
    """(tiles as an (ntiles, 5) array of x0, y0, z0, z1, run; grid) of the
    fused substep's work split for grid_ctas persistent CTAs."""
    n, g = C.c_int(), C.c_int()
    _check(lib().mhd_substep_plan(C.byref(p), int(grid_ctas), None, 0, C.byref(n), C.byref(g)))
    buf = (C.c_int * max(1, 5 * n.value))()
    _check(lib().mhd_substep_plan(C.byref(p), int(grid_ctas), buf, n.value, C.byref(n), C.byref(g)))
    return np.frombuffer(buf, dtype=np.int32)[: 5 * n.value].reshape(n.value, 5).copy(), g.value


def mhd_wait_selftest(stream: int = 0):
    """Runs the bounded-wait self-test: (return code, seconds the cut-down wait
    took, the kernels' own bound in seconds); MHD_ETIMEOUT is the expected
    code (the wait gave up and reported it)."""
    sec, bound = C.c_double(-1.0), C.c_double(-1.0)
    rc = lib().mhd_wait_selftest(C.c_void_p(stream), C.byref(sec), C.byref(bound))
    return rc, sec.value, bound.value


def mhd_padding_check(ctx: int) -> int:
    """Words of the state buffers' padding columns that are not NaN (0: intact)."""
    n = C.c_longlong()
    _check(lib().mhd_padding_check(C.c_void_p(ctx), C.byref(n)), ctx)
    return n.value


def mhd_spectrum_shells(p: MhdParams) -> int:
    n = C.c_int()
    _check(lib().mhd_spectrum_shells(C.byref(p), C.byref(n)))
    return n.value


def mhd_spectrum(ctx: int, max_shells: int) -> np.ndarray:
    """Magnetic energy spectrum E_B(m), m = 0 .. min(nshells, max_shells)-1
    (FP64 host array)."""
    n = C.c_int()
    out = np.zeros(max(int(max_shells), 1))
    _check(lib().mhd_spectrum(C.c_void_p(ctx), out.ctypes.data_as(C.POINTER(C.c_double)), int(max_shells),
                              C.byref(n)), ctx)
    return out[:min(n.value, int(max_shells))]


MHD_F32X2 = 2  # mhd_alu_peak: FP32 packed pairs


def mhd_alu_peak(dtype: int, stream: int = 0) -> tuple[float, float]:
    """Measured FMA throughput (flop/s, an FMA counts 2) and the median
    launch time in ms of the current device for MHD_F32, MHD_F64 or
    MHD_F32X2; synchronises the stream."""
    flops, ms = C.c_double(), C.c_double()
    _check(lib().mhd_alu_peak(int(dtype), C.c_void_p(stream or None), C.byref(flops), C.byref(ms)))
    return flops.value, ms.value


def default_box() -> float:
    return 2 * math.pi
