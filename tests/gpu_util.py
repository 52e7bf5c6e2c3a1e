"""Helpers shared by the GPU parity tests."""
import numpy as np

from oracle import oracle as O

FIELDS = ("lnrho", "ux", "uy", "uz", "Ax", "Ay", "Az")


def rel_linf(gpu, ref, floor=1e-9):
    """Per-field relative L-infinity error max|g - r| / max(max|r|, floor)
    (7 values).  The absolute floor keeps fields that are identically zero
    up to rounding (e.g. every derivative on a 1-point axis) from turning
    rounding noise into a relative error."""
    out = []
    for f in range(7):
        scale = max(np.abs(ref[f]).max(), floor)
        out.append(float(np.abs(gpu[f] - ref[f]).max() / scale))
    return np.array(out)


def rel_linf_state(gpu, ref, cs=1.0):
    """Relative L-infinity error of a state, per field, each normalised by
    the scale of its physical quantity: velocity components by max|u| over
    the vector, vector-potential components by max|A|, and ln rho by
    max(max|ln rho|, max|u| / cs) -- in isothermal gas dynamics density
    perturbations and velocity share that scale (delta rho / rho ~ u / cs).
    A per-field scale alone would turn rounding into a large relative error
    whenever one component is much smaller than its vector (e.g. ln rho a few
    steps after rest, where it is driven by a nearly cancelling div u)."""
    umax = max(np.abs(ref[1:4]).max(), 1e-300)
    amax = max(np.abs(ref[4:7]).max(), 1e-300)
    scales = [max(np.abs(ref[0]).max(), umax / cs), umax, umax, umax, amax, amax, amax]
    return np.array([float(np.abs(gpu[f] - ref[f]).max() / scales[f]) for f in range(7)])


def oracle_params(**kw):
    keys = {f for f in O.Params.__dataclass_fields__}
    return O.Params(**{k: v for k, v in kw.items() if k in keys})


def gpu_params(**kw):
    from paper_2012_08758_b300 import binding as B
    keys = {f for f, _ in B.MhdParams._fields_}
    d = {k: v for k, v in kw.items() if k in keys}
    if "dtype" in kw and isinstance(kw["dtype"], str):
        d["dtype"] = B.MHD_F64 if kw["dtype"] == "f64" else B.MHD_F32
    return d


def state_tol(dtype) -> float:
    """State tolerance against the FP64 oracle: FP64 1e-12, FP32 2e-5."""
    return 1e-12 if dtype in ("f64", 1) else 2e-5


def oracle_state(q0, nsteps, **kw):
    """The FP64 oracle's state after nsteps steps from q0 (a copy), and t."""
    q = np.ascontiguousarray(q0, dtype=np.float64).copy()
    t, _ = O.run(oracle_params(**kw), q, nsteps)
    return q, t


def per_field_linf(gpu, ref, rel_floor=1e-2):
    """Per-field relative L-infinity error, each field by its own max|q|, for
    the u and A components whose own scale is at least rel_floor of their
    vector's (a component far smaller than its vector -- e.g. u_x when the
    forcing wave vector lies along x -- has no scale of its own and is
    covered by the vector-scaled check).  Returns {field index: error}."""
    out = {}
    for lo in (1, 4):
        vec = max(np.abs(ref[lo:lo + 3]).max(), 1e-300)
        for f in range(lo, lo + 3):
            own = np.abs(ref[f]).max()
            if own >= rel_floor * vec:
                out[f] = float(np.abs(gpu[f] - ref[f]).max() / own)
    return out


def assert_state_matches(gpu, ref, dtype, cs=1.0, what=""):
    """State parity: every field within the tolerance scaled by its physical
    quantity (rel_linf_state), and every u / A component that is not
    degenerate within the same tolerance of its own max|q| (per_field_linf)."""
    tol = state_tol(dtype)
    scaled = rel_linf_state(gpu, ref, cs=cs)
    own = per_field_linf(gpu, ref)
    assert scaled.max() < tol, (what, "scaled", scaled, "per field", own)
    assert all(v < tol for v in own.values()), (what, "per field", own, "scaled", scaled)
    return scaled, own
