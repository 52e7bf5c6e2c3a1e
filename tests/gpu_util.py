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
