"""Helpers shared by the GPU parity tests."""
import numpy as np

from oracle import oracle as O

FIELDS = ("lnrho", "ux", "uy", "uz", "Ax", "Ay", "Az")


def rel_linf(gpu, ref):
    """Per-field relative L-infinity error max|g - r| / max|r| (7 values)."""
    out = []
    for f in range(7):
        scale = max(np.abs(ref[f]).max(), 1e-300)
        out.append(float(np.abs(gpu[f] - ref[f]).max() / scale))
    return np.array(out)


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
