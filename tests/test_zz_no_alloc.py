"""The allocation-free diagnostics entry point, for callers that cannot
allocate device memory (a plugin inside an application whose memory pool
owns the GPU, a fixed memory budget, a latency-critical loop where
cudaMalloc could synchronise the device or fail).  It must give what the
context-based mhd_diagnostics gives, call after call, while its only scratch
is the library's static device array.  Kept in a file of its own that pytest
collects last."""
import math

import numpy as np
import pytest

from paper_2012_08758_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype_name,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_diagnostics_match_context_path_on_consecutive_calls(dtype_name, tol):
    import torch

    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.run import Run

    nx, ny, nz, cs = 40, 24, 20, 1.2
    dt = B.MHD_F64 if dtype_name == "f64" else B.MHD_F32
    tdt = torch.float64 if dtype_name == "f64" else torch.float32
    states = [inputs.random_modes_state(nx, ny, nz, seed=s, amp=0.4) + inputs.noise_state(nx, ny, nz, seed=9 + s,
                                                                                          amp=0.01)
              for s in (1, 2)]
    run = Run(nx=nx, ny=ny, nz=nz, cs=cs, dtype=dt)
    stream = run.stream
    out = torch.full((B.MHD_NREDUCE,), float("nan"), dtype=torch.float64, device=run.device)
    for q in states:  # two calls in a row, different inputs, shared scratch
        run.set_state(q)
        ref = run.diagnostics()
        dense = torch.tensor(q, dtype=tdt, device=run.device).contiguous()
        torch.cuda.synchronize()
        B.mhd_diagnostics_noalloc(dense.data_ptr(), dt, nx, ny, nz, 2 * math.pi, 2 * math.pi, 2 * math.pi,
                                  cs, out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = dict(zip(B.REDUCE_NAMES, out.cpu().tolist()))
        for key in ("urms", "brms", "umax", "bmax", "ekin", "emag", "mass", "vmax"):
            assert got[key] == pytest.approx(ref[key], rel=tol), key
        # div B is rounding noise in both; both stay below the same bound
        bound = (1e-12 if dtype_name == "f64" else 1e-4) * ref["bmax"] * nx / (2 * math.pi)
        assert got["divb_max"] < bound and ref["divb_max"] < bound
    run.close()


def _dense_and_reference(run, q, tdt):
    import torch
    run.set_state(q)
    ref = run.diagnostics()
    dense = torch.tensor(q, dtype=tdt, device=run.device).contiguous()
    torch.cuda.synchronize()
    return dense, ref


def test_noalloc_larger_grid_then_smaller_grid_allocates_nothing():
    """A call on a larger grid (more blocks, more partials left in the
    shared scratch) and then one on a smaller grid: each equal to the context
    path, and neither changes the device memory in use -- neither torch's
    allocator nor the driver's free-memory count moves across a call."""
    import torch

    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.run import Run

    cs = 0.9
    shapes = [(64, 48, 40), (20, 12, 9)]  # 30 blocks of partials, then 1
    runs, denses, refs = [], [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        q = inputs.random_modes_state(nx, ny, nz, seed=20 + i, amp=0.3) + inputs.noise_state(nx, ny, nz,
                                                                                           seed=30 + i,
                                                                                           amp=0.01)
        run = Run(nx=nx, ny=ny, nz=nz, cs=cs, dtype=B.MHD_F64)
        d, r = _dense_and_reference(run, q, torch.float64)
        runs.append(run)
        denses.append(d)
        refs.append(r)
    stream = runs[0].stream
    out = torch.full((B.MHD_NREDUCE,), float("nan"), dtype=torch.float64, device=runs[0].device)
    L = 2 * math.pi

    def call(i):
        nx, ny, nz = shapes[i]
        B.mhd_diagnostics_noalloc(denses[i].data_ptr(), B.MHD_F64, nx, ny, nz, L, L, L, cs, out.data_ptr(),
                                  stream.cuda_stream)
        stream.synchronize()
        return dict(zip(B.REDUCE_NAMES, out.cpu().tolist()))

    call(0)  # first call in this context: the scratch address is looked up here
    torch.cuda.synchronize()
    for i in (0, 1, 0, 1):
        alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        got = call(i)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == alloc0
        assert torch.cuda.mem_get_info()[0] == free0
        for key in ("urms", "brms", "umax", "bmax", "ekin", "emag", "mass", "vmax"):
            assert got[key] == pytest.approx(refs[i][key], rel=1e-12), (shapes[i], key)
    for run in runs:
        run.close()


def test_noalloc_rejects_grids_above_its_limit():
    import torch

    from paper_2012_08758_b300 import binding as B

    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    n = 257  # 257^3 > 2^24 points
    with pytest.raises(B.MhdError) as e:
        B.mhd_diagnostics_noalloc(dummy.data_ptr(), B.MHD_F64, n, n, n, 1.0, 1.0, 1.0, 1.0, dummy.data_ptr())
    assert e.value.code == B.MHD_EINVAL and "no-allocation limit" in str(e.value)
