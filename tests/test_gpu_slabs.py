"""z-slab domain decomposition on one GPU (Sec. 3.3-3.4): the run cut into
1, 2, 3 or 4 slabs, with the halo exchange overlapped with the inner planes
or after the substep, gives the undecomposed run's state bit for bit and
stays within the FP64 oracle's tolerance; the diagnostics summed over the
slabs equal the undecomposed ones up to rounding."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_08758_b300 import inputs
from tests.gpu_util import assert_state_matches, oracle_params

pytestmark = pytest.mark.gpu

CASES = [
    # (nx, ny, nz), nslabs, overlap, extra params
    ((32, 32, 32), 2, True, dict(f0=0.02, sigma=1.0, seed=1)),
    ((32, 32, 32), 4, False, dict(f0=0.02, sigma=0.0, seed=2)),
    ((24, 20, 37), 3, True, dict(f0=0.05, sigma=0.5, seed=3, upwind=1)),        # ragged slabs 13/12/12
    ((20, 16, 12), 3, True, dict(f0=0.05, sigma=1.0, seed=4)),                  # 4-plane slabs: no inner split
    ((28, 24, 30), 2, True, dict(lx=4.0, ly=3.0, lz=3.5, f0=0.03, seed=5, forcing_mode=1)),
    ((16, 16, 16), 1, True, dict(f0=0.02, seed=6, dt_fixed=2e-3)),              # one slab: self-exchange
    ((70, 20, 24), 2, True, dict(f0=0.05, sigma=1.0, seed=7, kernel=2, tile=18)),  # paired-point kernel
    ((128, 16, 27), 3, False, dict(f0=0.05, sigma=0.3, seed=8, kernel=2, tile=22, upwind=1)),
    ((70, 20, 24), 4, True, dict(f0=0.05, sigma=1.0, seed=9, kernel=2, tile=25)),  # warp-specialised
    ((66, 30, 21), 3, False, dict(f0=0.05, sigma=0.5, seed=10, kernel=2, tile=26)),  # w through TMA
    ((72, 24, 18), 3, True, dict(f0=0.05, sigma=1.0, seed=11, kernel=2, tile=28)),  # interleaved w
]


def _state(shape, seed):
    nx, ny, nz = shape
    return inputs.random_modes_state(nx, ny, nz, seed=seed, amp=0.2) + inputs.noise_state(nx, ny, nz, seed=seed + 1,
                                                                                        amp=1e-3)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,nslabs,overlap,extra", CASES)
def test_slabs_equal_the_undecomposed_run(shape, nslabs, overlap, extra, dtype):
    if dtype == "f64" and extra.get("tile", 0) > 4:
        pytest.skip("FP32 tile")
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.run import Run
    from paper_2012_08758_b300.slabs import Slabs, slab_extents

    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=5e-3, eta=4e-3, dtype=B.MHD_F64 if dtype == "f64" else B.MHD_F32, **extra)
    q0 = _state(shape, 11)
    npd = np.float64 if dtype == "f64" else np.float32
    steps = 5
    run = Run(**kw)
    run.set_state(q0)
    run.step(steps)
    want, t_run, _ = run.get_state(dtype=npd)
    d_run = run.diagnostics()
    run.close()

    sl = Slabs(nslabs, overlap=overlap, **kw)
    assert sl.extents() == slab_extents(nz, nslabs)
    sl.set_state(q0)
    sl.step(2)
    sl.step(steps - 2)
    got, t, step = sl.get_state(dtype=npd)
    d = sl.diagnostics()
    sl.close()
    assert step == steps and t == t_run
    assert np.array_equal(got, want), float(np.abs(got.astype(np.float64) - want).max())
    for key in ("urms", "brms", "umax", "bmax", "ekin", "emag", "mass", "vmax"):
        assert d[key] == pytest.approx(d_run[key], rel=1e-12, abs=1e-300), key
    bound = (1e-11 if dtype == "f64" else 1e-3) * d_run["bmax"] * max(nx, ny, nz)
    assert d["divb_max"] < bound and d_run["divb_max"] < bound
    if dtype == "f64":
        q = q0.copy()
        O.run(oracle_params(**dict(kw, dtype="f64")), q, steps)
        assert_state_matches(got, q, "f64")


def test_slab_state_round_trip_and_validation():
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.slabs import Slabs

    q0 = _state((20, 12, 18), 3)
    with Slabs(3, nx=20, ny=12, nz=18, dtype=B.MHD_F64) as sl:
        sl.set_state(q0, t=1.5, step=7)
        got, t, step = sl.get_state()
        assert np.array_equal(got, q0) and t == 1.5 and step == 7
    with pytest.raises(B.MhdError):
        Slabs(4, nx=8, ny=8, nz=8)        # 2 planes per slab
    with pytest.raises(B.MhdError):
        Slabs(2, nx=8, ny=8, nz=16, kernel=B.MHD_KERNEL_SMEM)
