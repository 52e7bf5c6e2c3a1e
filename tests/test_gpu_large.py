"""Sampled right-hand sides (mhd_eval_rhs_at) and the largest grids.

A grid whose state does not fit the host (1024^3 FP32: 92 GB of device
memory, per-field offsets beyond 2^32 bytes) is checked point by point: the
device seed field is rebuilt on the host at the 7^3 neighbourhood of each
sampled point from the same counter-based generator, and the FP64 oracle
evaluates the right-hand side at the centre of that neighbourhood (a 7^3
periodic box with the large grid's spacing: every stencil of Sec. 2 -- the
diagonal mixed ones included -- reaches at most 3 points along each axis,
so the centre sees exactly the large grid's values)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_08758_b300 import inputs
from tests.gpu_util import gpu_params, oracle_params


def make_run(**kw):
    from paper_2012_08758_b300.run import Run
    return Run(**gpu_params(**kw))


def local_rhs(n, pts, seed, amp, **phys):
    """Oracle RHS of the seed-field state of an n^3 grid at the listed points,
    each from its own 7^3 neighbourhood (forcing off)."""
    h = 2 * math.pi / n
    p = O.Params(nx=7, ny=7, nz=7, lx=7 * h, ly=7 * h, lz=7 * h, **phys)
    d = np.arange(-3, 4)
    K, J, I = np.meshgrid(d, d, d, indexing="ij")
    out = []
    for (i, j, k) in pts:
        a = inputs.counter_seed_field_at(n, n, n, I.ravel() + i, J.ravel() + j, K.ravel() + k, seed=seed, amp=amp)
        q = np.zeros((7, 7, 7, 7))
        q[4:7] = a.reshape(3, 7, 7, 7)
        out.append(O.rhs_at(p, q, [(3, 3, 3)])[0])
    return np.array(out)


def test_local_neighbourhood_reproduces_the_full_grid_oracle():
    """The test device above, checked on the CPU: on a 24^3 grid the oracle's
    RHS at a point from the 7^3 neighbourhood equals its RHS from the whole
    grid (faces and corners included, where the neighbourhood wraps)."""
    n, seed, amp = 24, 5, 1e-2
    phys = dict(cs=1.0, nu=5e-3, eta=7e-3)
    q = inputs.counter_seed_field_state(n, seed=seed, amp=amp)
    pts = [(0, 0, 0), (23, 23, 23), (1, 22, 12), (12, 5, 0), (7, 13, 19)]
    full = O.rhs_at(O.Params(nx=n, ny=n, nz=n, **phys), q, pts)
    loc = local_rhs(n, pts, seed, amp, **phys)
    np.testing.assert_allclose(loc, full, rtol=0, atol=1e-12 * np.abs(full).max())


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kernel,tile", [(2, 0), (1, 0), (2, 26)])
def test_eval_rhs_at_equals_the_full_rhs(dtype, kernel, tile):
    """The sampled values are the full right-hand side's, bit for bit
    (forcing included; the default tile 28 reads w in the interleaved layout,
    tile 26 field by field), and the state is left untouched."""
    if dtype == "f64" and tile > 4:
        pytest.skip("FP32 tile")
    kw = dict(nx=37, ny=23, nz=19, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=3,
              dtype=dtype, kernel=kernel, tile=tile)
    q0 = inputs.random_modes_state(37, 23, 19, seed=8, amp=0.3)
    run = make_run(**kw)
    run.set_state(q0)
    full = run.eval_rhs(step=5, dt_forcing=0.01)
    rng = np.random.default_rng(1)
    pts = [(0, 0, 0), (36, 22, 18), (36, 0, 18)] + [tuple(int(v) for v in rng.integers(0, (37, 23, 19)))
                                                   for _ in range(50)]
    got = run.eval_rhs_at(pts, step=5, dt_forcing=0.01)
    want = np.array([[full[f, k, j, i] for f in range(7)] for (i, j, k) in pts])
    assert np.array_equal(got, want)
    q, _, _ = run.get_state()
    assert np.array_equal(q, run.get_state()[0])
    run.close()


@pytest.mark.gpu
def test_eval_rhs_at_rejects_points_outside_the_grid():
    from paper_2012_08758_b300 import binding as B
    run = make_run(nx=16, ny=12, nz=8, dtype="f32")
    run.set_state(inputs.random_modes_state(16, 12, 8, seed=2, amp=0.1))
    for bad in ([(16, 0, 0)], [(0, -1, 0)], [(0, 0, 8)]):
        with pytest.raises(B.MhdError):
            run.eval_rhs_at(bad)
    with pytest.raises(B.MhdError):
        run.eval_rhs_at(np.zeros((0, 3), dtype=np.int32))
    assert run.eval_rhs_at([(15, 11, 7)]).shape == (1, 7)  # the run is still usable
    run.close()


@pytest.mark.gpu
@pytest.mark.slow
def test_largest_grid_1024_cubed_sampled_rhs_and_invariants():
    """1024^3 FP32 in the benchmark's launch configuration: the device seed
    field (Sec. 4 initial condition) gives d u/dt = j x B / rho and
    d A/dt = eta lap A; 160 sampled points (faces, edges, corners, random)
    against the FP64 oracle within 1e-5 of each field's scale.  Then two
    steps: dt finite and positive, |div B| at FP32 rounding, the padding
    canaries intact."""
    from paper_2012_08758_b300 import binding as B
    n, seed, amp = 1024, 11, 1e-3
    phys = dict(cs=1.0, nu=5e-3, eta=5e-3)
    run = make_run(nx=n, ny=n, nz=n, dtype="f32", **phys)
    run.set_seed_field(seed, amp)
    rng = np.random.default_rng(4)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 0), (n - 1, 0, n - 1), (2, n - 3, n // 2),
           (n // 2, 1, n - 2), (n - 4, n // 3, 3), (5, 7, n - 1)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(152)]
    got = run.eval_rhs_at(pts)
    want = local_rhs(n, pts, seed, amp, **phys)
    scale = np.maximum(np.abs(want).max(axis=0), 1e-30)
    err = np.abs(got - want).max(axis=0) / scale
    assert err.max() < 1e-5, err
    assert np.abs(got[:, 0]).max() == 0.0  # u = 0: d ln rho/dt vanishes exactly
    run.step(2)
    t, dt_last, step = B.mhd_time(run.ctx)
    assert step == 2 and math.isfinite(dt_last) and dt_last > 0 and t == pytest.approx(2 * dt_last, rel=0.5)
    d = run.diagnostics()
    assert all(math.isfinite(v) for v in d.values())
    assert d["divb_max"] < 1e-4 * d["bmax"] * n / (2 * math.pi)
    assert B.mhd_padding_check(run.ctx) == 0
    run.close()


def _product_state(n, seed, amp=0.2):
    """Each field a sum of two products g(x) h(y) k(z) of random 1-D waves:
    built by broadcasting (cheap at 512^3), with non-zero mixed derivatives."""
    rng = np.random.default_rng(seed)
    c = np.arange(n) * (2 * math.pi / n)
    q = np.zeros((7, n, n, n), dtype=np.float32)
    for f in range(7):
        for _ in range(2):
            kx, ky, kz = rng.integers(1, 6, size=3)
            px, py, pz = rng.uniform(0, 2 * math.pi, size=3)
            a = amp * rng.standard_normal()
            gx = np.cos(kx * c + px).astype(np.float32)
            gy = np.cos(ky * c + py).astype(np.float32)
            gz = np.cos(kz * c + pz).astype(np.float32)
            q[f] += np.float32(a) * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return q


@pytest.mark.gpu
def test_bench_grid_512_cubed_step_sampled_against_oracle_windows():
    """The 512^3 FP32 grid in the benchmark's launch configuration (default
    tile and work split over every SM): one full step (three substeps),
    then 24 sampled points -- corners, faces, random -- against the FP64
    oracle stepping a 25^3 periodic window of the initial state around each
    point with the same dt.  One step reaches 3 substeps x 3 points = 9
    points along each axis, so the window's centre (12 from its edges) sees
    exactly the large grid's values.  Forcing off (its phase is tied to the
    global coordinates), viscosity and resistivity on."""
    n, w, r = 512, 25, 12
    phys = dict(cs=1.0, nu=5e-3, eta=5e-3, f0=0.0, dt_fixed=2e-3)
    q0 = _product_state(n, seed=21)
    run = make_run(nx=n, ny=n, nz=n, dtype="f32", **phys)
    run.set_state(q0)
    run.step(1)
    got, t, step = run.get_state(dtype=np.float32)
    run.close()
    assert step == 1 and t == pytest.approx(2e-3, rel=1e-12)
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 5), (n - 2, 3, n - 1), (255, 1, 510), (2, 300, 0)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(18)]
    h = 2 * math.pi / n
    p = oracle_params(nx=w, ny=w, nz=w, lx=w * h, ly=w * h, lz=w * h, **phys)
    scale = np.abs(q0.reshape(7, -1)).max(axis=1).astype(np.float64)
    d = np.arange(-r, r + 1)
    worst = 0.0
    for (i, j, k) in pts:
        win = q0[:, np.take(np.arange(n), k + d, mode="wrap")][:, :, np.take(np.arange(n), j + d, mode="wrap")][
            :, :, :, np.take(np.arange(n), i + d, mode="wrap")]
        qw = np.ascontiguousarray(win, dtype=np.float64)
        O.run(p, qw, 1)
        err = np.abs(got[:, k, j, i].astype(np.float64) - qw[:, r, r, r]) / scale
        worst = max(worst, float(err.max()))
        assert err.max() < 2e-5, ((i, j, k), err)
    assert worst > 0.0
