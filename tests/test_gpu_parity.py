"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances: states, relative L-infinity per field
with the scale of its physical quantity (tests/gpu_util.rel_linf_state) and,
for every u / A component that is not degenerate, with its own max|q|
(tests/gpu_util.per_field_linf): FP64 1e-12, FP32 2e-5; right-hand sides,
relative L-infinity per field: FP64 1e-12, FP32 1e-5."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_08758_b300 import inputs
from tests.gpu_util import (assert_state_matches, gpu_params, oracle_params, oracle_state, rel_linf,
                            rel_linf_state)
from tests.states import coords, k2sq_mod, rk3_gain

pytestmark = pytest.mark.gpu

C1 = dict(nx=32, ny=32, nz=32, nu=5e-3, eta=5e-3, f0=0.02, sigma=0.0, kmin=2.5, kmax=3.5, seed=1,
          cfl=0.4)


def make_run(**kw):
    from paper_2012_08758_b300.run import Run
    return Run(**gpu_params(**kw))


# --------------------------------------------------------------------------
# Forcing draw: integer k bit-exact, the rest to FP64 rounding
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed,sigma,shell", [(1, 0.0, (2.5, 3.5)), (123456789, 1.0, (4.5, 5.5)),
                                              (2**62 + 7, 0.3, (1.0, 2.0))])
def test_forcing_draw_matches_oracle(seed, sigma, shell):
    kw = dict(nx=16, ny=16, nz=16, f0=0.02, sigma=sigma, kmin=shell[0], kmax=shell[1], seed=seed)
    run = make_run(**kw)
    p = oracle_params(**kw)
    for step in (0, 1, 2, 17, 1000, 123456):
        g = run.forcing_draw(step)
        o = O.forcing_draw(p, step)
        assert g["k"] == o.k
        assert abs(g["phi"] - o.phi) < 1e-14
        for key in ("e", "a", "b"):
            np.testing.assert_allclose(g[key], getattr(o, key), atol=1e-14)
    run.close()


# --------------------------------------------------------------------------
# Right-hand side through the fused substep kernel
# --------------------------------------------------------------------------
SHAPES = [(32, 32, 32), (37, 23, 11), (40, 8, 20), (12, 9, 1), (16, 1, 1), (1, 1, 1)]


KERNELS = [(2, 0), (1, 0)]  # (kernel, tile): TMA default tile, plane ring
TMA_TILES = [(2, t) for t in range(1, 29)]


@pytest.mark.parametrize("kernel,tile", KERNELS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_rhs_matches_oracle(shape, dtype, tol, kernel, tile):
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.02, eta=0.03, cs=1.1, f0=0.05, sigma=0.7, kmin=1.0,
              kmax=2.0, seed=5, dtype=dtype, kernel=kernel, tile=tile)
    q = inputs.random_modes_state(nx, ny, nz, seed=3, amp=0.3) + inputs.noise_state(nx, ny, nz, seed=4,
                                                                                    amp=0.02)
    run = make_run(**kw)
    run.set_state(q)
    got = run.eval_rhs(step=9, dt_forcing=0.05)
    p = oracle_params(**kw)
    F = O.forcing_draw(p, 9, dt=0.05)
    want = O.rhs(p, q, F)
    # RHS fields here are O(0.1-10); a field that is zero up to rounding
    # (e.g. on a 1-point grid) is compared absolutely at tol * 1e-3
    err = rel_linf(got, want, floor=1e-3)
    assert err.max() < tol, err
    run.close()


@pytest.mark.parametrize("kernel,tile", KERNELS + [(2, 7)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_rhs_with_unequal_box_lengths(dtype, tol, kernel, tile):
    """Box lengths 4 x 3 x 2.5 (three different spacings and physical forcing
    wave vectors 2 pi k / L_a): the anisotropic weights of every stencil and
    the forcing phase per axis against the oracle."""
    if dtype == "f64" and tile == 7:
        pytest.skip("packed FP32 tile")
    nx, ny, nz = 36, 28, 20
    kw = dict(nx=nx, ny=ny, nz=nz, lx=4.0, ly=3.0, lz=2.5, nu=0.02, eta=0.03, cs=0.9, f0=0.05, sigma=0.6,
              kmin=1.0, kmax=2.5, seed=13, dtype=dtype, kernel=kernel, tile=tile)
    q = inputs.random_modes_state(nx, ny, nz, seed=23, amp=0.3) + inputs.noise_state(nx, ny, nz, seed=24,
                                                                                    amp=0.02)
    run = make_run(**kw)
    run.set_state(q)
    got = run.eval_rhs(step=4, dt_forcing=0.02)
    p = oracle_params(**kw)
    want = O.rhs(p, q, O.forcing_draw(p, 4, dt=0.02))
    err = rel_linf(got, want, floor=1e-3)
    assert err.max() < tol, err
    run.step(3)
    got_q, _, _ = run.get_state()
    q1 = q.copy()
    O.run(p, q1, 3)
    assert_state_matches(got_q, q1, dtype, cs=0.9)
    run.close()


# --------------------------------------------------------------------------
# Full steps (C1: 32^3, forcing, CFL dt, 20 steps)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,tile", KERNELS)
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_c1_step_parity(dtype, tol, kernel, tile):
    kw = dict(C1, dtype=dtype, kernel=kernel, tile=tile)
    q0 = inputs.seed_field_state(32, seed=0)
    run = make_run(**kw)
    run.set_state(q0)
    p = oracle_params(**kw)
    q = q0.copy()
    t_or = 0.0
    done = 0
    for target in (1, 20):
        run.step(target - done)
        t_o, dts = O.run(p, q, target - done, step0=done, t0=t_or)
        t_or = t_o
        done = target
        got, t_gpu, step_gpu = run.get_state()
        assert step_gpu == target
        assert abs(t_gpu - t_or) <= (1e-13 if dtype == "f64" else 1e-6) * t_or
        assert_state_matches(got, q, dtype, cs=1.0, what=f"after step {target}")
    run.close()


@pytest.mark.parametrize("kernel,tile", KERNELS)
@pytest.mark.parametrize("shape", [(37, 23, 11), (24, 24, 1), (1, 1, 1), (9, 40, 7)])
def test_ragged_and_degenerate_step_parity(shape, kernel, tile):
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0,
              seed=11, dtype="f64", kernel=kernel, tile=tile)
    q0 = inputs.random_modes_state(nx, ny, nz, seed=8, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(4)
    got, t, _ = run.get_state()
    q = q0.copy()
    O.run(oracle_params(**kw), q, 4)
    assert_state_matches(got, q, "f64")
    run.close()


@pytest.mark.parametrize("kernel,tile", TMA_TILES)
def test_every_tma_tile_fp32_step_parity(kernel, tile):
    """Each FP32 tile variant of the TMA kernel: ragged grid, 5 forced steps."""
    kw = dict(nx=45, ny=37, nz=29, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0,
              seed=4, dtype="f32", kernel=kernel, tile=tile)
    q0 = inputs.random_modes_state(45, 37, 29, seed=12, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(5)
    got, _, _ = run.get_state()
    q = q0.copy()
    O.run(oracle_params(**kw), q, 5)
    assert_state_matches(got, q, "f32")
    d = run.diagnostics()  # reductions run with this tile's block shape
    o = O.diagnostics(oracle_params(**kw), q)
    for key in ("urms", "brms", "ekin", "emag", "mass", "vmax"):
        assert d[key] == pytest.approx(o[key], rel=2e-5), key
    run.close()


@pytest.mark.parametrize("tile", [1, 2, 3, 4])
def test_every_fp64_tma_tile_step_parity(tile):
    """Each FP64 tile variant of the TMA kernel: ragged grid, 4 forced steps,
    1e-12 of the oracle."""
    kw = dict(nx=45, ny=37, nz=29, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0,
              seed=4, dtype="f64", kernel=2, tile=tile)
    q0 = inputs.random_modes_state(45, 37, 29, seed=12, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(4)
    got, _, _ = run.get_state()
    run.close()
    q = q0.copy()
    O.run(oracle_params(**kw), q, 4)
    assert_state_matches(got, q, "f64")


SCALAR_TMA_TILES = [1, 2, 3, 4, 5, 6, 9, 10, 11, 12, 13, 14, 15, 16]


@pytest.mark.parametrize("shape", [(45, 37, 29), (40, 40, 40)])
def test_tma_tiles_give_the_same_bits(shape):
    """The tile shape, stage count and barrier spacing of the TMA kernel
    change only the schedule, never a point's arithmetic: every scalar
    variant steps a forced run to the same bits (anisotropic and isotropic
    spacings; the work split differs per tile)."""
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=4,
              dtype="f32", kernel=2)
    from paper_2012_08758_b300 import binding as B
    q0 = inputs.random_modes_state(nx, ny, nz, seed=12, amp=0.2)
    ref = None
    for tile in SCALAR_TMA_TILES:
        run = make_run(tile=tile, **kw)
        run.set_state(q0)
        run.step(4)
        q, t, _ = run.get_state()
        b = run.reduce(B.MHD_BRMS)
        run.close()
        if ref is None:
            ref = (q, t, b)
        assert t == ref[1] and b == ref[2] and np.array_equal(q, ref[0]), tile


# --------------------------------------------------------------------------
# Paired-point FP32 kernel (two x-points per thread, 64-wide tiles)
# --------------------------------------------------------------------------
X2_TILES = [17, 19, 20, 25, 26, 28]


@pytest.mark.parametrize("tile", X2_TILES)
@pytest.mark.parametrize("shape", SHAPES + [(65, 9, 14), (128, 24, 16), (63, 40, 7)])
def test_paired_kernel_rhs_matches_oracle(shape, tile):
    """Ragged x extents (odd, one past a tile, one short of two tiles), thin
    and one-point axes: both points of a pair, and the lone last point."""
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.02, eta=0.03, cs=1.1, f0=0.05, sigma=0.7, kmin=1.0,
              kmax=2.0, seed=5, dtype="f32", kernel=2, tile=tile)
    q = inputs.random_modes_state(nx, ny, nz, seed=3, amp=0.3) + inputs.noise_state(nx, ny, nz, seed=4, amp=0.02)
    run = make_run(**kw)
    run.set_state(q)
    got = run.eval_rhs(step=9, dt_forcing=0.05)
    p = oracle_params(**kw)
    want = O.rhs(p, q, O.forcing_draw(p, 9, dt=0.05))
    err = rel_linf(got, want, floor=1e-3)
    assert err.max() < 1e-5, err
    run.close()


@pytest.mark.parametrize("tile", [17, 19])
def test_paired_kernel_steps_match_oracle(tile):
    """C1 (32^3, forcing, CFL dt) for 20 steps, and an anisotropic ragged box
    with once-per-step forcing and upwinding for 6 steps."""
    kw = dict(C1, dtype="f32", kernel=2, tile=tile)
    q0 = inputs.seed_field_state(32, seed=0)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(20)
    got, t, _ = run.get_state()
    run.close()
    want, t_or = oracle_state(q0, 20, **kw)
    assert abs(t - t_or) <= 1e-6 * t_or
    assert_state_matches(got, want, "f32")
    kw = dict(nx=70, ny=22, nz=18, lx=4.0, ly=3.0, lz=2.5, nu=0.01, eta=0.02, f0=0.05, sigma=1.0, kmin=1.0,
              kmax=2.5, seed=7, forcing_mode=1, upwind=1, dtype="f32", kernel=2, tile=tile)
    q0 = inputs.random_modes_state(70, 22, 18, seed=9, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(6)
    got, _, _ = run.get_state()
    run.close()
    want, _ = oracle_state(q0, 6, **kw)
    assert_state_matches(got, want, "f32")


@pytest.mark.parametrize("shape", [(128, 24, 16), (70, 22, 18), (64, 8, 1)])
def test_interleaved_w_layout_steps_bit_for_bit_like_tile_26(shape):
    """Tile 28 is tile 26 with w's fields 0-5 in the interleaved layout: the
    same arithmetic in the same order, so 5 forced, upwinded steps (and the
    RHS) agree bit for bit, ragged tiles and a single plane included."""
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.01, eta=0.02, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=7,
              upwind=1, dtype="f32", kernel=2)
    q0 = inputs.random_modes_state(nx, ny, nz, seed=9, amp=0.2)
    out = []
    for tile in (26, 28):
        run = make_run(tile=tile, **kw)
        run.set_state(q0)
        rhs = run.eval_rhs(step=2, dt_forcing=0.01)
        run.step(5)
        out.append((rhs, run.get_state()))
        run.close()
    (ra, (qa, ta, sa)), (rb, (qb, tb, sb)) = out
    assert np.array_equal(ra, rb)
    assert sa == sb == 5 and ta == tb and np.array_equal(qa, qb)


# --------------------------------------------------------------------------
# Upwinding of the continuity equation (upwind = 1)
# --------------------------------------------------------------------------
UPWIND_KERNELS = [(2, 0), (1, 0), (2, 1), (2, 7), (2, 17), (2, 25), (2, 26), (2, 28)]


@pytest.mark.parametrize("kernel,tile", UPWIND_KERNELS)
@pytest.mark.parametrize("shape", [(32, 32, 32), (37, 23, 11), (12, 9, 1)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_upwinded_rhs_matches_oracle(shape, dtype, tol, kernel, tile):
    if dtype == "f64" and tile > 4:
        pytest.skip("packed FP32 tile")
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.02, eta=0.03, cs=1.1, f0=0.05, sigma=0.7, kmin=1.0,
              kmax=2.0, seed=5, dtype=dtype, kernel=kernel, tile=tile, upwind=1)
    # flows of both signs on every axis, and grid-scale structure in ln rho
    q = inputs.random_modes_state(nx, ny, nz, seed=13, amp=0.4) + inputs.noise_state(nx, ny, nz, seed=14,
                                                                                     amp=0.05)
    run = make_run(**kw)
    run.set_state(q)
    got = run.eval_rhs(step=3, dt_forcing=0.05)
    p = oracle_params(**kw)
    want = O.rhs(p, q, O.forcing_draw(p, 3, dt=0.05))
    err = rel_linf(got, want, floor=1e-3)
    assert err.max() < tol, err
    # the upwinding changed the continuity equation and nothing else
    central = O.rhs(oracle_params(**dict(kw, upwind=0)), q, O.forcing_draw(p, 3, dt=0.05))
    assert np.abs(want[0] - central[0]).max() > 100 * tol * np.abs(want[0]).max()
    assert np.array_equal(want[1:], central[1:])
    run.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_upwinded_step_parity(dtype, tol):
    """C1 with upwinding: 32^3, forcing, CFL dt, 10 steps from a state with
    density and velocity structure."""
    kw = dict(C1, dtype=dtype, upwind=1)
    q0 = inputs.random_modes_state(32, 32, 32, seed=21, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(10)
    got, t_gpu, _ = run.get_state()
    q = q0.copy()
    t_or, _ = O.run(oracle_params(**kw), q, 10)
    assert abs(t_gpu - t_or) <= (1e-13 if dtype == "f64" else 1e-6) * t_or
    assert_state_matches(got, q, dtype, cs=1.0)
    run.close()


def test_forcing_once_per_step_mode():
    kw = dict(nx=20, ny=16, nz=12, nu=0.01, eta=0.01, f0=0.05, sigma=0.5, kmin=1.0, kmax=2.0,
              seed=3, forcing_mode=1, dtype="f64")
    q0 = inputs.random_modes_state(20, 16, 12, seed=2, amp=0.1)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(3)
    got, _, _ = run.get_state()
    q = q0.copy()
    O.run(oracle_params(**kw), q, 3)
    assert_state_matches(got, q, "f64")
    run.close()


def test_fixed_dt_and_clock():
    kw = dict(nx=16, ny=16, nz=16, dt_fixed=1.19209e-3, dtype="f64")
    q0 = inputs.uniform_state(16, seed=1, lo=0.0, hi=0.1)
    run = make_run(**kw)
    run.set_state(q0, t=2.0, step=7)
    run.step(5)
    got, t, step = run.get_state()
    assert step == 12 and abs(t - (2.0 + 5 * 1.19209e-3)) < 1e-14
    q = q0.copy()
    O.run(oracle_params(**kw), q, 5, step0=7)
    assert_state_matches(got, q, "f64")
    tt, dtl, st = run.time()
    assert dtl == 1.19209e-3 and st == 12
    run.close()


# --------------------------------------------------------------------------
# Closed forms checked directly on the GPU (also at full size)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,dtype,tol", [(24, "f64", 1e-13), (64, "f32", 2e-6)])
def test_beltrami_decay_on_gpu(n, dtype, tol):
    k, eta, dt, ns = 2, 0.05, 0.02, 6
    run = make_run(nx=n, ny=n, nz=n, eta=eta, nu=0.01, dt_fixed=dt, dtype=dtype)
    X, Y, Z = coords(n, n, n)
    q = np.zeros((7, n, n, n))
    q[4], q[5] = np.sin(k * Z), np.cos(k * Z)
    run.set_state(q)
    run.step(ns)
    got, _, _ = run.get_state()
    g = rk3_gain(-eta * k2sq_mod(k, 2 * math.pi / n) * dt) ** ns
    assert np.abs(got[4] - g * np.sin(k * Z)).max() < tol
    assert np.abs(got[5] - g * np.cos(k * Z)).max() < tol
    assert np.abs(got[[0, 1, 2, 3, 6]]).max() < tol
    run.close()


@pytest.mark.slow
def test_full_size_256_sampled_rhs_and_beltrami():
    """The 256^3 FP32 launch configuration of the benchmark: RHS at sampled
    points against the oracle point by point, and the Beltrami closed form
    after full steps."""
    n = 256
    kw = dict(nx=n, ny=n, nz=n, nu=2e-4, eta=2e-4, f0=0.02, sigma=1.0, kmin=2.5, kmax=3.5,
              seed=1, dtype="f32")
    q = inputs.random_modes_state(n, seed=21, amp=0.2, kmax=4, nmodes=4)
    q += inputs.noise_state(n, seed=22, amp=1e-3)
    run = make_run(**kw)
    run.set_state(q)
    got = run.eval_rhs(step=4, dt_forcing=0.01)
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(200)]
    pts += [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 3), (n - 3, 2, n - 1)]
    p = oracle_params(**kw)
    F = O.forcing_draw(p, 4, dt=0.01)
    want = O.rhs_at(p, q, pts, F)
    g = np.array([[got[f, k, j, i] for f in range(7)] for (i, j, k) in pts])
    scale = np.abs(want).max(axis=0)
    assert (np.abs(g - want).max(axis=0) / scale).max() < 1e-5
    run.close()
    del q, got
    k, eta, dt, ns = 3, 2e-3, 5e-3, 3
    run = make_run(nx=n, ny=n, nz=n, eta=eta, nu=2e-3, dt_fixed=dt, dtype="f32")
    X, Y, Z = coords(n, n, n)
    qb = np.zeros((7, n, n, n), dtype=np.float32)
    qb[4], qb[5] = np.sin(k * Z), np.cos(k * Z)
    run.set_state(qb)
    run.step(ns)
    out, _, _ = run.get_state(dtype=np.float32)
    gk = rk3_gain(-eta * k2sq_mod(k, 2 * math.pi / n) * dt) ** ns
    assert np.abs(out[4] - gk * np.sin(k * Z)).max() < 2e-6
    # FP32 rounding of the second-derivative stencils grows like eps/h^2
    # (the weights sum to 18.1/h^2 over three axes while the result is
    # ~k^2): j carries ~eps * 18.1 |A| / h^2, so j x B, and from it u, ln rho
    # and A_z, stay below t |B| eps 18.1 |A| / h^2 (~8e-5 here; exactly 0 in
    # exact arithmetic).
    h = 2 * math.pi / n
    bound = ns * dt * 3.0 * 6e-8 * 18.1 / h ** 2
    assert np.abs(out[[0, 1, 2, 3, 6]]).max() < bound
    run.close()


# --------------------------------------------------------------------------
# Diagnostics, state transfer, batching, determinism, failure detection
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-14), ("f32", 1e-5)])
def test_diagnostics_match_oracle(dtype, tol):
    """Volume means and maxima against the oracle.  In FP64 the per-point
    values round like the oracle's and the fixed-order FP64 sums (per-thread
    z sums, warp butterflies, tile partials) stay within a few ulp of its
    pairwise sums: 1e-14 relative (measured worst 4e-16 over five grids)."""
    kw = dict(nx=30, ny=20, nz=18, dtype=dtype)
    q = inputs.random_modes_state(30, 20, 18, seed=6, amp=0.4)
    run = make_run(**kw)
    run.set_state(q)
    d = run.diagnostics()
    o = O.diagnostics(oracle_params(**kw), q)
    for key in ("urms", "brms", "umax", "bmax", "ekin", "emag", "mass", "vmax"):
        assert d[key] == pytest.approx(o[key], rel=tol), key
    assert d["divb_max"] < (1e-12 if dtype == "f64" else 1e-4) * d["bmax"] * 30 / (2 * math.pi)
    run.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fused_brms_equals_full_diagnostics(dtype):
    """mhd_reduce(B_rms) runs its own one-pass kernel; it must give the B_rms
    of the full diagnostics (same per-point values, tiles and order)."""
    from paper_2012_08758_b300 import binding as B
    kw = dict(nx=37, ny=23, nz=19, dtype=dtype)
    q = inputs.random_modes_state(37, 23, 19, seed=31, amp=0.3) + inputs.noise_state(37, 23, 19, seed=32,
                                                                                    amp=0.05)
    run = make_run(**kw)
    run.set_state(q)
    fast = run.reduce(B.MHD_BRMS)
    full = run.diagnostics()["brms"]
    assert fast == pytest.approx(full, rel=1e-13)
    assert fast == pytest.approx(O.diagnostics(oracle_params(**kw), q)["brms"], rel=1e-14 if dtype == "f64" else 1e-5)
    run.close()


@pytest.mark.parametrize("kernel,tile", [(2, 0), (1, 0)])
def test_brms_sampling_leaves_the_run_unchanged(kernel, tile):
    """Sampling B_rms after every step (the TMA runs cache the CFL maximum of
    that sweep for the next step's prologue) gives bit-for-bit the run that
    is never sampled, and each sample equals the full diagnostics' B_rms."""
    from paper_2012_08758_b300 import binding as B
    kw = dict(nx=40, ny=24, nz=20, nu=5e-3, eta=5e-3, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=9,
              dtype="f32", kernel=kernel, tile=tile)
    q0 = inputs.random_modes_state(40, 24, 20, seed=14, amp=0.3)
    a, b = make_run(**kw), make_run(**kw)
    a.set_state(q0)
    b.set_state(q0)
    for _ in range(6):
        a.step(1)
        b.step(1)
        fast = a.reduce(B.MHD_BRMS)
        assert fast == pytest.approx(a.diagnostics()["brms"], rel=1e-13)
    qa, ta, sa = a.get_state()
    qb, tb, sb = b.get_state()
    assert sa == sb == 6 and ta == tb and np.array_equal(qa, qb)
    a.close()
    b.close()


def test_state_write_after_brms_drops_the_cached_maximum():
    """A B_rms reduction caches the CFL maximum of the current state; writing
    a new state (faster flow, same step number) must not reuse it: the next
    step takes the dt of the new state, as a fresh run does."""
    from paper_2012_08758_b300 import binding as B
    kw = dict(nx=24, ny=24, nz=24, nu=5e-3, eta=5e-3, f0=0.0, dtype="f32")
    slow = inputs.random_modes_state(24, 24, 24, seed=15, amp=0.05)
    fast = inputs.random_modes_state(24, 24, 24, seed=16, amp=0.6)
    a, b = make_run(**kw), make_run(**kw)
    a.set_state(slow)
    a.reduce(B.MHD_BRMS)
    a.set_state(fast)
    b.set_state(fast)
    a.step(1)
    b.step(1)
    (qa, ta, _), (qb, tb, _) = a.get_state(), b.get_state()
    assert ta == tb and np.array_equal(qa, qb)
    a.set_seed_field(3, 1e-3)  # the device initial condition is a state write too
    b.set_seed_field(3, 1e-3)
    a.reduce(B.MHD_BRMS)
    a.set_state(fast)
    b.set_state(fast)
    a.step(2)
    b.step(2)
    (qa, ta, _), (qb, tb, _) = a.get_state(), b.get_state()
    assert ta == tb and np.array_equal(qa, qb)
    a.close()
    b.close()


@pytest.mark.parametrize("kernel,tile", KERNELS)
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_ideal_mhd_step_parity(dtype, tol, kernel, tile):
    """nu = eta = 0 (ideal MHD): the diffusive time-step limit drops out
    (dt from the CFL speed alone) and the viscous and resistive terms vanish;
    five forced steps against the oracle."""
    kw = dict(nx=28, ny=24, nz=20, nu=0.0, eta=0.0, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=21,
              dtype=dtype, kernel=kernel, tile=tile)
    q0 = inputs.random_modes_state(28, 24, 20, seed=31, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(5)
    got, t, _ = run.get_state()
    q = q0.copy()
    t_o, _ = O.run(oracle_params(**kw), q, 5)
    assert abs(t - t_o) <= (1e-13 if dtype == "f64" else 1e-6) * t_o
    assert_state_matches(got, q, dtype)
    run.close()


def test_state_roundtrip_is_exact():
    q = inputs.noise_state(13, 7, 5, seed=1, amp=1.0)
    run = make_run(nx=13, ny=7, nz=5, dtype="f64")
    run.set_state(q, t=1.5, step=3)
    back, t, step = run.get_state()
    assert np.array_equal(back, q) and t == 1.5 and step == 3
    run.close()
    q32 = q.astype(np.float32)
    run = make_run(nx=13, ny=7, nz=5, dtype="f32")
    run.set_state(q32)
    back, _, _ = run.get_state(dtype=np.float32)
    assert np.array_equal(back, q32)
    run.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_checkpoint_resume_is_bit_for_bit(dtype, tmp_path):
    """A run checkpointed at step 4 and restored into a new context continues
    exactly as the uninterrupted run (state, t, forcing draws: the random
    numbers are counter-based, keyed by seed and step)."""
    from paper_2012_08758_b300.run import Run
    kw = dict(nx=24, ny=20, nz=16, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0,
              seed=2**62 + 9, dtype=dtype, upwind=1)
    a = make_run(**kw)
    a.set_seed_field(5, 1e-3)
    a.step(4)
    path = str(tmp_path / "ck.npz")
    a.checkpoint(path)
    a.step(6)
    qa, ta, sa = a.get_state()
    b = Run.restore(path)
    assert b.params.seed == 2**62 + 9 and b.params.upwind == 1
    b.step(6)
    qb, tb, sb = b.get_state()
    assert sa == sb == 10 and ta == tb
    assert np.array_equal(qa, qb)
    a.close()
    b.close()


@pytest.mark.parametrize("kernel,tile", [(2, 0), (1, 0), (2, 2), (2, 9), (2, 17), (2, 25), (2, 26)])
@pytest.mark.parametrize("shape,dtype", [((32, 32, 32), "f32"), ((37, 23, 11), "f64"), ((12, 9, 1), "f32"),
                                         ((16, 1, 1), "f64"), ((40, 8, 20), "f32")])
def test_padding_canaries_survive_every_entry_point(shape, dtype, kernel, tile):
    """The alignment padding of both state buffers holds NaN from creation on:
    no kernel of any entry point (uploads, seed field, steps with forcing and
    upwinding, RHS evaluation, diagnostics, B_rms, spectrum, batch steps,
    downloads) writes there, and since every result stays finite none reads it."""
    from paper_2012_08758_b300 import binding as B
    from paper_2012_08758_b300.run import Batch
    if dtype == "f64" and tile > 2:
        pytest.skip("FP32 tile")
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=4,
              dtype=dtype, kernel=kernel, tile=tile, upwind=1)
    run = make_run(**kw)
    assert B.mhd_padding_check(run.ctx) == 0
    run.set_state(inputs.random_modes_state(nx, ny, nz, seed=5, amp=0.2))
    run.step(3)
    run.eval_rhs(step=3, dt_forcing=0.01)
    d = run.diagnostics()
    assert np.isfinite(run.reduce(B.MHD_BRMS)) and all(np.isfinite(v) for v in d.values())
    if nx >= 2:
        assert np.all(np.isfinite(run.spectrum()))
    run.set_seed_field(7, 1e-3)
    other = make_run(**kw)
    other.set_state(inputs.random_modes_state(nx, ny, nz, seed=6, amp=0.2), step=1)
    b = Batch([run, other])
    b.step(4)
    b.close()
    for r in (run, other):
        q, _, _ = r.get_state()
        assert np.all(np.isfinite(q))
        assert B.mhd_padding_check(r.ctx) == 0
        r.close()


def test_batch_is_bitwise_identical_to_alone():
    from paper_2012_08758_b300.run import Batch
    cfgs = [dict(nx=32, ny=32, nz=32, f0=0.02, sigma=1.0, seed=1, nu=4e-3, eta=4e-3),
            dict(nx=48, ny=40, nz=24, f0=0.02, sigma=0.0, seed=2, nu=2e-3, eta=2e-3),
            dict(nx=17, ny=19, nz=23, f0=0.03, sigma=1.0, seed=3, nu=5e-3, eta=5e-3)]
    states = [inputs.seed_field_state(c["nx"], c["ny"], c["nz"], seed=i, amp=1e-3)
              for i, c in enumerate(cfgs)]
    alone = []
    for c, q in zip(cfgs, states):
        r = make_run(**c)
        r.set_state(q)
        r.step(7)
        alone.append(r.get_state(dtype=np.float32)[0])
        r.close()
    runs = [make_run(**c) for c in cfgs]
    for r, q in zip(runs, states):
        r.set_state(q)
    b = Batch(runs)
    b.step(5)  # graph of 5 steps
    b.step(2)  # replay path / direct remainder
    for c, q0, r, ref in zip(cfgs, states, runs, alone):
        got, t, step = r.get_state(dtype=np.float32)
        assert step == 7
        assert np.array_equal(got, ref)
        # and the batched run against the FP64 oracle from the same state
        want, t_or = oracle_state(q0, 7, **c)
        assert abs(t - t_or) <= 1e-6 * t_or
        assert_state_matches(got.astype(np.float64), want, "f32", what=str(c))
        d, o = r.diagnostics(), O.diagnostics(oracle_params(**c), want)
        for key in ("urms", "brms", "ekin", "emag", "mass", "vmax"):
            assert d[key] == pytest.approx(o[key], rel=2e-5), (c, key)
    b.close()
    for r in runs:
        r.close()


def test_fp64_batch_matches_oracle():
    """An FP64 batch of three runs of different sizes (one ragged, one
    anisotropic, forced and unforced, CFL and fixed dt), stepped with a
    captured graph and its remainder: each run within 1e-12 of the FP64
    oracle, diagnostics within 1e-12."""
    from paper_2012_08758_b300.run import Batch
    cfgs = [dict(nx=32, ny=32, nz=32, f0=0.02, sigma=1.0, seed=1, nu=4e-3, eta=4e-3, dtype="f64"),
            dict(nx=37, ny=23, nz=11, f0=0.05, sigma=0.0, seed=2, nu=5e-3, eta=3e-3, dtype="f64", upwind=1),
            dict(nx=24, ny=20, nz=28, lx=4.0, ly=3.0, lz=3.5, f0=0.0, seed=3, nu=5e-3, eta=5e-3,
                 dt_fixed=3e-3, dtype="f64")]
    states = [inputs.random_modes_state(c["nx"], c["ny"], c["nz"], seed=30 + i, amp=0.15)
              + inputs.noise_state(c["nx"], c["ny"], c["nz"], seed=40 + i, amp=1e-3)
              for i, c in enumerate(cfgs)]
    runs = [make_run(**c) for c in cfgs]
    for r, q in zip(runs, states):
        r.set_state(q)
    b = Batch(runs)
    b.step(4)
    b.step(2)
    for c, q0, r in zip(cfgs, states, runs):
        got, t, step = r.get_state()
        assert step == 6
        want, t_or = oracle_state(q0, 6, **c)
        assert abs(t - t_or) <= 1e-13 * t_or
        assert_state_matches(got, want, "f64", what=str(c))
        d, o = r.diagnostics(), O.diagnostics(oracle_params(**c), want)
        for key in ("urms", "brms", "ekin", "emag", "mass", "vmax", "umax", "bmax"):
            assert d[key] == pytest.approx(o[key], rel=1e-12), (c, key)
    b.close()
    for r in runs:
        r.close()


def test_batch_honours_each_runs_own_options():
    """Runs with different per-run options in one batch (upwinding on/off,
    forcing in every substep or once per step, fixed or CFL time step,
    anisotropic box) each give the result they give alone, bit for bit."""
    from paper_2012_08758_b300.run import Batch
    cfgs = [dict(nx=32, ny=32, nz=32, f0=0.02, sigma=1.0, seed=1, nu=4e-3, eta=4e-3, upwind=1),
            dict(nx=40, ny=24, nz=20, f0=0.05, sigma=0.5, seed=2, nu=3e-3, eta=2e-3, forcing_mode=1),
            dict(nx=24, ny=24, nz=36, f0=0.0, seed=3, nu=5e-3, eta=5e-3, dt_fixed=2e-3, upwind=1),
            dict(nx=33, ny=20, nz=18, lx=4.0, ly=3.0, lz=2.5, f0=0.03, sigma=1.0, seed=4, nu=4e-3, eta=4e-3)]
    states = [inputs.random_modes_state(c["nx"], c["ny"], c["nz"], seed=10 + i, amp=0.15)
              for i, c in enumerate(cfgs)]
    alone = []
    for c, q in zip(cfgs, states):
        r = make_run(**c)
        r.set_state(q)
        r.step(6)
        alone.append(r.get_state(dtype=np.float32)[0])
        r.close()
    runs = [make_run(**c) for c in cfgs]
    for r, q in zip(runs, states):
        r.set_state(q)
    b = Batch(runs)
    b.step(6)
    for c, q0, r, ref in zip(cfgs, states, runs, alone):
        got, _, step = r.get_state(dtype=np.float32)
        assert step == 6 and np.array_equal(got, ref)
        want, _ = oracle_state(q0, 6, **c)
        cs = c.get("cs", 1.0)
        assert_state_matches(got.astype(np.float64), want, "f32", cs=cs, what=str(c))
    b.close()
    for r in runs:
        r.close()


def test_runs_are_deterministic():
    outs = []
    for _ in range(2):
        r = make_run(**dict(C1, dtype="f32"))
        r.set_state(inputs.seed_field_state(32, seed=0))
        r.step(6)
        outs.append((r.get_state(dtype=np.float32)[0], r.diagnostics()))
        r.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_zero_steps_is_a_noop():
    q = inputs.noise_state(8, seed=2)
    r = make_run(nx=8, ny=8, nz=8, dtype="f64")
    r.set_state(q)
    r.step(0)
    back, t, st = r.get_state()
    assert np.array_equal(back, q) and t == 0.0 and st == 0
    r.close()


def test_bounded_wait_gives_up_and_leaves_the_gpu_usable():
    """Failure detection of the device waits without a fault: the self-test
    kernel waits, with the bounded mbarrier wait of every TMA kernel (poll
    count cut 1024-fold), on an mbarrier that nothing arrives on.  The wait
    must give up and report status bit 1 (MHD_ETIMEOUT), the kernels' own
    bound scaled from it must stay within a few seconds (about 1 s on B300), and afterwards the GPU runs
    forced steps that still match the oracle."""
    from paper_2012_08758_b300 import binding as B
    rc, seconds, bound = B.mhd_wait_selftest()
    assert rc == B.MHD_ETIMEOUT, (rc, B.mhd_last_error())
    assert 0.0 < seconds < 0.5 and 0.0 < bound < 5.0, (seconds, bound)
    kw = dict(C1, dtype="f64")
    q0 = inputs.random_modes_state(32, seed=2, amp=0.2)
    run = make_run(**kw)
    run.set_state(q0)
    run.step(2)
    got, _, _ = run.get_state()
    q = q0.copy()
    O.run(oracle_params(**kw), q, 2)
    assert_state_matches(got, q, "f64")
    run.close()


def test_blow_up_is_reported_not_hidden():
    """A NaN planted in the host-side upload makes the dt reduction
    non-finite; the next synchronising call reports it."""
    from paper_2012_08758_b300 import binding as B
    q = inputs.seed_field_state(16, seed=0)
    q[1, 3, 4, 5] = np.nan
    r = make_run(nx=16, ny=16, nz=16, dtype="f32")
    r.set_state(q)
    r.step(2)
    with pytest.raises(B.MhdError) as e:
        r.sync()
    assert e.value.code == B.MHD_ENONFINITE
    r.close()
