"""Magnetic energy spectrum E_B(k) (Sec. 5) on the GPU against the FP64
oracle: per shell within 1e-12 (FP64) / 1e-5 (FP32) of the total magnetic
energy, Parseval against the diagnostics, bitwise reproducibility, the state
left untouched, and growth rates of spectral channels within 1%."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_08758_b300 import inputs
from tests.gpu_util import gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def make_run(**kw):
    from paper_2012_08758_b300.run import Run
    return Run(**gpu_params(**kw))


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 20, 16), (17, 9, 12), (40, 8, 1), (16, 1, 9), (8, 1, 1)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_spectrum_matches_oracle(shape, dtype, tol):
    nx, ny, nz = shape
    kw = dict(nx=nx, ny=ny, nz=nz, dtype=dtype)
    q = inputs.random_modes_state(nx, ny, nz, seed=5, amp=0.3) + inputs.noise_state(nx, ny, nz, seed=6,
                                                                                    amp=0.01)
    run = make_run(**kw)
    run.set_state(q)
    got = run.spectrum()
    want = O.spectrum(oracle_params(**kw), q)
    assert got.shape == want.shape
    scale = max(want.sum(), 1e-300)
    assert np.abs(got - want).max() <= tol * scale, np.abs(got - want).max() / scale
    # Parseval against the real-space diagnostics of the same run
    assert got.sum() == pytest.approx(run.diagnostics()["emag"], rel=tol, abs=1e-300)
    run.close()


def test_spectrum_is_reproducible_and_leaves_the_run_unchanged():
    kw = dict(nx=24, ny=24, nz=24, nu=0.01, eta=0.01, f0=0.05, sigma=1.0, kmin=1.0, kmax=2.0, seed=3,
              dtype="f32")
    q0 = inputs.random_modes_state(24, 24, 24, seed=8, amp=0.2)
    a, b = make_run(**kw), make_run(**kw)
    a.set_state(q0)
    b.set_state(q0)
    for _ in range(3):
        a.step(2)
        b.step(2)
        s1, s2 = a.spectrum(), a.spectrum()
        assert np.array_equal(s1, s2)
    qa, ta, _ = a.get_state()
    qb, tb, _ = b.get_state()
    assert ta == tb and np.array_equal(qa, qb)
    assert np.array_equal(a.spectrum(), b.spectrum())
    a.close()
    b.close()


def test_channel_growth_rates_fp32_gpu_match_fp64_oracle():
    """Kinematic stage at 32^3 (helical forcing, seed field): lambda_k of the
    channels that hold most of the magnetic energy, FP32 GPU vs FP64 oracle
    over the same samples, within 1%."""
    from paper_2012_08758_b300.growth import channel_growth_rates, spectrum_series

    n, nsteps, every = 32, 160, 8
    kw = dict(nx=n, ny=n, nz=n, nu=5e-3, eta=5e-3, f0=0.02, sigma=1.0, kmin=2.5, kmax=3.5, seed=7,
              cfl=0.4)
    q0 = inputs.seed_field_state(n, seed=3, amp=1e-4)
    run = make_run(dtype="f32", **kw)
    run.set_state(q0)
    t_g, e_g = spectrum_series(run, nsteps, every)
    run.close()

    p = oracle_params(**kw)
    q = q0.copy()
    t_o, e_o = [0.0], [O.spectrum(p, q)]
    t = 0.0
    for k in range(0, nsteps, every):
        t, _ = O.run(p, q, every, step0=k, t0=t)
        t_o.append(t)
        e_o.append(O.spectrum(p, q))
    t_o, e_o = np.array(t_o), np.array(e_o)
    np.testing.assert_allclose(t_g, t_o, rtol=1e-5)
    # the channels that carry the energy at the end agree to FP32 rounding
    top = np.argsort(e_o[-1])[::-1][:6]
    np.testing.assert_allclose(e_g[:, top], e_o[:, top], rtol=1e-4)
    lam_g = channel_growth_rates(t_g, e_g, top)
    half = len(t_o) // 2
    for k in top:
        lam_o = 0.5 * O.growth_rate(t_o[half:], e_o[half:, k])
        assert abs(lam_g[k] - lam_o) <= 0.01 * abs(lam_o) + 1e-6, (k, lam_g[k], lam_o)


@pytest.mark.slow
def test_full_size_256_spectrum_matches_oracle():
    """The bench workload's grid (256^3, FP32): every shell against the FP64
    oracle's spectrum of the same state (the oracle's curl and numpy FFT take
    a few seconds), within 1e-5 of the total magnetic energy."""
    n = 256
    kw = dict(nx=n, ny=n, nz=n, dtype="f32")
    q = inputs.random_modes_state(n, n, n, seed=40, amp=0.2, kmax=8, nmodes=12) + \
        inputs.noise_state(n, n, n, seed=41, amp=1e-3)
    run = make_run(**kw)
    run.set_state(q)
    got = run.spectrum()
    run.close()
    want = O.spectrum(oracle_params(**kw), q)
    assert got.shape == want.shape == (223,)
    assert np.abs(got - want).max() <= 1e-5 * want.sum()
