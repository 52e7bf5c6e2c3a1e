"""Kinematic-stage growth rate of ln B_rms: the FP32 GPU run against the FP64
oracle on the same seed and the same fit window must agree within 1%."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2012_08758_b300 import inputs
from tests.gpu_util import gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def test_growth_rate_fp32_gpu_matches_fp64_oracle():
    from paper_2012_08758_b300.growth import brms_series, growth_rate
    from paper_2012_08758_b300.run import Run

    n, nsteps, every = 32, 160, 8
    kw = dict(nx=n, ny=n, nz=n, nu=5e-3, eta=5e-3, f0=0.02, sigma=1.0, kmin=2.5, kmax=3.5, seed=7,
              cfl=0.4)
    q0 = inputs.seed_field_state(n, seed=3, amp=1e-4)
    run = Run(dtype=0, **gpu_params(**kw))
    run.set_state(q0)
    t_g, b_g = brms_series(run, nsteps, every)
    run.close()

    p = oracle_params(**kw)
    q = q0.copy()
    t_o, b_o = [0.0], [O.diagnostics(p, q)["brms"]]
    t = 0.0
    for k in range(0, nsteps, every):
        t, _ = O.run(p, q, every, step0=k, t0=t)
        t_o.append(t)
        b_o.append(O.diagnostics(p, q)["brms"])
    t_o, b_o = np.array(t_o), np.array(b_o)
    np.testing.assert_allclose(t_g, t_o, rtol=1e-5)
    np.testing.assert_allclose(b_g, b_o, rtol=1e-5)
    # fit window: the second half of each run's own samples (the same step
    # range on both sides; a window in absolute time would let rounding of
    # t move a boundary sample in or out)
    half = len(t_o) // 2
    lam_o = growth_rate(t_o[half:], b_o[half:])
    lam_g = growth_rate(t_g[half:], b_g[half:])
    assert abs(lam_g - lam_o) <= 0.01 * abs(lam_o), (lam_g, lam_o)
    # the fit itself against the oracle's library fit of the same samples
    assert abs(lam_o - O.growth_rate(t_o[half:], b_o[half:])) < 1e-12 * max(1.0, abs(lam_o))
