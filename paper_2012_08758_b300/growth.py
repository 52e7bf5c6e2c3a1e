"""Growth rate of the magnetic field (Sec. 4, after Eq. 7): B_rms ~ exp(lambda t)
during the kinematic stage; lambda is the least-squares slope of ln B_rms
against t over a fixed window, computed on the host in FP64.  The growth
rates lambda_k of single spectral channels (Sec. 5) follow from the
magnetic spectrum the same way."""
from __future__ import annotations

import numpy as np

from . import binding as B


def growth_rate(t, brms, window=None) -> float:
    """Slope of ln(brms) versus t by linear least squares (FP64).

    window: (t_a, t_b) to restrict the fit, or None for all samples.  To
    compare two runs, fit the same samples of each (e.g. via fit_last);
    an absolute time window can take a boundary sample in one run and not in
    the other when their times differ by rounding."""
    t = np.asarray(t, dtype=np.float64)
    y = np.log(np.asarray(brms, dtype=np.float64))
    if window is not None:
        m = (t >= window[0]) & (t <= window[1])
        t, y = t[m], y[m]
    if t.size < 2:
        raise ValueError("need at least two samples in the window")
    A = np.stack([t, np.ones_like(t)], axis=1)
    slope, _ = np.linalg.lstsq(A, y, rcond=None)[0]
    return float(slope)


def fit_last(t, brms, fraction: float = 0.5) -> float:
    """Growth rate over the last `fraction` of the samples."""
    t = np.asarray(t)
    k = int(len(t) * (1.0 - fraction))
    return growth_rate(t[k:], np.asarray(brms)[k:])


def channel_growth_rates(t, spectra, channels, fraction: float = 0.5) -> dict:
    """Growth rates lambda_k of spectral channels (Sec. 5, power spectra):
    during the kinematic stage E_B(k) ~ exp(2 lambda_k t), so lambda_k is half
    the least-squares slope of ln E_B(k) against t over the last `fraction`
    of the samples, in the units of the B_rms growth rate.
    spectra: one E_B array per sample time (shells 0, 1, ...)."""
    t = np.asarray(t, dtype=np.float64)
    S = np.asarray(spectra, dtype=np.float64)
    k0 = int(len(t) * (1.0 - fraction))
    return {int(k): 0.5 * growth_rate(t[k0:], S[k0:, k]) for k in channels}


def spectrum_series(run, nsteps: int, every: int = 1):
    """Steps `run` nsteps times, taking (t, E_B) every `every` steps (and at
    the start).  Returns the times and a (samples, shells) array."""
    ts, es = [run.time()[0]], [run.spectrum()]
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        run.step(k)
        done += k
        ts.append(run.time()[0])
        es.append(run.spectrum())
    return np.array(ts), np.array(es)


def brms_series(run, nsteps: int, every: int = 1):
    """Steps `run` (a Run) nsteps times, sampling (t, B_rms) every `every`
    steps (and at the start).  Returns two numpy arrays."""
    ts, bs = [], []
    t, _, _ = run.time()
    ts.append(t)
    bs.append(run.reduce(B.MHD_BRMS))
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        run.step(k)
        done += k
        t, _, _ = run.time()
        ts.append(t)
        bs.append(run.reduce(B.MHD_BRMS))
    return np.array(ts), np.array(bs)
