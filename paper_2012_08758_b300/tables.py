"""Kinematic growth rates at the setup of the paper's Tables 1 and 2 (Sec. 4
and Sec. 5.1 "Growth rates"): periodic box of side 2 pi, c_s = 1, nu = eta,
forcing on the shell 4.5 <= |k| <= 5.5, weak delta-correlated seed field
(amplitude 1e-5), upwinding of the continuity equation, CFL 0.4.

All requested rows are stepped together as one FP32 batch until t = tmax,
with B_rms and u_rms sampled every `chunk` steps.  lambda = least-squares
slope of ln B_rms over t in [t_start, t_b], t_b the end of the run or the
first sample with B_rms > sat * u_rms (the field starts to act back on the
flow); Re_M = <u_rms> over that window / (eta k_f), k_f the mean |k| of the
shell.

The forcing scale f0 defaults to 0.029: with the paper's f0 = 0.08 and Eq. 5
as printed (dt the time step) the first row of Table 1 (64^3, eta = 5e-3,
helical) reaches u_rms ~ 0.25 (Re_M 9.9 against the printed 3.6), so f0 is
calibrated once on that row and held fixed for every other row; the forcing
formula itself (Eqs. 4-6) is unchanged."""
from __future__ import annotations

import math
import time

import numpy as np

from . import binding as B
from . import inputs
from .growth import growth_rate

SHELL = (4.5, 5.5)
F0_CALIBRATED = 0.029


def shell_mean_k(kmin: float = SHELL[0], kmax: float = SHELL[1]) -> float:
    K = int(math.floor(kmax))
    ks = [math.sqrt(a * a + b * b + c * c) for a in range(-K, K + 1) for b in range(-K, K + 1)
          for c in range(-K, K + 1) if kmin <= math.sqrt(a * a + b * b + c * c) <= kmax]
    return sum(ks) / len(ks)


def row_seed(index: int, realisation: int) -> int:
    """Forcing seed of a row: its index in the run list and its realisation."""
    return 1000 + index + 7919 * realisation


def run_rows(rows, f0: float = F0_CALIBRATED, tmax: float = 400.0, chunk: int = 200, upwind: int = 1,
             t_start: float = 100.0, sat: float = 0.1, spectra: bool = False, series: bool = False,
             device=None) -> dict:
    """rows: dicts with sigma, n, eta (and optionally lam, rem: the paper's
    values, copied into the result, and realisation).  Returns the per-row
    growth rates, Re_M, seeds and fit windows."""
    from .run import Batch, Run

    kf = shell_mean_k()
    runs, samples, specs, live = [], [], [], []
    for i, r in enumerate(rows):
        seed = row_seed(i, r.get("realisation", 0))
        run = Run(n=r["n"], nu=r["eta"], eta=r["eta"], f0=f0, kmin=SHELL[0], kmax=SHELL[1], sigma=r["sigma"],
                  seed=seed, upwind=upwind, cfl=0.4, device=device)
        run.set_state(inputs.seed_field_state(r["n"], seed=i, amp=1e-5))
        d = run.diagnostics()
        runs.append(run)
        samples.append([(0.0, d["brms"], d["urms"])])
        specs.append([run.spectrum()] if spectra else [])
        live.append(i)
    status = ["ok"] * len(rows)
    t0 = time.perf_counter()
    steps = 0
    batch = None
    while live:
        if batch is None:
            batch = Batch([runs[i] for i in live])
        batch.step(chunk)
        steps += chunk
        done = []
        for i in live:
            try:
                d = runs[i].diagnostics()
            except B.MhdError as e:
                status[i] = f"failed: {e}"
                done.append(i)
                continue
            t = runs[i].time()[0]
            samples[i].append((t, d["brms"], d["urms"]))
            if spectra:
                specs[i].append(runs[i].spectrum())
            if t >= tmax:
                done.append(i)
        if done:
            batch.close()
            batch = None
            live = [i for i in live if i not in done]
    wall = time.perf_counter() - t0
    out = []
    for i, r in enumerate(rows):
        runs[i].close()
        ts, bs, us = (np.array(c) for c in zip(*samples[i]))
        m = ts >= t_start
        hit = np.nonzero(m & (bs > sat * us))[0]
        if len(hit):
            m &= ts < ts[hit[0]]
        res = dict(sigma=r["sigma"], n=r["n"], eta=r["eta"], lambda_paper=r.get("lam"), rem_paper=r.get("rem"),
                   realisation=r.get("realisation", 0), seed=row_seed(i, r.get("realisation", 0)),
                   seed_field_seed=i, status=status[i], t_end=float(ts[-1]), samples=int(len(ts)))
        if series:
            res["series"] = {"t": ts.tolist(), "brms": bs.tolist(), "urms": us.tolist()}
        if status[i] == "ok" and m.sum() >= 3:
            res.update(lambda_=growth_rate(ts[m], bs[m]), rem=float(us[m].mean() / (r["eta"] * kf)),
                       window=[float(ts[m][0]), float(ts[m][-1])], window_samples=int(m.sum()))
            if spectra:
                E = np.array(specs[i])[m]
                res["lambda_k"] = {k: 0.5 * growth_rate(ts[m], E[:, k]) for k in (1, 5, 9) if k < E.shape[1]}
        out.append(res)
    return {"f0": f0, "k_f": kf, "shell": list(SHELL), "tmax": tmax, "chunk": chunk, "upwind": upwind,
            "t_start": t_start, "saturation_threshold": sat, "steps": steps, "wall_s": wall, "rows": out}
