"""Serving loop for dynamo-run requests with continuous batching.

A request asks for a forced run (grid N^3, magnetic Reynolds number Re_M at
magnetic Prandtl number 1, forcing helicity sigma, a step budget).  The
server admits queued requests in arrival order while their device footprint
fits the HBM budget and a slot is free, keeps every admitted run's state on
the device, and steps all admitted runs together (one launch per kernel stage
over the combined tile table, replayed from a CUDA graph) in chunks; after
each chunk it samples B_rms of every run, retires runs whose budget is spent
(result: growth rate of ln B_rms, final diagnostics, latency) and admits
runs that arrived meanwhile.  A run's result does not depend on what it was
batched with.  A run that blows up (non-finite time step: the paper's
under-resolved runs "crash early") or is cancelled is retired with that
status at the next chunk boundary and frees its slot; the others go on.

Physics parameters (Sec. 4): L = 2 pi, c_s = 1, f0 = 0.02, forcing shell
2.5 <= |k| <= 3.5 (k_f = 3.13), nu = eta = u_rms0 / (Re_M k_f) with u_rms0 the
calibrated rms velocity of the forced flow (Eq. 7)."""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import binding as B
from . import inputs
from .growth import fit_last

KF = 3.134  # mean |k| of the integer shell 2.5 <= |k| <= 3.5 (98 vectors)


@dataclass
class Request:
    id: int
    arrival: float      # seconds after the start of serving
    n: int
    re_m: float
    sigma: float
    steps: int
    seed: int


@dataclass
class Result:
    id: int
    n: int
    steps: int
    arrival: float
    admitted: float
    finished: float
    growth_rate: float
    diagnostics: dict
    t: list = field(repr=False, default_factory=list)
    brms: list = field(repr=False, default_factory=list)
    status: str = "ok"

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def run_params(req: Request, urms0: float = 0.05, dtype=B.MHD_F32, **extra) -> dict:
    nu = urms0 / (req.re_m * KF)
    p = dict(nx=req.n, ny=req.n, nz=req.n, nu=nu, eta=nu, f0=0.02, kmin=2.5, kmax=3.5,
             sigma=req.sigma, seed=req.seed, dtype=dtype, cfl=0.4)
    p.update(extra)
    return p


SEED_FIELD_AMP = 1e-5
SEED_FIELD_KEY = 1 << 32  # offset of the seed-field stream from the forcing stream


def seed_field_key(req: Request) -> int:
    return req.seed + SEED_FIELD_KEY


def initial_state(req: Request) -> np.ndarray:
    """Uniform density, no flow, weak delta-correlated seed field (Sec. 4):
    the host copy of what start() generates on the device."""
    return inputs.counter_seed_field_state(req.n, seed=seed_field_key(req), amp=SEED_FIELD_AMP)


def start(run, req: Request) -> None:
    """Puts a run into its request's initial state, generated on the device
    (no host arrays, no upload)."""
    run.set_seed_field(seed_field_key(req), SEED_FIELD_AMP)


class Server:
    def __init__(self, device=None, budget_bytes: float = 150e9, max_active: int = 64,
                 chunk: int = 50, urms0: float = 0.05, dtype=B.MHD_F32, kernel: int = 0, tile: int = 0,
                 time_scale: float = 1.0, window: float = 0.5, run_factory=None, batch_factory=None):
        self.device = device
        self.budget = budget_bytes
        self.max_active = max_active
        self.chunk = chunk
        self.urms0 = urms0
        self.dtype = dtype
        self.kernel, self.tile = kernel, tile
        self.time_scale = time_scale  # wall seconds per unit of request arrival time
        self.window = window          # fit ln B_rms over the last `window` fraction of the run
        self.used = 0.0
        self.active = []              # [Run, Request, remaining, admitted, ts, bs, nbytes]
        self.results: list[Result] = []
        self.stepped_cells = 0
        self.cancelled: set[int] = set()
        # constructors of runs and batches (the GPU Run and Batch unless given)
        self._run_factory = run_factory
        self._batch_factory = batch_factory

    def cancel(self, request_id: int) -> None:
        """Drops a queued request, or retires an active one at the next chunk
        boundary with status "cancelled"."""
        self.cancelled.add(request_id)

    def _make_run(self, **params):
        if self._run_factory is not None:
            return self._run_factory(**params)
        from .run import Run
        return Run(device=self.device, **params)

    def _make_batch(self, runs):
        if self._batch_factory is not None:
            return self._batch_factory(runs)
        from .run import Batch
        return Batch(runs)

    def footprint(self, req: Request) -> int:
        p = B.mhd_default_params(**run_params(req, self.urms0, self.dtype, kernel=self.kernel,
                                              tile=self.tile))
        return B.mhd_workspace_bytes(p) + 256

    def _admit(self, req: Request, now: float) -> None:
        nbytes = self.footprint(req)
        run = self._make_run(**run_params(req, self.urms0, self.dtype, kernel=self.kernel, tile=self.tile))
        start(run, req)
        b0 = run.reduce(B.MHD_BRMS)
        self.active.append([run, req, req.steps, now, [0.0], [b0], nbytes])
        self.used += nbytes

    def _retire(self, entry, now: float, status: str = "ok") -> None:
        run, req, _, admitted, ts, bs, nbytes = entry
        diag = run.diagnostics() if status == "ok" else {}
        lam = fit_last(ts, bs, self.window) if status == "ok" and len(ts) > 2 else float("nan")
        self.results.append(Result(req.id, req.n, req.steps, req.arrival, admitted, now, lam, diag,
                                   list(ts), list(bs), status))
        run.close()
        self.used -= nbytes

    def serve(self, requests, realtime: bool = True) -> list[Result]:
        """Serves all requests; arrival times are honoured in wall time (scaled
        by time_scale) when realtime is True, otherwise all arrive at once."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        batch, batch_ids = None, None
        while pending or queue or self.active:
            tn = now()
            while pending and (not realtime or pending[0].arrival * self.time_scale <= tn):
                r = pending.pop(0)
                queue.append(r)
            if self.cancelled:
                queue = [r for r in queue if r.id not in self.cancelled]
                pending = [r for r in pending if r.id not in self.cancelled]
            while queue and len(self.active) < self.max_active:
                need = self.footprint(queue[0])
                if self.used + need > self.budget and self.active:
                    break
                if need > self.budget:
                    raise MemoryError(f"request {queue[0].id} needs {need} B, above the budget")
                self._admit(queue.pop(0), now())
            if not self.active:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival * self.time_scale - now()))
                continue
            ids = [id(e[0]) for e in self.active]
            if ids != batch_ids:
                if batch is not None:
                    batch.close()
                batch = self._make_batch([e[0] for e in self.active])
                batch_ids = ids
            k = min(self.chunk, min(e[2] for e in self.active))
            batch.step(k)
            ended = []
            for e in self.active:
                e[2] -= k
                self.stepped_cells += k * e[0].cells
                try:
                    tt, _, _ = e[0].time()
                    b = e[0].reduce(B.MHD_BRMS)
                except B.MhdError as err:  # blew up: retire it, keep the others
                    ended.append((e, f"failed: {err}"))
                    continue
                e[4].append(tt)
                e[5].append(b)
                if e[1].id in self.cancelled:
                    ended.append((e, "cancelled"))
                elif e[2] == 0:
                    ended.append((e, "ok"))
            if ended:
                tn = now()
                for e, status in ended:
                    self.active.remove(e)
                    self._retire(e, tn, status)
        if batch is not None:
            batch.close()
        return self.results


def summarize(results, wall: float, stepped_cells: int) -> dict:
    lat = np.array([r.latency for r in results])
    return {
        "requests": len(results),
        "failed": sum(1 for r in results if r.status != "ok"),
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "cell_updates_per_s": stepped_cells / wall,
        "wall_s": wall,
    }


def requests_from_inputs(n: int = 200, seed: int = 2025, rate: float = 1.0, **kw) -> list[Request]:
    return [Request(r["id"], r["arrival"], r["n"], r["re_m"], r["sigma"], r["steps"], r["seed"])
            for r in inputs.serving_requests(n=n, seed=seed, rate=rate, **kw)]
