"""Tile-shape autotuner.

Every substep kernel variant (the TMA kernel's tile shapes and stage counts,
and the shared-memory plane-ring kernel) computes identical results; their
speed depends on the grid size, the dtype and, for a batch, the mix of runs.
The tuner times each candidate on the device with CUDA events around a few
steps of a scratch run (or of the whole batch) and keeps the fastest per key,
in memory and optionally in a JSON file.  Runtime autotuning of the problem
decomposition is the approach the paper's library takes (Sec. 3.2)."""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import binding as B
from . import inputs

# (kernel, tile) candidates per dtype
CANDIDATES = {
    B.MHD_F32: [(B.MHD_KERNEL_TMA, 1), (B.MHD_KERNEL_TMA, 2), (B.MHD_KERNEL_TMA, 3),
                (B.MHD_KERNEL_TMA, 4), (B.MHD_KERNEL_TMA, 5), (B.MHD_KERNEL_TMA, 6),
                (B.MHD_KERNEL_TMA, 7), (B.MHD_KERNEL_TMA, 8), (B.MHD_KERNEL_TMA, 9), (B.MHD_KERNEL_TMA, 10),
                (B.MHD_KERNEL_TMA, 11), (B.MHD_KERNEL_TMA, 12), (B.MHD_KERNEL_TMA, 13), (B.MHD_KERNEL_TMA, 14),
                (B.MHD_KERNEL_TMA, 15), (B.MHD_KERNEL_TMA, 16), (B.MHD_KERNEL_TMA, 17), (B.MHD_KERNEL_TMA, 18),
                (B.MHD_KERNEL_TMA, 19), (B.MHD_KERNEL_TMA, 20), (B.MHD_KERNEL_TMA, 21), (B.MHD_KERNEL_TMA, 22), (B.MHD_KERNEL_TMA, 23), (B.MHD_KERNEL_TMA, 24),
                (B.MHD_KERNEL_TMA, 25), (B.MHD_KERNEL_TMA, 26), (B.MHD_KERNEL_TMA, 27), (B.MHD_KERNEL_TMA, 28),
                (B.MHD_KERNEL_SMEM, 0)],
    B.MHD_F64: [(B.MHD_KERNEL_TMA, 1), (B.MHD_KERNEL_TMA, 2), (B.MHD_KERNEL_TMA, 3), (B.MHD_KERNEL_TMA, 4),
                (B.MHD_KERNEL_SMEM, 0)],
}

_lock = threading.Lock()
_cache: dict[str, dict] = {}


def _key(shapes, dtype) -> str:
    return f"{int(dtype)}:" + ",".join(f"{a}x{b}x{c}" for a, b, c in sorted(shapes))


def load_cache(path: str) -> None:
    if os.path.exists(path):
        with open(path) as f:
            with _lock:
                _cache.update(json.load(f))


def save_cache(path: str) -> None:
    with _lock:
        data = dict(_cache)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_runs(runs, steps: int) -> float:
    """Milliseconds per step of the given runs stepped together."""
    import torch

    from .run import Batch

    stream = runs[0].stream
    b = Batch(runs) if len(runs) > 1 else None
    step = (lambda k: b.step(k)) if b else (lambda k: runs[0].step(k))
    step(2)  # warm-up (also captures the batch graph)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(steps)
    e1.record(stream)
    e1.synchronize()
    for r in runs:
        r.sync()
    if b:
        b.close()
    return e0.elapsed_time(e1) / steps


def tune(shapes, dtype=B.MHD_F32, steps: int = 4, device=None, params=None) -> dict:
    """Best (kernel, tile) for runs of the given grid shapes stepped together
    (one shape: a single run).  Returns {'kernel', 'tile', 'ms': {...}}."""
    from .run import Run

    shapes = [tuple(int(v) for v in s) for s in shapes]
    key = _key(shapes, dtype)
    with _lock:
        if key in _cache:
            return _cache[key]
    params = dict(params or {})
    timings = {}
    for kernel, tile in CANDIDATES[int(dtype)]:
        runs = []
        try:
            for i, (nx, ny, nz) in enumerate(shapes):
                r = Run(nx=nx, ny=ny, nz=nz, dtype=dtype, kernel=kernel, tile=tile, device=device,
                        seed=1 + i, **params)
                r.set_state(inputs.noise_state(nx, ny, nz, seed=i, amp=1e-3))
                runs.append(r)
            timings[f"{kernel}:{tile}"] = _time_runs(runs, steps)
        except B.MhdError:
            continue
        finally:
            for r in runs:
                r.close()
    best = min(timings, key=timings.get)
    k, t = (int(v) for v in best.split(":"))
    res = {"kernel": k, "tile": t, "ms": timings}
    with _lock:
        _cache[key] = res
    return res
