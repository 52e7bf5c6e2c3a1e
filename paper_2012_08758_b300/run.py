"""Convenience wrappers over the C ABI: a ``Run`` owns one context whose
device workspace is a PyTorch CUDA tensor and whose stream is a PyTorch
stream; a ``Batch`` steps several runs together (one launch per kernel stage,
CUDA-graph replay)."""
from __future__ import annotations

import numpy as np

from . import binding as B


_STREAMS = {}


def default_stream(device):
    """One non-legacy PyTorch stream per device, shared by all runs on it
    (runs of a batch must share a stream; graph capture needs a non-legacy
    stream)."""
    import torch

    key = str(device)
    if key not in _STREAMS:
        _STREAMS[key] = torch.cuda.Stream(device=device)
    return _STREAMS[key]


class Run:
    """One simulation on one GPU.

    Keyword arguments are fields of ``mhd_params`` (nx, ny, nz, nu, eta, f0,
    sigma, seed, dtype, ...).  ``n`` sets nx = ny = nz."""

    def __init__(self, n: int | None = None, device=None, stream=None, **params):
        import torch

        if n is not None:
            params.setdefault("nx", n)
            params.setdefault("ny", n)
            params.setdefault("nz", n)
        self.params = B.mhd_default_params(**params)
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else default_stream(self.device)
        self.nbytes = B.mhd_workspace_bytes(self.params)
        # allocate on the run's stream so the caching allocator never hands
        # this block to another stream while the library still uses it
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            self._ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
            ptr = self._ws.data_ptr()
            ptr = (ptr + 255) // 256 * 256
            self.ctx = B.mhd_create(self.params, self.stream.cuda_stream, ptr, self.nbytes)

    @property
    def shape(self):
        p = self.params
        return (7, p.nz, p.ny, p.nx)

    @property
    def cells(self) -> int:
        p = self.params
        return p.nx * p.ny * p.nz

    def set_state(self, q: np.ndarray, t: float = 0.0, step: int = 0) -> None:
        assert q.shape == self.shape, (q.shape, self.shape)
        B.mhd_set_state(self.ctx, q, t, step)

    def params_dict(self) -> dict:
        return {name: getattr(self.params, name) for name, _ in self.params._fields_}

    def checkpoint(self, path: str) -> None:
        """Writes the state (in the working precision, so a restore is exact),
        t, the step index and the parameters to an .npz file.  The forcing's
        random numbers are counter-based (seed, step), so no generator state
        is needed: a restored run continues bit for bit."""
        wp = np.float32 if self.params.dtype == B.MHD_F32 else np.float64
        q, t, step = self.get_state(dtype=wp)
        kinds = dict(B.MhdParams._fields_)
        params = {}
        for name, value in self.params_dict().items():
            dt = np.uint64 if kinds[name] is B.C.c_uint64 else (np.int64 if kinds[name] is B.C.c_int else np.float64)
            params["param_" + name] = np.asarray(value, dtype=dt)
        np.savez(path, q=q, t=np.float64(t), step=np.int64(step), **params)

    @classmethod
    def restore(cls, path: str, device=None, stream=None) -> "Run":
        """A new Run with the parameters, state, t and step of a checkpoint."""
        d = np.load(path)
        p = {key[len("param_"):]: d[key].item() for key in d.files if key.startswith("param_")}
        r = cls(device=device, stream=stream, **p)
        r.set_state(d["q"], float(d["t"]), int(d["step"]))
        return r

    def set_seed_field(self, seed: int, amp: float = 1e-5) -> None:
        """ln rho = 0, u = 0, A = amp * N(0,1) per point, generated on the device."""
        B.mhd_set_seed_field(self.ctx, seed, amp)

    def get_state(self, dtype=np.float64):
        return B.mhd_get_state(self.ctx, shape=self.shape, dtype=dtype)

    def step(self, n: int = 1) -> None:
        B.mhd_step(self.ctx, n)

    def diagnostics(self) -> dict:
        return B.mhd_diagnostics(self.ctx)

    def spectrum(self) -> np.ndarray:
        """Magnetic energy spectrum E_B(m) of the current state (cubic box)."""
        return B.mhd_spectrum(self.ctx, B.mhd_spectrum_shells(self.params))

    def reduce(self, kind: int) -> float:
        return B.mhd_reduce(self.ctx, kind)

    def time(self):
        return B.mhd_time(self.ctx)

    def sync(self) -> None:
        B.mhd_sync(self.ctx)

    def forcing_draw(self, step: int) -> dict:
        return B.mhd_forcing_draw(self.ctx, step)

    def eval_rhs(self, step: int = 0, dt_forcing: float = 0.0, dtype=np.float64):
        return B.mhd_eval_rhs(self.ctx, self.shape, step, dt_forcing, dtype)

    def eval_rhs_at(self, points, step: int = 0, dt_forcing: float = 0.0) -> np.ndarray:
        """dq/dt at the listed (i, j, k) points only: array (len(points), 7)."""
        return B.mhd_eval_rhs_at(self.ctx, points, step, dt_forcing)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            B.mhd_destroy(self.ctx)
            self.ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent runs stepped together; each run's result is the one it
    gives alone."""

    def __init__(self, runs):
        self.runs = list(runs)
        self.handle = B.mhd_batch_create([r.ctx for r in self.runs])

    def step(self, n: int = 1) -> None:
        B.mhd_batch_step(self.handle, n)

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.mhd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
