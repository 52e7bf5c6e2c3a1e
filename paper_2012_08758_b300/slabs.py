"""z-slab domain decomposition (Sec. 3.3 "Domain decomposition" and 3.4
"Functions and data dependencies" of the paper).

The grid is cut along z into slabs; every substep, each slab needs the three
planes (the stencil radius) nearest each of its z faces from the neighbouring
slab across that face, and the time step is the minimum over all slabs.

* ``slab_extents`` / ``exchange_plan``: which planes each slab holds and
  which planes travel where at every exchange (the same rule as the C
  library's ``mhd_slabs_*``).
* ``Slabs``: a decomposed run on one GPU through the C ABI (``mhd_slabs_*``):
  one context per slab, the exchange as device copies overlapped with the
  inner planes' computation.
* ``DistSlabExchange``: the same exchange between processes, one slab per
  rank, over ``torch.distributed`` point-to-point messages, with a host-side
  heartbeat so that a rank that left between steps is detected before the
  next exchange instead of hanging it.
"""
from __future__ import annotations

import datetime
from dataclasses import dataclass

import numpy as np

from . import binding as B

RAD = 3  # stencil radius of the 6th-order scheme: planes exchanged per face


def slab_extents(nz: int, nslabs: int) -> list[tuple[int, int]]:
    """(first global plane, plane count) of each slab: nz // nslabs planes,
    the first nz % nslabs slabs one more.  Each slab needs >= RAD planes."""
    if nslabs < 1 or nz < RAD * nslabs:
        raise ValueError(f"{nz} planes cannot give {nslabs} slabs of at least {RAD}")
    out, z = [], 0
    for k in range(nslabs):
        n = nz // nslabs + (1 if k < nz % nslabs else 0)
        out.append((z, n))
        z += n
    return out


@dataclass(frozen=True)
class Transfer:
    """Planes [src_lo, src_lo + RAD) of slab src (interior indices) go to
    ghost planes [dst_lo, dst_lo + RAD) of slab dst (ghost indices: -RAD..-1
    below the slab, n..n+RAD-1 above it)."""
    src: int
    src_lo: int
    dst: int
    dst_lo: int


def exchange_plan(nz: int, nslabs: int) -> list[Transfer]:
    """The transfers of one exchange (periodic in the slab index): slab k's
    top RAD planes fill the bottom ghosts of slab k+1, and slab k+1's bottom
    RAD planes fill the top ghosts of slab k."""
    ext = slab_extents(nz, nslabs)
    plan = []
    for k in range(nslabs):
        up = (k + 1) % nslabs
        nk = ext[k][1]
        plan.append(Transfer(k, nk - RAD, up, -RAD))
        plan.append(Transfer(up, 0, k, nk))
    return plan


class Slabs:
    """A run decomposed into z-slabs on one GPU (C ABI ``mhd_slabs_*``).
    Keyword arguments are ``mhd_params`` fields; ``overlap`` runs the
    exchange on a second stream while the inner planes are computed."""

    def __init__(self, nslabs: int, n: int | None = None, overlap: bool = True, stream=None, **params):
        if n is not None:
            params.setdefault("nx", n)
            params.setdefault("ny", n)
            params.setdefault("nz", n)
        self.params = B.mhd_default_params(**params)
        self.nslabs = nslabs
        self.stream = stream
        self.handle = B.mhd_slabs_create(self.params, nslabs, 1 if overlap else 0,
                                         stream.cuda_stream if stream is not None else 0)

    @property
    def shape(self):
        p = self.params
        return (7, p.nz, p.ny, p.nx)

    def extents(self):
        return [B.mhd_slabs_extent(self.handle, k) for k in range(self.nslabs)]

    def set_state(self, q: np.ndarray, t: float = 0.0, step: int = 0) -> None:
        B.mhd_slabs_set_state(self.handle, q, t, step)

    def get_state(self, dtype=np.float64):
        return B.mhd_slabs_get_state(self.handle, self.shape, dtype)

    def step(self, n: int = 1) -> None:
        B.mhd_slabs_step(self.handle, n)

    def diagnostics(self) -> dict:
        return B.mhd_slabs_diagnostics(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            B.mhd_slabs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SlabPeerLost(RuntimeError):
    """A neighbouring rank did not reach the exchange (it left or died)."""


class DistSlabExchange:
    """Halo exchange of one slab per rank over torch.distributed.

    The slab is a tensor of shape (F, n + 2 RAD, ...) whose first RAD and
    last RAD planes along dim 1 are ghosts.  ``exchange(step, slab)`` sends
    the slab's RAD interior planes nearest each face to the neighbour across
    it and receives that neighbour's planes into the ghosts (ring of ranks,
    periodic).  Before exchanging, each rank posts a heartbeat for this
    exchange in the process group's store and waits (at most
    ``heartbeat_timeout`` seconds) for its neighbours' heartbeats; a missing
    one raises SlabPeerLost, so a rank that left between steps is found on the
    host before any message of the next exchange is posted.
    ``dt_min(local_dt)`` is the time step's all-reduce (the minimum over all
    slabs; the CFL maxima's maximum)."""

    def __init__(self, store=None, heartbeat_timeout: float = 2.0, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.store = store
        self.timeout = datetime.timedelta(seconds=heartbeat_timeout)
        self.up = (self.rank + 1) % self.world
        self.down = (self.rank - 1) % self.world

    def _heartbeat(self, tag: str) -> None:
        if self.store is None or self.world == 1:
            return
        self.store.set(f"slab/{tag}/{self.rank}", "1")
        for peer in {self.up, self.down}:
            try:
                self.store.wait([f"slab/{tag}/{peer}"], self.timeout)
            except Exception as e:  # the store's timeout: the peer never arrived
                raise SlabPeerLost(f"rank {peer} did not reach exchange {tag} (rank {self.rank})") from e

    def exchange(self, tag, slab) -> None:
        import torch

        self._heartbeat(str(tag))
        n = slab.shape[1] - 2 * RAD
        if self.world == 1:  # periodic wrap onto itself
            slab[:, :RAD] = slab[:, n:n + RAD]
            slab[:, n + RAD:] = slab[:, RAD:2 * RAD]
            return
        top = slab[:, n:n + RAD].contiguous()            # interior planes n-RAD .. n-1
        bottom = slab[:, RAD:2 * RAD].contiguous()       # interior planes 0 .. RAD-1
        from_down = torch.empty_like(top)                # -> ghost planes -RAD .. -1
        from_up = torch.empty_like(bottom)               # -> ghost planes n .. n+RAD-1
        P2P = self.dist.P2POp
        ops = [P2P(self.dist.isend, top, self.up, self.group, 1),
               P2P(self.dist.isend, bottom, self.down, self.group, 2),
               P2P(self.dist.irecv, from_down, self.down, self.group, 1),
               P2P(self.dist.irecv, from_up, self.up, self.group, 2)]
        for r in self.dist.batch_isend_irecv(ops):
            r.wait()
        slab[:, :RAD] = from_down
        slab[:, n + RAD:] = from_up

    def dt_min(self, local_dt: float) -> float:
        import torch

        t = torch.tensor([local_dt], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return float(t.item())
