"""The z-slab decomposition's host logic on CPU: the exchange plan against
brute force, and the halo exchange between processes (gloo, one slab per
rank) -- ghost planes equal to the periodic neighbours' planes of the whole
grid, the time step's all-reduce, and a rank that leaves between steps being
reported by the heartbeat to the others before their next exchange."""
import datetime
import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2012_08758_b300.slabs import RAD, exchange_plan, slab_extents


@pytest.mark.parametrize("nz,ns", [(12, 1), (12, 2), (13, 3), (40, 4), (9, 3)])
def test_extents_cover_the_grid(nz, ns):
    ext = slab_extents(nz, ns)
    assert [z for z, _ in ext] == list(np.cumsum([0] + [n for _, n in ext])[:-1])
    assert sum(n for _, n in ext) == nz and min(n for _, n in ext) >= RAD
    assert max(n for _, n in ext) - min(n for _, n in ext) <= 1


def test_too_thin_slabs_are_rejected():
    with pytest.raises(ValueError):
        slab_extents(8, 3)


@pytest.mark.parametrize("nz,ns", [(12, 1), (13, 2), (40, 4), (9, 3)])
def test_plan_fills_every_ghost_plane_with_its_periodic_source(nz, ns):
    """Brute force: ghost plane g of slab k (global plane z0_k + g, wrapped)
    must receive that global plane, from whichever slab holds it."""
    ext = slab_extents(nz, ns)
    owner = {}
    for k, (z0, n) in enumerate(ext):
        for i in range(n):
            owner[z0 + i] = (k, i)
    got = {}
    for t in exchange_plan(nz, ns):
        for d in range(RAD):
            key = (t.dst, t.dst_lo + d)
            assert key not in got, "ghost plane filled twice"
            got[key] = (t.src, t.src_lo + d)
    for k, (z0, n) in enumerate(ext):
        for g in list(range(-RAD, 0)) + list(range(n, n + RAD)):
            assert got[(k, g)] == owner[(z0 + g) % nz], (k, g)
    assert len(got) == 2 * RAD * ns


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, nz, leave_rank):
    import torch
    import torch.distributed as dist

    from paper_2012_08758_b300.slabs import DistSlabExchange, SlabPeerLost
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    store = dist.TCPStore("127.0.0.1", port + 1, world, rank == 0, timeout=datetime.timedelta(seconds=20))
    dist.init_process_group("gloo", store=dist.PrefixStore("pg", store), rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    try:
        rng = np.random.default_rng(5)
        glob = rng.standard_normal((7, nz, 4, 5))  # the same whole grid on every rank
        z0, n = slab_extents(nz, world)[rank]
        slab = torch.zeros((7, n + 2 * RAD, 4, 5), dtype=torch.float64)
        slab[:, RAD:RAD + n] = torch.from_numpy(glob[:, z0:z0 + n])
        ex = DistSlabExchange(store=store, heartbeat_timeout=2.0)
        ex.exchange(0, slab)
        want = glob[:, [(z0 + g) % nz for g in range(-RAD, n + RAD)]]
        ok = bool(np.array_equal(slab.numpy(), want))
        dt = ex.dt_min(0.01 * (rank + 1))
        if rank == leave_rank:  # leaves between steps: never joins exchange 1
            q.put((rank, "left", ok, dt))
            return
        t0 = time.perf_counter()
        try:
            slab[:, RAD:RAD + n] += 1.0
            ex.exchange(1, slab)
            want = want + 1.0
            q.put((rank, "ok", ok and bool(np.array_equal(slab.numpy(), want)), dt))
        except SlabPeerLost as e:
            q.put((rank, "peer_lost", ok, time.perf_counter() - t0, str(e)))
    except Exception as e:
        q.put((rank, "error", type(e).__name__, str(e)[:200]))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, nz, leave_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, nz, leave_rank)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return {o[0]: o for o in out}


@pytest.mark.parametrize("world,nz", [(2, 11), (3, 12)])
def test_exchange_fills_ghosts_across_ranks(world, nz):
    out = _run(world, nz)
    for r in range(world):
        assert out[r][1] == "ok" and out[r][2] is True, out[r]
        assert out[r][3] == pytest.approx(0.01)  # min over the ranks' dt


def test_rank_leaving_between_steps_is_detected_before_the_next_exchange():
    out = _run(2, 10, leave_rank=1)
    assert out[1][1] == "left" and out[1][2] is True
    assert out[0][1] == "peer_lost", out[0]
    assert out[0][2] is True and out[0][3] < 10.0  # the heartbeat, not a hang
    assert "rank 1" in out[0][4]
