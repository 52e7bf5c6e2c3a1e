"""Host logic of the multi-GPU replica path, run as world-size-2 gloo process
groups on CPU: max of the per-rank timings, whole-job throughput, distinct
replica seeds, and a rank that fails before the timing collective being
reported to the other rank by a short process-group timeout (no GPU)."""
import datetime
import os
import socket

import pytest
import torch.multiprocessing as mp


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, fail_rank):
    import torch.distributed as dist

    from paper_2012_08758_b300 import replicas as RP
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    try:
        assert RP.env() == (world, rank, rank)
        RP.barrier()
        if rank == fail_rank:
            raise RuntimeError("replica blew up")
        t = RP.max_over_ranks(1.0 + rank)
        q.put((rank, "ok", t, RP.job_throughput(world, 100.0, t), RP.replica_seed(7, rank)))
    except Exception as e:  # reported to the parent
        q.put((rank, "error", type(e).__name__, str(e)[:80], None))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return sorted(out)


def test_max_over_ranks_and_job_throughput():
    out = _run(2)
    assert [o[1] for o in out] == ["ok", "ok"]
    assert all(o[2] == 2.0 for o in out)            # max of 1.0 and 2.0
    assert all(o[3] == 2 * 100.0 / 2.0 for o in out)
    assert out[0][4] != out[1][4]                     # distinct replica seeds


def test_failed_rank_is_detected_by_the_others():
    out = _run(2, fail_rank=1)
    status = {o[0]: o for o in out}
    assert status[1][1] == "error" and "blew up" in status[1][3]
    assert status[0][1] == "error"  # the collective gives up instead of hanging
