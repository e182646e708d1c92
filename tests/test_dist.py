"""Multi-rank host logic on CPU with gloo, world size 2: sharding of
independent systems, the max-over-ranks step time, and a lost rank detected
by a short collective timeout (host-side fault injection; no GPU)."""
import multiprocessing as mp
import os
import socket

import pytest

from paper_2108_01186_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import torch.distributed as dist
        timeout = 5 if mode == "lost" else 60
        D.init("gloo", timeout_s=timeout)
        if mode == "ok":
            units = D.shard(64, rank, world)
            t = D.max_over_ranks(10.0 + rank)
            D.barrier()
            q.put((rank, units, t))
        else:
            if rank == 1:
                q.put((rank, "left", None))
                q.close()
                q.join_thread()        # the message is out before the process dies
                os._exit(0)            # leaves between steps, nothing in flight
            try:
                D.max_over_ranks(1.0)
                q.put((rank, "no error", None))
            except Exception as e:     # the collective ends with an error
                q.put((rank, "error", type(e).__name__))
        dist.destroy_process_group() if dist.is_initialized() and mode == "ok" else None
    except Exception as e:
        q.put((rank, "exception", repr(e)))


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda x: x[0])


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            got = [u for r in range(world) for u in D.shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(D.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def test_two_gloo_ranks_shard_and_max_time():
    out = _run("ok")
    assert out[0][1] + out[1][1] == list(range(64))
    assert out[0][2] == 11.0 and out[1][2] == 11.0


def test_lost_rank_is_detected_by_collective_timeout():
    out = _run("lost")
    assert out[1][1] == "left"
    assert out[0][1] == "error"
