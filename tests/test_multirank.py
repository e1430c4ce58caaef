"""The N>1 host logic of bench.py with world-size-2 gloo ranks on CPU.

Frames shard across ranks with no data-path collective (weak scaling); the only
collectives are the barrier and the max/sum reductions of the timing, tested here.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    frames = bench.frames_for_rank(r, w, 240, 240)
    bench.barrier(w)
    mx = bench.reduce_max(float(10 + rank), w)
    sm = bench.reduce_sum(float(len(frames)), w)
    q.put((rank, frames, mx, sm, (r, w, lr)))
    dist.destroy_process_group()


def test_frames_shard_without_overlap_and_timing_reduces():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    f0, f1 = out[0][1], out[1][1]
    assert not set(f0[:120]) & set(f1[:120])              # disjoint frames per rank
    assert sorted(set(f0) | set(f1)) == list(range(240))  # together they cover the trajectory
    assert all(o[2] == 11.0 for o in out)                  # max over ranks
    assert all(o[3] == 480.0 for o in out)                 # total frames of the job
    assert out[1][4] == (1, 2, 1)


def test_single_rank_defaults():
    assert bench.frames_for_rank(0, 1, 5, 240) == [0, 48, 96, 144, 192]   # spread evenly
    assert bench.frames_for_rank(0, 1, 240, 240) == list(range(240))
    assert bench.frames_for_rank(0, 1, 300, 240)[238:242] == [238, 239, 0, 1]
    assert bench.frames_for_rank(1, 2, 4, 240) == [30, 90, 150, 210]
    assert bench.reduce_max(3.0, 1) == 3.0
    a = bench.parse_args([])
    assert a.gpus == 1 and a.steps > 0 and a.warmup >= 3
