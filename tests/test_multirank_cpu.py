"""The N > 1 host path on CPU: two gloo ranks shard the frames of a workload,
each renders its share with the CPU oracle (standing in for its GPU), the
results gathered on rank 0 equal the single-process render frame by frame,
and the step time is the maximum over ranks.  No GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1611_03079_b300 import shard, workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, frames, out_q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.shard_frames(frames, rank, world)
    res = {i: oracle.render(frames[i]["c"], frames[i]["rect"], frames[i]["W"], frames[i]["H"],
                            frames[i]["max_iter"], frames[i]["mode"], frames[i]["precision"], threads=1)
           for i in mine}
    t = shard.max_over_ranks(float(rank + 1))
    allres = shard.gather_to_rank0(res)
    if rank == 0:
        merged = {}
        for d in allres:
            merged.update(d)
        out_q.put((t, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_assignment_is_a_partition():
    frames = wl.path_animation(n=40, seed=3) + wl.throughput_sweep(64)
    for world in (1, 2, 3, 8):
        parts = [shard.shard_frames(frames, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(frames)))
        loads = [sum(shard.frame_cost(frames[i]) for i in p) for p in parts]
        if world > 1:
            assert max(loads) <= 2.0 * (sum(loads) / world) + max(shard.frame_cost(f) for f in frames)
    with pytest.raises(ValueError):
        shard.shard_frames(frames, 2, 2)


def test_two_gloo_ranks_match_single_process():
    frames = []
    for f in wl.random_views(6, seed=55):
        frames.append(f)
    for f in wl.throughput_sweep(48)[:4]:
        frames.append(f)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, frames, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, merged = q.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 2.0
    import oracle
    assert sorted(merged) == list(range(len(frames)))
    for i, f in enumerate(frames):
        ref = oracle.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], f["mode"], f["precision"])
        assert (merged[i] == ref).all()
