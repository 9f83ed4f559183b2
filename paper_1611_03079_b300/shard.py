"""Host-side sharding of rendering work across ranks (one process per GPU).

Frames (and rows) are independent, so ranks exchange nothing on the data
path: each rank renders its own share, and only timings (max over ranks) and,
if wanted, results (gather to rank 0) cross process boundaries.  Works with
any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""


def frame_cost(f):
    """Work estimate of a frame: pixels x iteration limit (binary64 frames
    weighted by the measured ~74x narrower pipe)."""
    w = 74.0 if f.get("precision", 0) == 1 else 1.0
    return float(f["W"]) * float(f["H"]) * float(f["max_iter"]) * w


def shard_frames(frames, rank, world):
    """Indices of the frames assigned to `rank`: longest-processing-time
    greedy assignment (largest cost first to the least loaded rank), ties
    broken by rank, deterministic on every rank."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(frames)), key=lambda i: (-frame_cost(frames[i]), i))
    load = [0.0] * world
    owner = [0] * len(frames)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += frame_cost(frames[i])
    return [i for i in range(len(frames)) if owner[i] == rank]


def max_over_ranks(value, device=None):
    """The maximum of a float over all ranks (the job's step time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj):
    """Gather a picklable object from every rank; rank 0 gets the list, the
    others None."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
