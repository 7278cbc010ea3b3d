"""Coordination of independent replicas, one process per GPU.

The streaming checksum does not shard into an exchange: every rank streams its
own buffer on its own GPU and the per-rank results are independent problems
(weak scaling).  torch.distributed is used only around the timed region:

- rank 0 chooses the measured point and every rank runs it (broadcast);
- a barrier brackets the timed steps on every rank (the caller's);
- the timed interval of the job is the maximum over ranks (all-reduce MAX);
- every rank's result triple is gathered so rank 0 can check that ranks which
  read identical buffers agree (all-gather of a few integers).

These helpers take the process-group module and the tensor device explicitly
so that the same code runs over NCCL (CUDA tensors) and gloo (CPU tensors).
"""
from __future__ import annotations


def broadcast_choice(index: int, dist=None) -> int:
    """Rank 0's choice on every rank."""
    if dist is None:
        return int(index)
    box = [int(index)]
    dist.broadcast_object_list(box, src=0)
    return int(box[0])


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The maximum of `value` over all ranks (the job's timed interval)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(sum_u32: int, xor_u64: int, issued: int, dist=None, device="cpu") -> list[tuple[int, int, int]]:
    """Every rank's (sum_u32, xor_u64, issued_loads), in rank order, on every
    rank.  The 64-bit XOR travels as two 32-bit halves (int64 tensors hold
    them without sign trouble)."""
    own = (int(sum_u32), int(xor_u64), int(issued))
    if dist is None:
        return [own]
    import torch
    words = [own[0], own[1] & 0xFFFFFFFF, own[1] >> 32, own[2]]
    t = torch.tensor(words, dtype=torch.int64, device=device)
    out = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    res = []
    for o in out:
        w = [int(v) for v in o.cpu().tolist()]
        res.append((w[0], w[1] | (w[2] << 32), w[3]))
    return res


def job_gbs(bytes_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the bytes every rank streamed over all timed
    steps, divided by the slowest rank's interval (decimal GB/s)."""
    if max_ms <= 0:
        raise ValueError("timed interval must be positive")
    return world * bytes_per_rank * steps / (max_ms * 1e6)
