"""Sharding one camera's fingerprint across ranks (one process per GPU).

The MLE sums of Sec. III-A / III-B, num = sum_i W_i I_i and den = sum_i I_i^2,
run over independent SDA groups, so ranks can take disjoint, contiguous runs
of whole groups and one sum all-reduce of num/den (2 * 4 B per pixel-channel)
completes the fingerprint.  Group boundaries stay at multiples of d, so every
rank sees the same groups a single process would (the ragged last group, if
any, goes to the last rank that has groups).

Independent cameras need no exchange at all (weak scaling); this module is for
one camera spread over several GPUs.
"""
from __future__ import annotations


def partition_groups(m: int, d: int, world: int):
    """[(f0, f1)] per rank: frames f0..f1-1 hold a contiguous run of whole
    groups; groups are split as evenly as possible (earlier ranks take the
    extra ones).  Ranks beyond the group count get (m, m)."""
    if m < 1 or d < 1 or world < 1:
        raise ValueError("m, d and world must be >= 1")
    g = (m + d - 1) // d
    base, extra = divmod(g, world)
    out, g0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        f0, f1 = min(m, g0 * d), min(m, (g0 + n) * d)
        out.append((f0, f1))
        g0 += n
    return out


def accumulate_sharded(accumulate, frames, d: int, num, den, rank: int, world: int, group=None,
                       reduce: bool = True):
    """Each rank accumulates its run of groups with ``accumulate(frames_slice,
    d, num, den)`` into its own num/den (zero-initialised by the caller), then,
    with ``reduce`` and world > 1, num and den are summed across ranks with
    torch.distributed.all_reduce.  Returns the (f0, f1) run this rank
    processed."""
    f0, f1 = partition_groups(len(frames), d, world)[rank]
    if f1 > f0:
        accumulate(frames[f0:f1], d, num, den)
    if reduce and world > 1:
        import torch.distributed as dist
        dist.all_reduce(num, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(den, op=dist.ReduceOp.SUM, group=group)
    return f0, f1
