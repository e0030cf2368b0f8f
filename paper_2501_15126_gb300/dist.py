"""Host-side multi-rank logic: Gray-range sharding and the combination of
partial sums (Sec. II-A: Gray-index ranges are independent, so one permanent
splits across ranks with a single exchange of partial sums at the end).

All functions work on any torch.distributed backend (gloo on CPU in the
tests, NCCL on GPUs); the exchange is one all_gather of a few words, and the
combination runs in rank order on every rank, so every rank gets the same bits.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

MASK64 = (1 << 64) - 1


def shard_range(total: int, world: int, rank: int, align: int = 32):
    """[lo, hi) of the Gray indices [0, total) owned by `rank`: contiguous,
    multiples of `align` except the end of the last shard."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    units = (total + align - 1) // align
    lo = units * rank // world * align
    hi = min(total, units * (rank + 1) // world * align)
    return lo, hi


def _gather(values, device):
    t = torch.tensor(values, dtype=torch.float64 if isinstance(values[0], float) else torch.int64, device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [o.cpu().tolist() for o in out]


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def combine_f64(hi: float, lo: float, device="cpu"):
    """Sums every rank's (hi, lo) partial with compensated additions in rank order."""
    parts = _gather([hi, lo], device)
    s, e = 0.0, 0.0
    for h, l in parts:
        s, err = _two_sum(s, h)
        e += err + l
    return s + e, e - ((s + e) - s)


def combine_exact(words, device="cpu") -> int:
    """Sums every rank's partial given as little-endian 64-bit words, modulo 2^(64 len(words))."""
    w = len(words)
    signed = [(x - (1 << 64)) if x >> 63 else x for x in words]   # int64 transport
    parts = _gather(signed, device)
    total = 0
    for p in parts:
        total += sum((v & MASK64) << (64 * i) for i, v in enumerate(p))
    return total % (1 << (64 * w))


def max_over_ranks(value: float, device="cpu") -> float:
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
