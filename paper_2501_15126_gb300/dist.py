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


def finish_exact(total: int, n: int, words: int) -> int:
    """The permanent from a whole walk's doubled Nijenhuis-Wilf sum S modulo
    2^(64 words): S = (-1)^(n-1) 2^(n-1) perm, so the low n-1 bits are zero and
    the rest is perm with its sign (the library's own finishing step, applied to
    a sum combined across ranks)."""
    bits = 64 * words
    if total & ((1 << (n - 1)) - 1):
        raise ValueError("combined exact sum is not divisible by 2^(n-1)")
    v = total >> (n - 1)
    width = bits - (n - 1)
    if v >> (width - 1):
        v -= 1 << width
    return -v if (n - 1) % 2 else v


def combine_shards(n: int, walk, words: int = 0, device="cpu"):
    """One permanent from this rank's shard of the Gray range [0, 2^(n-1)):
    `walk(lo, hi)` returns the shard's raw partial sum -- (hi, lo) doubles, or
    `words` little-endian 64-bit words of the doubled exact sum modulo
    2^(64 words) -- and an opaque record; one all_gather and the finishing step
    give every rank the same value.  A rank whose shard is empty (more ranks
    than 32-index units, tiny n) contributes zero without calling `walk`.
    Returns (value, the record or None)."""
    lo, hi = shard_range(1 << (n - 1), dist.get_world_size(), dist.get_rank())
    if lo == hi:
        part, rec = ([0] * words if words else (0.0, 0.0)), None
    else:
        part, rec = walk(lo, hi)
    if words:
        return finish_exact(combine_exact(list(part), device), n, words), rec
    s_hi, s_lo = combine_f64(part[0], part[1], device)
    f = 2.0 if n % 2 else -2.0          # 4 (n mod 2) - 2, Algorithm 1
    return (s_hi + s_lo) * f, rec


def permanent_sharded(a, device="cpu", **kw):
    """One permanent split across the ranks of the default process group:
    this rank walks its shard of the Gray range on its GPU through the C ABI
    (perm_plan_create + perm_compute with g_lo/g_hi), then one all_gather of
    the partial sums and the finishing step give every rank the same value.
    Integer inputs walk one ring, 2^(64 w), on every rank (w from the
    matrix's bound, as a sub-range of it takes by default), so the partial
    sums add up.  Returns (value, this rank's Result, or None for an empty
    shard)."""
    import numpy as np
    from paper_2501_15126_gb300 import _abi as A
    a = np.asarray(a)
    n = a.shape[0]
    words = 0
    if np.issubdtype(a.dtype, np.integer):
        words = kw.get("exact_words") or A.inspect(a).exact_words or 3
        kw["exact_words"] = words

    def walk(lo, hi):
        r = A.permanent(a, g_lo=lo, g_hi=hi, **kw)
        if words:
            return [int(r.partial[i]) for i in range(words)], r
        return (r.f64, r.f64_lo), r

    return combine_shards(n, walk, words, device)


def max_over_ranks(value: float, device="cpu") -> float:
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
