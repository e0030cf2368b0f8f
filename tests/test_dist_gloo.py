"""World-size-2 gloo tests (CPU) of the multi-rank host logic: each rank walks
its shard of the Gray range with the oracle, the partial sums are exchanged
and combined, and the result equals the single-rank walk; timing takes the
max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

MASK128 = (1 << 128) - 1


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2501_15126_gb300 import dist as pd
        from paper_2501_15126_gb300 import synth
        n = 17
        af = synth.single_er(n, 0.3, 9, values="f64")
        ai = synth.single_er(n, 0.3, 9, values="01")
        lo, hi = pd.shard_range(1 << (n - 1), world, rank)
        s, _ = oracle.nw_range(af, lo, hi)
        f_hi, f_lo = pd.combine_f64(s.hi, s.lo)
        part = oracle.nw2_range(ai, lo, hi)
        words = [part & ((1 << 64) - 1), part >> 64]
        tot = pd.combine_exact(words)
        mx = pd.max_over_ranks(float(rank + 1))
        q.put((rank, f_hi, f_lo, tot, mx, lo, hi))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_rank_shards_combine_to_the_whole(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    import oracle
    from paper_2501_15126_gb300 import synth
    n = 17
    af = synth.single_er(n, 0.3, 9, values="f64")
    ai = synth.single_er(n, 0.3, 9, values="01")
    whole, absum = oracle.nw_range(af, 0, 1 << (n - 1))
    whole_i = oracle.nw2_range(ai, 0, 1 << (n - 1))
    assert out[0][5] == 0 and out[-1][6] == 1 << (n - 1) and out[0][6] == out[1][5]
    for r in out:
        assert abs((r[1] + r[2]) - float(whole)) <= 1e-15 * float(absum)
        assert r[3] == whole_i
        assert r[4] == float(world)
    # every rank combined to the same bits
    assert len({(r[1], r[2], r[3]) for r in out}) == 1


def test_shard_range_covers_exactly():
    from paper_2501_15126_gb300 import dist as pd
    for total in (32, 1000, 1 << 20, (1 << 35)):
        for world in (1, 2, 3, 8):
            shards = [pd.shard_range(total, world, r) for r in range(world)]
            assert shards[0][0] == 0 and shards[-1][1] == total
            for (a, b), (c, d) in zip(shards, shards[1:]):
                assert b == c
            for a, b in shards[:-1]:
                assert a % 32 == 0 and b % 32 == 0
