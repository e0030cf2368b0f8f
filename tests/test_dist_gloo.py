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


def tiny_worker(rank, world, port, q):
    """combine_shards with oracle walks of tiny matrices: with more ranks than
    32-index units some shards are empty, rank 0's included ([0, 0))."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2501_15126_gb300 import dist as pd
        from paper_2501_15126_gb300 import synth
        got = []
        for n in (4, 6, 7, 8):
            af = synth.single_er(n, 0.6, 30 + n, values="f64")
            ai = synth.single_er(n, 0.6, 30 + n, values="01")
            calls = []

            def walk_f(lo, hi):
                calls.append((lo, hi))
                s, _ = oracle.nw_range(af, lo, hi)
                return (s.hi, s.lo), (lo, hi)

            def walk_i(lo, hi):
                part = oracle.nw2_range(ai, lo, hi)
                return [part & ((1 << 64) - 1), part >> 64], (lo, hi)

            vf, rec = pd.combine_shards(n, walk_f, 0)
            vi, _ = pd.combine_shards(n, walk_i, 2)
            got.append((n, vf, vi, rec, calls))
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_empty_shards_contribute_nothing():
    """Three ranks, n = 4..8 (8 to 128 Gray indices: one to four 32-index
    units), so some ranks own no indices; the combined permanent still equals
    brute force (Eq. 1) on every rank, and an empty shard never walks."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    world = 3
    procs = [ctx.Process(target=tiny_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2501_15126_gb300 import dist as pd
    from paper_2501_15126_gb300 import synth
    for k, n in enumerate((4, 6, 7, 8)):
        af = synth.single_er(n, 0.6, 30 + n, values="f64")
        ai = synth.single_er(n, 0.6, 30 + n, values="01")
        want_f, want_i = float(oracle.brute(af)), oracle.brute_int(ai)
        walked = []
        for rank, got in out:
            gn, vf, vi, rec, calls = got[k]
            assert gn == n
            assert abs(vf - want_f) <= 1e-12 * abs(want_f)
            assert vi == want_i
            lo, hi = pd.shard_range(1 << (n - 1), world, rank)
            assert calls == ([] if lo == hi else [(lo, hi)])
            assert rec == (None if lo == hi else (lo, hi))
            walked += calls
        assert sum(hi - lo for lo, hi in walked) == 1 << (n - 1)
        assert any(pd.shard_range(1 << (n - 1), world, r)[1] == 0 for r in range(world)) == (n <= 7)


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


def test_finish_exact_matches_the_oracle_finishing():
    """The host-side finishing of a combined exact sum (Algorithm 1 with doubled
    x: S = (-1)^(n-1) 2^(n-1) perm modulo 2^(64 w)) against Eq. 2."""
    import oracle
    from paper_2501_15126_gb300 import dist as pd
    from paper_2501_15126_gb300 import synth
    for n, seed in ((9, 1), (14, 2), (17, 3)):
        a = synth.single_er(n, 0.4, seed, values="01")
        a[0, :] *= -1 if seed == 2 else 1
        s = oracle.nw2_range(a, 0, 1 << (n - 1))
        assert pd.finish_exact(s, n, 2) == oracle.ryser_gray(a)


def gpu_shard_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2501_15126_gb300 import dist as pd
        from paper_2501_15126_gb300 import synth
        af = synth.single_er(24, 0.25, 19, values="f64")
        ai = synth.single_er(24, 0.25, 19, values="01")
        vf, rf = pd.permanent_sharded(af)
        vi, ri = pd.permanent_sharded(ai)
        q.put((rank, vf, vi, rf.steps, ri.steps))
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_two_processes_shard_one_permanent_through_the_c_abi():
    """Two processes (sharing the one GPU; their kernels never wait on each
    other) each walk half of the Gray range of one n=24 permanent through
    perm_plan_create + perm_compute; the partial sums are combined over gloo.
    FP64 within 1e-9 of the oracle, exact bit-identical to Eq. 2."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=gpu_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    import oracle
    from paper_2501_15126_gb300 import synth
    af = synth.single_er(24, 0.25, 19, values="f64")
    ai = synth.single_er(24, 0.25, 19, values="01")
    want_f = float(oracle.nw_perm(af, threads=8)[0])
    want_i = oracle.ryser_gray(ai)
    for r in out:
        assert abs(r[1] - want_f) <= 1e-9 * abs(want_f)
        assert r[2] == want_i
        assert r[3] == r[4] == 1 << 22
