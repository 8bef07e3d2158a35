"""Multi-rank path on CPU: two gloo ranks shard the copies of a cut circuit, each
computes its partial amplitude block (with the FP64 oracle standing in for a
rank's GPU), and one sum-reduce reproduces the full cut-and-sum; the slowest-rank
timing reduction used by bench.py is checked too."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1802_06952_gb300 import dist as sdist


def test_copy_ranges_partition():
    for copies in (1, 7, 16, 256, 16384):
        for world in (1, 2, 3, 8):
            rs = sdist.copy_ranges(copies, world)
            assert rs[0][0] == 0 and rs[-1][1] == copies
            assert all(a[1] == b[0] for a, b in zip(rs[:-1], rs[1:]))
            sizes = [e - b for b, e in rs]
            assert max(sizes) - min(sizes) <= 1


def test_copy_lists_partition():
    for c in (0, 3, 8, 14):
        for world in (1, 2, 3, 8):
            ls = sdist.copy_lists(c, world)
            allk = np.sort(np.concatenate(ls))
            assert np.array_equal(allk, np.arange(1 << c, dtype=np.uint64))
            sizes = [x.size for x in ls]
            assert max(sizes) - min(sizes) <= 1


def test_copy_lists_are_subtrees_of_the_copy_tree():
    """The 64-qubit circuit's copy tree (8x8, depth 22, c = 16, levels fixing 4, 8,
    12 and 16 copy bits, read from the library's plan): dealt out by copy_lists, the
    ranks' tree nodes add up to the full tree's at every level (no node evolved
    twice), while contiguous ranges of k make every rank evolve every node of the
    early levels."""
    import paper_1802_06952_gb300 as sim
    circ = sim.sim_build_circuit(8, 8, 22, 0, 4)
    plan, c, copies, nu, nl = sim.sim_cut(circ, 4)
    try:
        for half in (0, 1):
            bits = [int(b1) for (_, _, b1, _) in sim.sim_plan_levels(plan, half)]
            assert bits[-1] == c == 16
            full = [1 << b for b in bits]
            for world in (2, 4, 8, 16):
                nodes = np.array([sdist.tree_nodes(lst, bits) for lst in sdist.copy_lists(c, world)])
                assert list(nodes.sum(axis=0)) == [max(f, world) if f < world else f for f in full]
                ranged = np.array([sdist.tree_nodes(np.arange(b, e, dtype=np.uint64), bits)
                                   for b, e in sdist.copy_ranges(copies, world)])
                assert ranged[:, 0].sum() == world * full[0]
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from oracle import circuit as oc
        gates, plan = oc.grid_cut(4, 5, 16, 3, 2)
        rng = np.random.default_rng(0)
        su = np.sort(rng.choice(1 << plan.n_u, 40, replace=False)).astype(np.uint64)
        sl = np.sort(rng.choice(1 << plan.n_l, 30, replace=False)).astype(np.uint64)
        b, e = sdist.rank_range(plan.copies, world, rank)
        part = oracle.cut_amplitudes(plan, su, sl, b, e)
        block = torch.from_numpy(part.copy())
        sdist.reduce_amplitudes(block)
        slowest = sdist.max_over_ranks(1.5 + rank)
        q.put((rank, block.numpy(), slowest, (b, e)))
    finally:
        dist.destroy_process_group()


def test_two_rank_copy_sharding_sum_reduce():
    import oracle
    from oracle import circuit as oc
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gates, plan = oc.grid_cut(4, 5, 16, 3, 2)
    rng = np.random.default_rng(0)
    su = np.sort(rng.choice(1 << plan.n_u, 40, replace=False)).astype(np.uint64)
    sl = np.sort(rng.choice(1 << plan.n_l, 30, replace=False)).astype(np.uint64)
    ref = oracle.cut_amplitudes(plan, su, sl)
    ranges = sorted(g[3] for g in got)
    assert ranges[0][0] == 0 and ranges[-1][1] == plan.copies and ranges[0][1] == ranges[1][0]
    for rank, block, slowest, _ in got:
        assert np.max(np.abs(block - ref)) <= 1e-15
        assert slowest == 2.5
