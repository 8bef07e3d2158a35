"""Copy sharding through libsim (Supplementary B: the partitions are independent;
Supplementary A, Eq. 8 summed over all of them).  Two gloo ranks, two processes on
cuda:0, each evolve their own subtree of the copy tree (dist.copy_lists) with
sim_evolve_halves_list and contract it into a partial amplitude block
(sim_amplitudes: split-fp16 and FP64 plain).  The blocks are copied to the host and
summed over gloo (dist.reduce_amplitudes); the sum is the oracle's cut-and-sum over
all copies.  The ranks' kernels never wait on each other: the only exchange is the
host-side reduce after both ranks' GPU work has finished."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(4, 5, 16, 3, 2, 60, 50), (6, 5, 16, 1, 3, 300, 200)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _selection(R, C, b, nsu, nsl, seed):
    rng = np.random.default_rng(seed)
    nu, nl = b * C, (R - b) * C
    su = np.sort(rng.choice(1 << nu, nsu, replace=False)).astype(np.uint64)
    sl = np.sort(rng.choice(1 << nl, nsl, replace=False)).astype(np.uint64)
    return su, sl


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    try:
        import paper_1802_06952_gb300 as sim
        from paper_1802_06952_gb300 import dist as sdist
        torch.cuda.set_device(0)
        sim.lib()
        for (R, C, d, seed, b, nsu, nsl) in CASES:
            su, sl = _selection(R, C, b, nsu, nsl, seed)
            circ = sim.sim_build_circuit(R, C, d, seed, b)
            plan, c, copies, nu, nl = sim.sim_cut(circ, b)
            mine = sdist.rank_list(c, world, rank)
            blocks = []
            for prec, kind, dt in ((sim.SIM_C64, sim.SIM_SPLIT_FP16, torch.complex64),
                                   (sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, torch.complex128)):
                h = sim.sim_evolve_halves_list(plan, prec, mine, su, sl)
                blk = torch.zeros((sl.size, su.size), dtype=dt, device="cuda")
                sim.sim_amplitudes(h, kind, False, blk)
                sim.sim_status()
                sim.sim_destroy_halves(h)
                host = blk.cpu()
                sdist.reduce_amplitudes(host)
                blocks.append(host.numpy())
            sim.sim_destroy_cut(plan)
            sim.sim_destroy_circuit(circ)
            out.append((int(mine.size), blocks))
        sim.sim_release_cache()
        q.put((rank, out, None))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, None, repr(e)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_cuda0_and_reduce_partial_blocks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06952_gb300 import build
    build.build()
    import oracle
    from oracle import circuit as oc
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, out, err in got:
        assert err is None, (rank, err)
    for i, (R, C, d, seed, b, nsu, nsl) in enumerate(CASES):
        gates, plan = oc.grid_cut(R, C, d, seed, b)
        su, sl = _selection(R, C, b, nsu, nsl, seed)
        ref = oracle.cut_amplitudes(plan, su, sl)
        scale = np.max(np.abs(ref))
        assert sum(out[i][0] for _, out, _ in got) == plan.copies
        for rank, out, _ in got:
            split, plain = out[i][1]
            assert np.max(np.abs(split - ref)) <= 1e-5 * scale, (rank, i)
            assert np.max(np.abs(plain - ref)) <= 1e-12 * scale, (rank, i)
