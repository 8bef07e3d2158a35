"""GPU parity of batches of circuits (sim_batch_*), through the C-ABI: every
circuit's full amplitude vector is produced into the shared output buffer; its
statistics and a random subset of amplitudes are checked against the oracle's
uncut state vector, for fixed choices, the autotuner and graph replays."""
import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-5
# grids 5x4 and 6x4 (20 and 24 qubits), cut at the middle row, depths spanning
# c = 4, 6 and 8 cut CZs (layers 7, 8, 15, 16)
DESCS = [(5, 4, 12, 0, 2), (6, 4, 16, 1, 3), (5, 4, 20, 2, 2), (6, 4, 13, 3, 3), (6, 4, 19, 4, 3),
         (5, 4, 16, 5, 2)]
S = 2048


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06952_gb300 import build
    build.build()
    sim.lib()
    torch.cuda.set_device(0)
    yield
    sim.sim_release_cache()


@pytest.fixture(scope="module")
def reference():
    rng = np.random.default_rng(21)
    idx, ref, cs = [], [], []
    for (R, C, d, seed, b) in DESCS:
        gates, plan = oc.grid_cut(R, C, d, seed, b)
        cs.append(plan.c)
        sv = oracle.statevector(R * C, gates)
        ii = rng.choice(1 << (R * C), S, replace=False).astype(np.uint64)
        idx.append(ii)
        ref.append(sv[ii.astype(np.int64)])
    return np.stack(idx), np.stack(ref), cs


def check(st, sub, reference):
    idx, ref, cs = reference
    for i in range(len(DESCS)):
        assert abs(st[i, 0] - 1.0) <= 1e-5          # sum |A|^2 over all 2^n amplitudes
        assert abs(st[i, 1] - 1.0) <= 1e-5          # mean 2^n |A|^2
        err = np.max(np.abs(sub[i] - ref[i])) / np.max(np.abs(ref[i]))
        assert err <= TOL_SPLIT, (i, err)


@pytest.mark.parametrize("contraction", [sim.SIM_SPLIT_BF16, sim.SIM_SPLIT_FP16])
def test_batch_fixed_choices(reference, contraction):
    idx, ref, cs = reference
    assert sorted(set(cs)) == [4, 6, 8]
    b = sim.sim_batch_create(DESCS, idx, contraction=contraction)
    try:
        sim.sim_batch_run(b)
        sim.sim_status()
        st, sub = sim.sim_batch_results(b, len(DESCS), S)
        check(st, sub, reference)
        for i, (R, C, d, seed, cut) in enumerate(DESCS):
            info, ms = sim.sim_batch_info(b, i)
            assert info["n"] == R * C and info["c"] == cs[i] and info["fuse"] == 13 and ms == 0
    finally:
        sim.sim_destroy_batch(b)


def test_batch_autotuned_graph_replays(reference):
    """Autotuned choices, then an uncaptured run, a captured run and a replay: the
    amplitudes of all three are identical and match the oracle."""
    idx, ref, cs = reference
    b = sim.sim_batch_create(DESCS, idx, autotune=True, use_graph=True)
    try:
        subs = []
        for r in range(3):
            sim.sim_batch_run(b)
            sim.sim_status()
            st, sub = sim.sim_batch_results(b, len(DESCS), S)
            check(st, sub, reference)
            subs.append(sub)
        assert np.array_equal(subs[0], subs[1]) and np.array_equal(subs[1], subs[2])
        shapes = {}
        for i in range(len(DESCS)):
            info, ms = sim.sim_batch_info(b, i)
            assert 10 <= info["fuse"] <= 13 and info["single_cta"] in (0, 1) and info["group"] in (8, 16, 32)
            key = (DESCS[i][0], cs[i])
            shapes.setdefault(key, []).append((info["fuse"], info["single_cta"], info["group"], ms))
        for key, rows in shapes.items():
            assert len({r[:3] for r in rows}) == 1          # one choice per shape
            assert rows[0][3] > 0 and all(r[3] == 0 for r in rows[1:])   # tuned on the first circuit only
    finally:
        sim.sim_destroy_batch(b)


def test_batch_with_gate_lists_and_t_in_pool():
    """A batch mixing a generated circuit, an explicit gate list with controlled X
    gates across the cut, and a circuit of the T-in-pool rule: statistics and a
    random subset of every full vector against the oracle's uncut state vector."""
    from circuits import cx_cut_circuit
    R, C, b, depth, gates_cx = cx_cut_circuit(1)
    descs = [(5, 4, 16, 0, 2), (R, C, depth, 0, b, oc.to_text(R, C, depth, 0, gates_cx), False),
             (5, 4, 16, 3, 2, None, True)]
    gate_lists = [oc.generate(5, 4, 16, 0, 2), gates_cx, oc.generate(5, 4, 16, 3, 2, t_in_pool=True)]
    rng = np.random.default_rng(5)
    n_sub = 512
    idx = np.stack([rng.choice(1 << 16, n_sub, replace=False) for _ in descs]).astype(np.uint64)
    bat = sim.sim_batch_create(descs, idx)
    try:
        sim.sim_batch_run(bat)
        sim.sim_status()
        st, sub = sim.sim_batch_results(bat, len(descs), n_sub)
        for i, (d, g) in enumerate(zip(descs, gate_lists)):
            n = d[0] * d[1]
            sv = oracle.statevector(n, g)
            ref = sv[idx[i].astype(np.int64) % (1 << n)]
            assert abs(st[i, 0] - 1.0) <= 1e-5
            got = sub[i]
            assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= TOL_SPLIT, i
    finally:
        sim.sim_destroy_batch(bat)
