"""Selected leaf entries computed from an ancestor's state (sim_opts.sparse_leaves):
the same leaves and amplitudes as whole leaf states swept and gathered, and the
oracle's cut-and-sum, through the C-ABI.

The ops of the last d copy-tree levels act non-diagonally on a qubit set Q; an
entry x of a leaf is then those ops applied to the 2^|Q| entries of its ancestor d
levels up that agree with x outside Q (Section 2.3.1: only the selected entries are
needed).  Forced mode takes the largest d with |Q| <= 10: on these 8- to 12-qubit
halves that reaches up to the root level, so the slots of several levels are
applied in one evaluation."""
import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def rel(a, b):
    s = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (s if s > 0 else 1.0)


def leaves(h, copies, nsu, nsl):
    out = []
    for k in copies:
        for half, n in ((0, nsu), (1, nsl)):
            buf = torch.zeros(n, dtype=torch.complex64, device="cuda")
            sim.sim_halves_leaf(h, half, int(k), buf)
            out.append(buf.cpu().numpy())
    return out


def sweep_launches(fn):
    sim.sim_profile_read(reset=True)
    sim.sim_profile_enable(True)
    r = fn()
    torch.cuda.synchronize()
    sim.sim_profile_enable(False)
    return r, sim.sim_profile_read(reset=True)["launches"][sim.SIM_PHASE_SWEEP]


def check(circ, gplan, b, copies, su, sl, copy_list=None):
    plan, c, ncopies, nu, nl = sim.sim_cut(circ, b)
    try:
        def evolve(mode):
            opts = {"sparse_leaves": mode}
            if copy_list is None:
                return sim.sim_evolve_halves(plan, sim.SIM_C64, 0, ncopies, su, sl, opts)
            return sim.sim_evolve_halves_list(plan, sim.SIM_C64, copy_list, su, sl, opts)

        hs, n_sparse = sweep_launches(lambda: evolve(1))
        hw, n_whole = sweep_launches(lambda: evolve(-1))
        try:
            # the sparse route runs no passes of the levels it covers
            assert n_sparse < n_whole
            ks = list(copy_list) if copy_list is not None else [0, ncopies // 3, ncopies - 1]
            for a, w in zip(leaves(hs, ks, su.size, sl.size), leaves(hw, ks, su.size, sl.size)):
                assert rel(a, w) <= 1e-6
            outs = []
            for h in (hs, hw):
                o = torch.zeros((sl.size, su.size), dtype=torch.complex64, device="cuda")
                sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, o)
                sim.sim_status()
                outs.append(o.cpu().numpy())
            if copy_list is None:
                ref = oracle.cut_amplitudes(gplan, su, sl)
            else:
                ref = sum(oracle.cut_amplitudes(gplan, su, sl, int(k), int(k) + 1) for k in copy_list)
            assert rel(outs[0], ref) <= TOL
            assert rel(outs[1], ref) <= TOL
        finally:
            sim.sim_destroy_halves(hs)
            sim.sim_destroy_halves(hw)
    finally:
        sim.sim_destroy_cut(plan)


@pytest.mark.parametrize("R,C,d,seed,b,nsu,nsl", [
    (4, 5, 16, 0, 2, 37, 101),     # 10 + 10 qubits, ragged selections
    (6, 4, 17, 2, 3, 64, 5),       # 12 + 12 qubits
    (4, 6, 22, 1, 2, 1, 300),      # single upper entry, deep circuit
])
def test_sparse_leaves_match_whole_leaves_and_oracle(R, C, d, seed, b, nsu, nsl):
    gates, gplan = oc.grid_cut(R, C, d, seed, b)
    rng = np.random.default_rng(seed + 11)
    su = np.sort(rng.choice(1 << gplan.n_u, nsu, replace=False)).astype(np.uint64)
    sl = np.sort(rng.choice(1 << gplan.n_l, nsl, replace=False)).astype(np.uint64)
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    try:
        check(circ, gplan, b, gplan.copies, su, sl)
    finally:
        sim.sim_destroy_circuit(circ)


@pytest.mark.parametrize("name", ["CX", "CT", "CY2"])
def test_sparse_leaves_with_controlled_gate_cuts_and_a_copy_list(name):
    from circuits import cx_cut_circuit
    R, C, b, depth, gates = cx_cut_circuit(3, name)
    n, n_u = R * C, b * C
    gplan = oc.CutPlan(n, n_u, gates)
    rng = np.random.default_rng(4)
    su = np.sort(rng.choice(1 << n_u, 40, replace=False)).astype(np.uint64)
    sl = np.sort(rng.choice(1 << (n - n_u), 23, replace=False)).astype(np.uint64)
    circ = sim.sim_build_circuit(gate_list=oc.to_text(R, C, depth, 0, gates))
    try:
        lst = np.array([gplan.copies - 1, 0, gplan.copies // 2 + 1], dtype=np.uint64)
        check(circ, gplan, b, gplan.copies, su, sl, copy_list=lst)
    finally:
        sim.sim_destroy_circuit(circ)


def test_sparse_leaves_option_checked():
    circ = sim.sim_build_circuit(4, 4, 10, 0, 2)
    plan, c, copies, nu, nl = sim.sim_cut(circ, 2)
    try:
        with pytest.raises(sim.SimError) as e:
            sim.sim_evolve_halves(plan, sim.SIM_C64, 0, copies, None, None, {"sparse_leaves": 2})
        assert e.value.code == sim.SIM_EINVAL
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)
