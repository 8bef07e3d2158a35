"""GPU parity of multi-part cuts (Section 3, Fig. 3) through the C-ABI: the grid in
three or four row bands, each part evolved for all its copies, the parts contracted
boundary by boundary.  References: the oracle's uncut state vector (the rewrite is
an identity) and its multi-part cut-and-sum on selections.

Tolerances: FP64 plain <= 1e-12; split fp16 <= 1e-5 (two or three chained
contractions).  Split bf16 is refused for chained contractions (SIM_EUNSUPPORTED):
each step can leave 3 * 2^-16 of the magnitude sum of its products, and the steps'
roundings add up past 1e-5."""
import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref))) / float(np.max(np.abs(ref)))


def run(R, C, d, seed, rows, precision, kind, sels=None, opts=None):
    circ = sim.sim_build_circuit(R, C, d, seed, rows[0])
    plan, t, cs, nq = sim.sim_cut_multi(circ, rows)
    try:
        shape = [(1 << nq[p]) if sels is None or sels[p] is None else len(sels[p]) for p in range(t)][::-1]
        dt = torch.complex128 if kind == sim.SIM_FP64_PLAIN else torch.complex64
        out = torch.zeros(shape, dtype=dt, device="cuda")
        sim.sim_multi_amplitudes(plan, precision, kind, out, sels, opts)
        return out.cpu().numpy(), cs, nq
    finally:
        sim.sim_destroy_multi(plan)
        sim.sim_destroy_circuit(circ)


@pytest.mark.parametrize("R,C,d,seed,rows", [(6, 3, 12, 1, [2, 4]), (8, 2, 12, 0, [2, 4, 6]), (5, 4, 14, 2, [2, 4])])
def test_multi_part_full_vector(R, C, d, seed, rows):
    gates = oc.generate(R, C, d, seed, rows[0])
    mp = oc.MultiCutPlan(R, C, rows, gates)
    ref = oracle.statevector(R * C, gates).reshape([1 << q for q in mp.nq][::-1])
    got, cs, nq = run(R, C, d, seed, rows, sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN)
    assert cs == [mp.c(j) for j in range(1, mp.t)] and nq == mp.nq
    assert rel_err(got, ref) <= 1e-12
    got, _, _ = run(R, C, d, seed, rows, sim.SIM_C64, sim.SIM_SPLIT_FP16)
    assert rel_err(got, ref) <= 1e-5
    with pytest.raises(sim.SimError) as ei:
        run(R, C, d, seed, rows, sim.SIM_C64, sim.SIM_SPLIT_BF16)
    assert ei.value.code == sim.SIM_EUNSUPPORTED and "FP16" in str(ei.value)


def test_multi_part_selections_and_options():
    """27 qubits in three 9-qubit parts, ragged selections per part; both pass
    formations and a narrower fuse width give the same amplitudes."""
    R, C, d, seed, rows = 9, 3, 14, 3, [3, 6]
    gates = oc.generate(R, C, d, seed, rows[0])
    mp = oc.MultiCutPlan(R, C, rows, gates)
    rng = np.random.default_rng(1)
    sels = [np.sort(rng.permutation(1 << q)[:k]).astype(np.uint64) for q, k in zip(mp.nq, (50, 61, 37))]
    ref = oracle.multi_cut_amplitudes(mp, [s.astype(np.int64) for s in sels])
    got, _, _ = run(R, C, d, seed, rows, sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, sels)
    assert rel_err(got, ref) <= 1e-12
    for opts in (None, {"pass_order": 1}, {"fuse_qubits": 8}):
        got, _, _ = run(R, C, d, seed, rows, sim.SIM_C64, sim.SIM_SPLIT_FP16, sels, opts)
        assert rel_err(got, ref) <= 1e-5, opts
    # a part given in full among selected ones
    sels2 = [sels[0], None, sels[2]]
    ref2 = oracle.multi_cut_amplitudes(mp, [sels[0].astype(np.int64), None, sels[2].astype(np.int64)])
    got, _, _ = run(R, C, d, seed, rows, sim.SIM_C64, sim.SIM_SPLIT_FP16, sels2)
    assert rel_err(got, ref2) <= 1e-5


def test_multi_part_argument_errors():
    circ = sim.sim_build_circuit(6, 3, 12, 1, 2)
    plan, t, cs, nq = sim.sim_cut_multi(circ, [2, 4])
    try:
        out = torch.zeros((64, 64, 64), dtype=torch.complex64, device="cuda")
        for prec, kind in ((sim.SIM_C64, sim.SIM_FP64_PLAIN), (sim.SIM_C128_PLAIN, sim.SIM_SPLIT_BF16)):
            with pytest.raises(sim.SimError) as e:
                sim.sim_multi_amplitudes(plan, prec, kind, out)
            assert e.value.code == sim.SIM_EINVAL
        with pytest.raises(sim.SimError) as e:
            sim.sim_multi_amplitudes(plan, sim.SIM_C64, sim.SIM_SPLIT_FP16, out,
                                     [np.array([64], dtype=np.uint64), None, None])
        assert e.value.code == sim.SIM_EINVAL
    finally:
        sim.sim_destroy_multi(plan)
        sim.sim_destroy_circuit(circ)


def test_multi_part_40q_selection():
    """40 qubits (8x5, depth 10) in parts of 10, 15 and 15 qubits (c = 5 + 5, the
    middle part with 1024 copies): 16 seeded indices per part against the oracle's
    multi-part sum; the two-part cut of the same circuit at the matching entries."""
    R, C, d, seed, rows = 8, 5, 10, 0, [2, 5]
    gates = oc.generate(R, C, d, seed, rows[0])
    mp = oc.MultiCutPlan(R, C, rows, gates)
    rng = np.random.default_rng(2)
    sels = [np.sort(rng.permutation(1 << q)[:16]).astype(np.uint64) for q in mp.nq]
    ref = oracle.multi_cut_amplitudes(mp, [s.astype(np.int64) for s in sels])
    got, cs, nq = run(R, C, d, seed, rows, sim.SIM_C64, sim.SIM_SPLIT_FP16, sels)
    assert cs == [5, 5] and rel_err(got, ref) <= 1e-5
    gotp, _, _ = run(R, C, d, seed, rows, sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, sels)
    assert rel_err(gotp, ref) <= 1e-12
    # the same amplitudes through two 20-qubit halves (cut between rows 3 and 4)
    x = (sels[0][None, None, :] | (sels[1][None, :, None] << np.uint64(10)) |
         (sels[2][:, None, None] << np.uint64(25))).reshape(-1)
    xu, xl = x & np.uint64((1 << 20) - 1), x >> np.uint64(20)
    su, iu = np.unique(xu, return_inverse=True)
    sl, il = np.unique(xl, return_inverse=True)
    circ = sim.sim_build_circuit(R, C, d, seed, rows[0])
    plan, c2, copies, nu, nl = sim.sim_cut(circ, 4)
    try:
        h = sim.sim_evolve_halves(plan, sim.SIM_C128_PLAIN, 0, copies, su, sl)
        out = torch.zeros((sl.size, su.size), dtype=torch.complex128, device="cuda")
        sim.sim_amplitudes(h, sim.SIM_FP64_PLAIN, False, out)
        sim.sim_status()
        two = out.cpu().numpy()[il, iu].reshape(ref.shape)
        sim.sim_destroy_halves(h)
        assert rel_err(two, ref) <= 1e-12
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)


def test_multi_part_rejects_too_many_copies():
    """8x8 at depth 22 cut into 24/16/24 rows: the middle part carries the copy bits
    of both boundaries (32 here), above 24, which is refused before any work
    (SIM_EUNSUPPORTED)."""
    circ = sim.sim_build_circuit(8, 8, 22, 0, 3)
    plan, t, cs, nq = sim.sim_cut_multi(circ, [3, 5])
    try:
        assert cs[0] + cs[1] > 24
        out = torch.zeros(8, dtype=torch.complex64, device="cuda")
        sels = [np.arange(2, dtype=np.uint64)] * 3
        with pytest.raises(sim.SimError) as e:
            sim.sim_multi_amplitudes(plan, sim.SIM_C64, sim.SIM_SPLIT_FP16, out, sels)
        assert e.value.code == sim.SIM_EUNSUPPORTED
    finally:
        sim.sim_destroy_multi(plan)
        sim.sim_destroy_circuit(circ)
