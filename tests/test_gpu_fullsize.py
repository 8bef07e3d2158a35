"""GPU parity against the FP64 oracle at full half size, through the C-ABI.

  30-qubit halves   one copy of a 60-qubit 6x10 grid circuit (depth 16, cut between
                    rows 2 and 3): both 2^30-entry leaves of the complex64 fused
                    sweeps (both pass formations) and of the plain complex128 path,
                    on 4096 seeded entries each, against the oracle's gate-by-gate
                    FP64 half-states (Supplementary A, Eqs. 4-5 per half), and the
                    4096 x 4096 amplitude block of that copy (Eq. 8 with one term)
  64-qubit halves   one seeded copy of the 8x8, depth-22 circuit: the upper
                    32-qubit leaf (64 GB in FP64 on the host, about four minutes of
                    oracle time) against the oracle, and the split block against the
                    plain FP64 path's; with SIM_LONG_TESTS=1 both leaves and the
                    block against the oracle
  Born sampling     2^16 Born-rule samples of the full 2^30-amplitude vector of the
                    30-qubit 6x5 depth-16 circuit: proposals bit-exact against the
                    oracle's stream, decisions against the oracle's on its own FP64
                    amplitudes (Section 3: measurement outcomes)

The GPU's sweeps over 2^30 and 2^32 entries reach qubit strides and copy-tree
chunkings that the smaller parity tests never meet.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-5
TOL_PLAIN = 1e-12
LONG = os.environ.get("SIM_LONG_TESTS") == "1"


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
    scale = float(np.max(np.abs(ref)))
    diff = float(np.max(np.abs(got - ref)))
    return diff if scale == 0 else diff / scale


def leaf(h, half, k, n, dt):
    buf = torch.zeros(n, dtype=dt, device="cuda")
    sim.sim_halves_leaf(h, half, k, buf)
    return buf.cpu().numpy().astype(np.complex128)


def halves_case(R, C, d, seed, b, nsel, copy_seed, halves=(0, 1)):
    """One seeded copy of the circuit: GPU leaves (complex64 fused sweeps in both
    pass formations, complex128 plain path) on nsel seeded entries per half and the
    split-fp16 / FP64 contractions of that copy, against the oracle's half-states
    of `halves` (the block against the oracle when both are given, else the split
    block against the plain FP64 path's block)."""
    gates, oplan = oc.grid_cut(R, C, d, seed, b)
    rng = np.random.default_rng(copy_seed)
    k = int(rng.integers(0, oplan.copies))
    su = np.sort(rng.choice(1 << oplan.n_u, nsel, replace=False)).astype(np.uint64)
    sl = np.sort(rng.choice(1 << oplan.n_l, nsel, replace=False)).astype(np.uint64)
    # the oracle's half-states, one at a time (2^n complex128 each), at the selections
    want = [None, None]
    for half, sel in ((0, su), (1, sl)):
        if half in halves:
            hs = oracle.half_state(oplan, half, k)
            want[half] = hs[sel.astype(np.int64)].copy()
            del hs
    outer = want[1][:, None] * want[0][None, :] if len(halves) == 2 else None
    blocks = {}
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    plan, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        assert (c, nu, nl) == (oplan.c, oplan.n_u, oplan.n_l)
        lst = np.array([k], dtype=np.uint64)
        for order in (0, 1):
            h = sim.sim_evolve_halves_list(plan, sim.SIM_C64, lst, su, sl, opts={"pass_order": order})
            try:
                for half, n in ((0, su.size), (1, sl.size)):
                    if want[half] is not None:
                        got = leaf(h, half, k, n, torch.complex64)
                        assert rel_err(got, want[half]) <= TOL_SPLIT, (order, half)
                out = torch.zeros((sl.size, su.size), dtype=torch.complex64, device="cuda")
                sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, out)
                sim.sim_status()
                blocks[order] = out.cpu().numpy()
                if outer is not None:
                    assert rel_err(blocks[order], outer) <= TOL_SPLIT, order
                del out
            finally:
                sim.sim_destroy_halves(h)
            sim.sim_release_cache()
        hp = sim.sim_evolve_halves_list(plan, sim.SIM_C128_PLAIN, lst, su, sl)
        try:
            for half, n in ((0, su.size), (1, sl.size)):
                if want[half] is not None:
                    assert rel_err(leaf(hp, half, k, n, torch.complex128), want[half]) <= TOL_PLAIN, half
            outp = torch.zeros((sl.size, su.size), dtype=torch.complex128, device="cuda")
            sim.sim_amplitudes(hp, sim.SIM_FP64_PLAIN, False, outp)
            sim.sim_status()
            plain = outp.cpu().numpy()
            if outer is not None:
                assert rel_err(plain, outer) <= TOL_PLAIN
            else:
                for order, blk in blocks.items():
                    assert rel_err(blk, plain) <= TOL_SPLIT, order
        finally:
            sim.sim_destroy_halves(hp)
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)
        sim.sim_release_cache()


def test_30q_halves_match_oracle():
    halves_case(6, 10, 16, 0, 3, 4096, 30)


def test_64q_halves_match_oracle():
    """The upper 32-qubit leaf against the oracle (about four minutes of oracle time
    on 16 cores); both leaves and the block with SIM_LONG_TESTS=1 (about eight)."""
    halves_case(8, 8, 22, 0, 4, 4096, 64, halves=(0, 1) if LONG else (0,))


def test_born_samples_2to30_match_oracle():
    """Born-rule samples of all 2^30 amplitudes of the 30-qubit 6x5 depth-16 circuit
    (seed 0, split-fp16 contraction): every accepted index is the oracle's proposal
    at that ordinal (bit-exact stream), and accept / reject decisions agree with the
    oracle's on its own FP64 amplitudes except where u * p_max and p are closer than
    the amplitude error allows."""
    R, C, d, seed, b = 6, 5, 16, 0, 3
    n = R * C
    gates, oplan = oc.grid_cut(R, C, d, seed, b)
    ref = oracle.cut_amplitudes(oplan).ravel()          # x = x_u + 2^15 x_l, FP64
    p_o = ref.real * ref.real + ref.imag * ref.imag
    del ref
    pmax_o = float(p_o.max())
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    plan, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        h = sim.sim_evolve_halves(plan, sim.SIM_C64, 0, copies)
        out = torch.empty((1 << nl, 1 << nu), dtype=torch.complex64, device="cuda")
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, out)
        sim.sim_status()
        sim.sim_destroy_halves(h)
        S, sseed = 1 << 16, 2024
        idx, ords, xeb = sim.sim_born_sample(out, n, sseed, S, 1 << 26)
        del out
        assert idx.size == S and np.all(np.diff(ords.astype(np.int64)) > 0)
        # the measured bound: 2^n p_max against the oracle's
        assert abs(xeb[2] - pmax_o * 2.0 ** n) <= 3e-5 * pmax_o * 2.0 ** n
        i_all, u_all = oracle.born_proposals(sseed, 1 << n, 0, int(ords[-1]) + 1)
        assert np.array_equal(i_all[ords.astype(np.int64)], idx)
        gap = u_all * pmax_o - p_o[i_all.astype(np.int64)]
        acc_gpu = np.zeros(i_all.size, dtype=bool)
        acc_gpu[ords.astype(np.int64)] = True
        differ = acc_gpu != (gap < 0)
        assert np.all(np.abs(gap[differ]) <= 3e-5 * pmax_o)
        assert differ.sum() <= max(3, int(1e-4 * i_all.size))
        # cross-entropy of the samples on the oracle's probabilities
        lin, log = oracle.cross_entropy(p_o[idx.astype(np.int64)], n)
        assert abs(lin - xeb[0]) <= 1e-3 and abs(log - xeb[1]) <= 1e-3
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)
