"""sim_amplitudes_noalloc: the split tensor-core contraction for callers that
cannot let the library allocate device memory while they run (their device memory
already belongs to their own allocator, or cudaMalloc / cudaFree would stall a
latency-bound loop).  Its scratch is a fixed device array inside the library.

Checked through the C-ABI against sim_amplitudes on the same evolved halves, on
two calls in a row (the array keeps the previous call's contents), within the
tolerance the other parity tests use; the 16-qubit full vector also against the
oracle's uncut state vector; and the device's free memory is the same before and
after a call on a shape the entry point has not seen.  This file is named so that
pytest collects it last.
"""
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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def evolved(R, C, d, seed, b, sel_u=None, sel_l=None):
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    plan, c, copies, nu, nl = sim.sim_cut(circ, b)
    h = sim.sim_evolve_halves(plan, sim.SIM_C64, 0, copies, sel_u, sel_l)
    M = (1 << nl) if sel_l is None else len(sel_l)
    N = (1 << nu) if sel_u is None else len(sel_u)
    return circ, plan, h, M, N


def release(*objs):
    circ, plan, h = objs[:3]
    sim.sim_destroy_halves(h)
    sim.sim_destroy_cut(plan)
    sim.sim_destroy_circuit(circ)


def test_noalloc_matches_sim_amplitudes_twice():
    cases = [(4, 4, 10, 0, 2, None, None, sim.SIM_SPLIT_BF16),
             (4, 5, 16, 3, 2, np.arange(0, 1024, 3, dtype=np.uint64), np.arange(5, 1024, 7, dtype=np.uint64),
              sim.SIM_SPLIT_FP16)]
    outs = []
    for (R, C, d, seed, b, su, sl, kind) in cases:
        circ, plan, h, M, N = evolved(R, C, d, seed, b, su, sl)
        try:
            ref = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
            sim.sim_amplitudes(h, kind, False, ref)
            sim.sim_status()
            got = torch.full((M, N), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
            sim.sim_amplitudes_noalloc(h, kind, False, got)
            r = ref.cpu().numpy()
            assert rel(got.cpu().numpy(), r) <= TOL
            if su is None:
                # the full 16-qubit vector is the oracle's uncut state vector
                want = oracle.statevector(R * C, oc.generate(R, C, d, seed, b)).reshape(M, N)
                assert rel(got.cpu().numpy(), want) <= TOL
            # a second call in a row on the same output, accumulating: 2x the result
            sim.sim_amplitudes_noalloc(h, kind, True, got)
            assert rel(got.cpu().numpy(), 2 * r) <= TOL
            outs.append(got.cpu().numpy())
        finally:
            release(circ, plan, h)
    assert len(outs) == 2


def test_noalloc_allocates_nothing():
    """After a first call (which loads the library's module on this device, and with
    it the fixed array), a call on a shape not seen before leaves the device's free
    memory unchanged: no cudaMalloc behind it, no pool growth."""
    first = evolved(4, 5, 16, 1, 2, np.arange(0, 1024, 5, dtype=np.uint64), np.arange(0, 1024, 3, dtype=np.uint64))
    second = evolved(4, 5, 16, 2, 2, np.arange(1, 1024, 2, dtype=np.uint64), np.arange(2, 1024, 9, dtype=np.uint64))
    try:
        o1 = torch.zeros((first[3], first[4]), dtype=torch.complex64, device="cuda")
        o2 = torch.zeros((second[3], second[4]), dtype=torch.complex64, device="cuda")
        ref = torch.zeros_like(o2)
        sim.sim_amplitudes(second[2], sim.SIM_SPLIT_FP16, False, ref)
        sim.sim_amplitudes_noalloc(first[2], sim.SIM_SPLIT_FP16, False, o1)
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        sim.sim_amplitudes_noalloc(second[2], sim.SIM_SPLIT_FP16, False, o2)
        torch.cuda.synchronize()
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after == free_before
        assert rel(o2.cpu().numpy(), ref.cpu().numpy()) <= TOL
    finally:
        release(*first)
        release(*second)


def test_noalloc_rejects_oversized_and_host_output():
    # 30 qubits, 256 copies: the split operands need ~200 MB, more than the fixed scratch
    circ, plan, h, M, N = evolved(6, 5, 16, 0, 3, np.arange(8192, dtype=np.uint64), np.arange(8192, dtype=np.uint64))
    try:
        out = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
        with pytest.raises(sim.SimError) as e:
            sim.sim_amplitudes_noalloc(h, sim.SIM_SPLIT_BF16, False, out)
        assert e.value.code == sim.SIM_EINVAL and "scratch" in sim.sim_last_error()
        small = evolved(4, 4, 10, 1, 2)
        try:
            host = torch.zeros((256, 256), dtype=torch.complex64)
            with pytest.raises(sim.SimError) as e2:
                sim.sim_amplitudes_noalloc(small[2], sim.SIM_SPLIT_BF16, False, host)
            assert e2.value.code == sim.SIM_EINVAL
        finally:
            release(*small)
    finally:
        release(circ, plan, h)


def test_noalloc_with_output_phase_cuts():
    """Output-phase cuts (sim_cut_ex): the fixed-scratch contraction signs the block
    like sim_amplitudes, also when it accumulates into an earlier result.  Four
    copies: split-fp16 (split-bf16 is refused below 16 copies, here as elsewhere)."""
    circ = sim.sim_build_circuit(4, 4, 9, 0, 2)
    plan, c, copies, nu, nl = sim.sim_cut_ex(circ, 2, output_phase_cuts=True)
    try:
        assert c == 2
        h = sim.sim_evolve_halves(plan, sim.SIM_C64, 0, copies)
        ref = torch.zeros((1 << nl, 1 << nu), dtype=torch.complex64, device="cuda")
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, ref)
        got = torch.zeros_like(ref)
        sim.sim_amplitudes_noalloc(h, sim.SIM_SPLIT_FP16, False, got)
        assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL
        sim.sim_amplitudes_noalloc(h, sim.SIM_SPLIT_FP16, True, got)
        assert rel(got.cpu().numpy(), 2 * ref.cpu().numpy()) <= TOL
        with pytest.raises(sim.SimError) as e:
            sim.sim_amplitudes_noalloc(h, sim.SIM_SPLIT_BF16, False, got)
        assert e.value.code == sim.SIM_EUNSUPPORTED
        sim.sim_destroy_halves(h)
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)
