"""Randomized GPU parity (fixed seed, so deterministic): random small grids, depths,
circuit seeds, cut rows, fuse widths, sweep kernels, pass formations and the
output-phase option, half of them with controlled X, T and Y^1/2 gates across the
cut added (Supplementary A, Eq. 1), each full vector against the oracle's uncut
state vector.

Tolerances: split fp16 and split bf16 <= 1e-5, FP64 plain <= 1e-12.  Split bf16 is
refused (SIM_EUNSUPPORTED) below 16 copies, where too few products average its
per-product error 3 * 2^-16 below 1e-5; that refusal is checked too."""
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


def cases(count=120, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        R, C = int(rng.integers(2, 6)), int(rng.integers(1, 6))
        n = R * C
        if n < 4 or n > 20:
            continue
        b = int(rng.integers(1, R))
        d = int(rng.integers(3, 26))
        out.append((R, C, d, int(rng.integers(0, 10 ** 6)), b, int(rng.integers(4, 14)), int(rng.integers(0, 3)),
                    int(rng.integers(0, 2)), bool(rng.integers(0, 2)), bool(rng.integers(0, 2))))
    return out


@pytest.mark.parametrize("R,C,d,seed,b,fuse,kernel,order,phase,cu", cases())
def test_random_circuit_full_vector(R, C, d, seed, b, fuse, kernel, order, phase, cu):
    if cu:
        from circuits import with_cross_controlled
        gates = with_cross_controlled(R, C, d, seed, b, np.random.default_rng(seed))
        circ = sim.sim_build_circuit(gate_list=oc.to_text(R, C, d, seed, gates))
    else:
        gates = oc.generate(R, C, d, seed, b)
        circ = sim.sim_build_circuit(R, C, d, seed, b)
    ref = oracle.statevector(R * C, gates).reshape(1 << ((R - b) * C), 1 << (b * C))
    plan, c, copies, nu, nl = sim.sim_cut_ex(circ, b, output_phase_cuts=phase)
    opts = {"fuse_qubits": fuse, "sweep_kernel": kernel, "pass_order": order}
    try:
        for prec, kind in ((sim.SIM_C64, sim.SIM_SPLIT_FP16), (sim.SIM_C64, sim.SIM_SPLIT_BF16),
                           (sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN)):
            h = sim.sim_evolve_halves(plan, prec, 0, copies, opts=opts)
            dt = torch.complex128 if kind == sim.SIM_FP64_PLAIN else torch.complex64
            out = torch.zeros((1 << nl, 1 << nu), dtype=dt, device="cuda")
            try:
                if kind == sim.SIM_SPLIT_BF16 and copies < 16:
                    with pytest.raises(sim.SimError) as ei:
                        sim.sim_amplitudes(h, kind, False, out)
                    assert ei.value.code == sim.SIM_EUNSUPPORTED
                    continue
                sim.sim_amplitudes(h, kind, False, out)
                sim.sim_status()
            finally:
                sim.sim_destroy_halves(h)
            tol = 1e-12 if kind == sim.SIM_FP64_PLAIN else 1e-5
            assert rel_err(out.cpu().numpy(), ref) <= tol, (kind, c)
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)
