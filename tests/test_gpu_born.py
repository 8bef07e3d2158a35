"""GPU parity of Born-rule sampling (sim_born_sample) against the oracle's sampler:
the proposal stream is bit-exact, and every accept / reject decision agrees with
the oracle's, except where u * p_max and p differ by less than the amplitude error
allows; the cross-entropy statistics agree within that error."""
import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# p = |A|^2 from amplitudes within 1e-5 of max|A| differs by at most ~2e-5 of p_max
TOL_P = 3e-5


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


@pytest.mark.parametrize("R,C,d,seed,sseed", [(4, 4, 12, 3, 42), (4, 5, 16, 1, 7)])
def test_born_samples_match_oracle(R, C, d, seed, sseed):
    n = R * C
    b = R // 2
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    psi = oracle.statevector(n, gates)
    p_o = np.abs(psi) ** 2
    pmax_o = float(p_o.max())
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    cp, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        h = sim.sim_evolve_halves(cp, sim.SIM_C64, 0, copies)
        out = torch.zeros((1 << nl, 1 << nu), dtype=torch.complex64, device="cuda")
        sim.sim_amplitudes(h, sim.SIM_SPLIT_BF16, False, out)
        sim.sim_status()
        sim.sim_destroy_halves(h)
        S = 20000
        idx, ords, xeb = sim.sim_born_sample(out, n, sseed, S, 50_000_000)
        assert idx.size == S and np.all(np.diff(ords.astype(np.int64)) > 0)
        # proposals: bit-exact indices at the accepted ordinals
        i_all, u_all = oracle.born_proposals(sseed, 1 << n, 0, int(ords[-1]) + 1)
        assert np.array_equal(i_all[ords.astype(np.int64)], idx)
        # decisions over every proposal up to the last accepted one
        gap = u_all * pmax_o - p_o[i_all.astype(np.int64)]
        acc_gpu = np.zeros(i_all.size, dtype=bool)
        acc_gpu[ords.astype(np.int64)] = True
        acc_orc = gap < 0
        differ = acc_gpu != acc_orc
        assert np.all(np.abs(gap[differ]) <= TOL_P * pmax_o)
        assert differ.sum() <= max(3, int(1e-4 * i_all.size))
        # cross-entropy statistics and the measured bound
        lin, lg = oracle.cross_entropy(p_o[idx.astype(np.int64)], n)
        assert abs(xeb[0] - lin) < 1e-4 and abs(xeb[1] - lg) < 1e-4
        assert abs(xeb[2] - pmax_o * 2.0 ** n) <= 3e-5 * pmax_o * 2.0 ** n
        # Born samples of these circuits: both statistics near 1 (Eq. 7)
        assert 0.7 < xeb[0] < 1.3 and 0.7 < xeb[1] < 1.3
    finally:
        sim.sim_destroy_cut(cp)
        sim.sim_destroy_circuit(circ)


def test_born_sample_arguments():
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(sim.SimError):
        sim.sim_born_sample(x, 4, 0, 0, 100)
    # all-zero block: no sample, bound 0
    idx, ords, xeb = sim.sim_born_sample(x, 4, 0, 10, 1000)
    assert idx.size == 0 and xeb[2] == 0.0
