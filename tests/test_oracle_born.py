"""Pins of the oracle's Born-rule sampler and cross-entropy statistics (Section 3,
measurement outcomes; Eq. 7), against values that do not come from the oracle:
the published splitmix64 outputs, exact cases (uniform and zero probabilities),
frequencies against the probabilities of a small distribution, and the exact
moments of a random circuit's output distribution."""
import math

import numpy as np
import pytest

import oracle
from oracle import circuit as oc


def test_counter_stream_is_the_published_splitmix64():
    # splitmix64 seeded with 1234567: first outputs of the published reference generator
    got = [int(x) for x in oracle.splitmix64_at(1234567, [0, 1, 2])]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    # counter c of the stream is the c-th output of the sequential generator
    r = oc.SplitMix64(99)
    seq = [r.next() for _ in range(1000)]
    assert [int(x) for x in oracle.splitmix64_at(99, np.arange(1000))] == seq


def test_proposal_mapping():
    """i_c = r_{2c} mod count, u_c = (r_{2c+1} >> 11) 2^-53, from the sequential stream."""
    r = oc.SplitMix64(5)
    seq = [r.next() for _ in range(40)]
    i, u = oracle.born_proposals(5, 1000, 0, 20)
    assert [int(x) for x in i] == [seq[2 * c] % 1000 for c in range(20)]
    assert list(u) == [(seq[2 * c + 1] >> 11) * 2.0 ** -53 for c in range(20)]
    assert (u >= 0).all() and (u < 1).all()


def test_uniform_block_accepts_every_proposal():
    """|A|^2 equal everywhere: u * p_max < p holds for every u < 1, so the samples are
    the proposals in order; the statistics are exactly (0, gamma)."""
    n = 10
    amps = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    idx, ords, pmax = oracle.born_sample(amps, 7, 500, 10_000)
    i, u = oracle.born_proposals(7, 1 << n, 0, 500)
    assert np.array_equal(ords, np.arange(500, dtype=np.uint64)) and np.array_equal(idx, i)
    lin, lg = oracle.cross_entropy(np.abs(amps[idx.astype(np.int64)]) ** 2, n)
    assert lin == 0.0 and abs(lg - oracle.EULER_GAMMA) < 1e-15


def test_frequencies_follow_the_probabilities():
    """A distribution with an exact zero: that entry is never drawn, and the sample
    frequencies match p within 5 standard deviations."""
    p = np.arange(8, dtype=np.float64) / 28.0
    amps = np.sqrt(p) * np.exp(1j * np.arange(8))
    S = 200_000
    idx, ords, pmax = oracle.born_sample(amps, 3, S, 10 * S)
    assert idx.size == S and pmax == pytest.approx(7 / 28)
    freq = np.bincount(idx.astype(np.int64), minlength=8) / S
    assert freq[0] == 0.0
    sigma = np.sqrt(p * (1 - p) / S)
    assert np.all(np.abs(freq - p) <= 5 * sigma + 1e-12)
    # acceptance rate = mean(p) / p_max = (1/8) / (7/28)
    assert ords[-1] + 1 == pytest.approx(S / (0.125 / 0.25), rel=0.02)


def test_random_circuit_cross_entropy_matches_exact_moments():
    """Born samples of a 16-qubit random circuit: the sample means of w and ln w
    (w = 2^n p) against their exact expectations over the state, sum_x p w and
    sum_x p ln w, within 5 standard errors; both near the Eq. 7 values (2, 1 - gamma)."""
    n = 16
    gates, plan = oc.grid_cut(4, 4, 20, 11, 2)
    psi = oracle.statevector(n, gates)
    p = np.abs(psi) ** 2
    w = p * 2.0 ** n
    S = 100_000
    idx, ords, pmax = oracle.born_sample(psi, 17, S, 100 * S)
    ws = w[idx.astype(np.int64)]
    lin, lg = oracle.cross_entropy(p[idx.astype(np.int64)], n)
    e_w = float(np.sum(p * w))
    pos = p > 0
    e_lnw = float(np.sum(p[pos] * np.log(w[pos])))
    sd_w = math.sqrt(float(np.sum(p * (w - e_w) ** 2)) / S)
    sd_lnw = math.sqrt(float(np.sum(p[pos] * (np.log(w[pos]) - e_lnw) ** 2)) / S)
    assert abs((lin + 1) - e_w) <= 5 * sd_w
    assert abs((lg - oracle.EULER_GAMMA) - e_lnw) <= 5 * sd_lnw
    assert abs(e_w - 2.0) < 0.1 and abs(e_lnw - (1 - oracle.EULER_GAMMA)) < 0.1
