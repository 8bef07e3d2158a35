"""Pins of the oracle's circuit generator and cut plan against counts printed in the
paper (tests/golden/paper_counts.txt: Table 2, Fig. 4 and Fig. 3 captions, Fig. 1 /
Sections 2.1, 3) and the partition ordering Section 3 states for Fig. 3,
plus the generator's structural invariants (Supplementary A, Eq. 3)."""
import numpy as np
import pytest

import oracle
from oracle import circuit as oc
from conftest import golden_rows


@pytest.mark.parametrize("row", golden_rows("table2"))
def test_table2_cut_counts(row):
    paper_depth, in_layer, total, n_e = row
    gates, plan = oc.grid_cut(8, 7, paper_depth + 1, seed=0, b=4)
    per = plan.cuts_per_layer()
    assert per.get(paper_depth, 0) == in_layer
    assert plan.c == total
    assert plan.n_equivalent() == n_e


@pytest.mark.parametrize("row", golden_rows("fig4"))
def test_fig4_cz_totals(row):
    R, C, total = row
    for seed in (0, 1):
        gates = oc.generate(R, C, 22 + 1, seed, R // 2)
        assert sum(1 for g in gates if g[1] == "CZ") == total


def test_fig1_example():
    (R, C, depth, c, copies, halves, qh, n_e), = golden_rows("fig1")
    gates, plan = oc.grid_cut(R, C, depth + 1, seed=0, b=R // 2)
    assert plan.c == c and plan.copies == copies
    assert 2 * plan.copies == halves and plan.n_u == qh and plan.n_l == qh
    assert plan.n_equivalent() == n_e
    assert sorted(plan.cuts_per_layer()) == [7, 8]


def test_fig3_two_part_equivalent_qubits():
    (R, C, paper_depth, n_e), = golden_rows("fig3")
    gates, plan = oc.grid_cut(R, C, paper_depth + 1, seed=0, b=R // 2)
    assert plan.n_equivalent() == n_e


def test_fig3_partition_ordering():
    """Section 3 / Fig. 3: with the complexity of a partition counted as its largest
    part plus its transformed CZs, three or four parts are no worse than two at small
    depth, and two parts are best at depths around 22 and 30.  Fig. 3c's three-part
    split of the 64-qubit circuit has 24 qubits in its largest part."""
    R = C = 8

    def cost(d):
        g2 = oc.generate(R, C, d + 1, 0, 4)
        two = 32 + oc.CutPlan(64, 32, g2).c
        m3 = oc.MultiCutPlan(R, C, [3, 5], oc.generate(R, C, d + 1, 0, 3))
        m4 = oc.MultiCutPlan(R, C, [2, 4, 6], oc.generate(R, C, d + 1, 0, 2))
        return two, max(m3.nq) + m3.c_total, max(m4.nq) + m4.c_total, m3

    for d in (6, 8, 10, 12):
        two, three, four, _ = cost(d)
        assert three <= two and four <= two
    for d in (22, 30):
        two, three, four, m3 = cost(d)
        assert two < three and two < four
        assert max(m3.nq) == 24


@pytest.mark.parametrize("R,C,d,c", [(4, 4, 10, 4), (6, 5, 16, 8), (6, 7, 22, 14), (8, 8, 22, 16)])
def test_config_cut_counts(R, C, d, c):
    _, plan = oc.grid_cut(R, C, d, 0, R // 2)
    assert plan.c == c


@pytest.mark.parametrize("R,C,d,seed", [(4, 4, 10, 0), (6, 5, 16, 3), (8, 8, 22, 9)])
def test_generator_invariants(R, C, d, seed):
    gates = oc.generate(R, C, d, seed, R // 2)
    n = R * C
    first = {}
    for t in range(d):
        layer = [g for g in gates if g[0] == t]
        used = []
        for g in layer:
            used += list(g[2:])
        assert len(used) == len(set(used)), "qubit used twice in a layer"
        if t == 0:
            assert sorted(g[2] for g in layer) == list(range(n)) and all(g[1] == "H" for g in layer)
        if t == 1:
            assert all(g[1] == "CZ" for g in layer)
        for g in layer:
            if g[1] in ("T", "X2", "Y2"):
                q = g[2]
                assert (g[1] == "T") == (q not in first)
                first.setdefault(q, t)
                prev = {x for h in gates if h[0] == t - 1 and h[1] == "CZ" for x in h[2:]}
                assert q in prev
    # every vertical and horizontal coupler is used once per 8 cycles
    allc = [tuple(sorted(g[2:])) for g in gates if g[1] == "CZ" and 1 <= g[0] <= 8]
    ncoup = R * (C - 1) + (R - 1) * C
    if d > 8:
        assert len(allc) == len(set(allc)) == ncoup


def test_text_roundtrip():
    gates = oc.generate(4, 5, 12, 7)
    txt = oc.to_text(4, 5, 12, 7, gates)
    R, C, d, s, g2 = oc.parse_text(txt)
    assert (R, C, d, s) == (4, 5, 12, 7) and g2 == gates


def test_splitmix64_published_vector():
    # splitmix64 seeded with 1234567: first outputs of the published reference generator.
    r = oc.SplitMix64(1234567)
    got = [r.next() for _ in range(3)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_floyd_select_distinct_sorted_uniform():
    su, sl = oracle.select(10, 300, 4, 16, seed=11)
    assert su.size == 300 and np.all(np.diff(su.astype(np.int64)) > 0) and su.max() < 1024
    assert np.array_equal(sl, np.arange(16))
    # uniformity: each element of a 16-set drawn 4-at-a-time appears with p = 1/4
    counts = np.zeros(16)
    trials = 4000
    for s in range(trials):
        a, _ = oracle.select(4, 4, 1, 1, seed=s)
        counts[a.astype(np.int64)] += 1
    expect = trials * 4 / 16
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 40.0  # 15 dof; p ~ 5e-4


def test_eq7_cdf_is_the_integral_of_the_density():
    """Eq. 7: f(z) = (1/a) exp(z - (1/a)(e^z + a - 1)); at a = 1 its CDF is the
    closed form the statistics use, and u = F(z) of an Exp(1) w = e^z is uniform."""
    from scipy.integrate import quad
    alpha = 1.0
    f = lambda z: (1 / alpha) * np.exp(z - (1 / alpha) * (np.exp(z) + alpha - 1))
    for z0 in (-6.0, -1.0, 0.0, 0.7, 2.0):
        val, _ = quad(f, -60, z0)
        assert abs(val - oracle.gumbel_cdf(z0)) < 1e-10
    rng = np.random.default_rng(5)
    w = rng.exponential(size=200000)
    u = oracle.gumbel_cdf(np.log(w))
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002


def test_stats_closed_forms():
    # Porter-Thomas: 2^n|A|^2 ~ Exp(1): mean 1, mean ln = -Euler gamma, KS small
    rng = np.random.default_rng(0)
    n = 18
    a = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) / np.sqrt(2 * (1 << n))
    st, hist = oracle.stats(a, n)
    assert abs(st[1] - 1) < 0.01 and abs(st[2] + np.euler_gamma) < 0.01 and st[3] < 0.01
    assert hist.sum() == a.size
    # uniform vector: every z = 0, so KS = max |1[z>=0] - F| ~ F(0) = 1 - 1/e
    u = np.full(1 << 10, 2.0 ** -5, dtype=complex)
    st2, _ = oracle.stats(u, 10)
    assert abs(st2[0] - 1) < 1e-12 and abs(st2[2]) < 1e-12
    assert abs(st2[3] - (1 - np.exp(-1))) < 0.01
