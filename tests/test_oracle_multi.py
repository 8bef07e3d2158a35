"""Pins of the oracle's multi-part cut-and-sum (Section 3, Fig. 3: the grid cut into
three or four row bands, every crossing CZ rewritten by Eq. 1), against facts that
do not come from it: the uncut state vector (the rewrite is an identity), the
two-part cut-and-sum of Supplementary A, Eq. 8 as the special case, brute-force
counts of the crossing CZs, and the bijection of each part's copy index."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import circuit as oc


@pytest.mark.parametrize("R,C,d,seed,rows", [(6, 3, 12, 1, [2, 4]), (6, 3, 16, 4, [1, 3]), (5, 3, 14, 2, [2, 3]),
                                              (8, 2, 12, 0, [2, 4, 6]), (4, 4, 10, 3, [1, 2, 3])])
def test_multi_part_equals_uncut(R, C, d, seed, rows):
    gates = oc.generate(R, C, d, seed, rows[0])
    mp = oc.MultiCutPlan(R, C, rows, gates)
    assert mp.t == len(rows) + 1 and sum(mp.nq) == R * C
    ref = oracle.statevector(R * C, gates)
    got = oracle.multi_cut_amplitudes(mp).reshape(-1)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_two_parts_is_the_half_cut():
    R, C, d, seed, b = 4, 4, 10, 0, 2
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    mp = oc.MultiCutPlan(R, C, [b], gates)
    assert mp.c(1) == plan.c == 4
    got = oracle.multi_cut_amplitudes(mp)
    ref = oracle.cut_amplitudes(plan)
    assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("R,C,d,rows", [(8, 8, 22, [3, 5]), (8, 8, 22, [2, 4, 6]), (6, 7, 22, [2, 4])])
def test_cut_counts_per_boundary(R, C, d, rows):
    """c_j = CZs with one qubit above row r_j and one below, counted from the gate list."""
    gates = oc.generate(R, C, d, 0, rows[0])
    mp = oc.MultiCutPlan(R, C, rows, gates)
    for j, r in enumerate(rows, start=1):
        brute = sum(1 for g in gates if g[1] == "CZ" and min(g[2], g[3]) < r * C <= max(g[2], g[3]))
        assert mp.c(j) == brute
    assert mp.c_total == sum(mp.c(j) for j in range(1, mp.t))
    # a part's slots are the cuts of the boundaries above and below it
    for p in range(mp.t):
        want = (mp.c(p) if p > 0 else 0) + (mp.c(p + 1) if p < mp.t - 1 else 0)
        assert mp.part_bits(p) == want


def test_part_index_is_a_bijection():
    gates = oc.generate(8, 2, 16, 5, 2)
    mp = oc.MultiCutPlan(8, 2, [2, 4, 6], gates)
    for p in range(mp.t):
        na = 1 << mp.c(p) if p > 0 else 1
        nb = 1 << mp.c(p + 1) if p < mp.t - 1 else 1
        ks = {mp.part_index(p, la, lb) for la, lb in itertools.product(range(na), range(nb))}
        assert ks == set(range(1 << mp.part_bits(p)))


def test_selections_index_the_full_result():
    R, C, d, seed, rows = 6, 3, 12, 1, [2, 4]
    gates = oc.generate(R, C, d, seed, rows[0])
    mp = oc.MultiCutPlan(R, C, rows, gates)
    full = oracle.multi_cut_amplitudes(mp)           # [n2, n1, n0]
    rng = np.random.default_rng(0)
    sels = [np.sort(rng.permutation(1 << q)[:k]) for q, k in zip(mp.nq, (5, 7, 3))]
    got = oracle.multi_cut_amplitudes(mp, sels)
    want = full[np.ix_(sels[2], sels[1], sels[0])]
    assert np.max(np.abs(got - want)) < 1e-15
