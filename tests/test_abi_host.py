"""CPU tests of the C-ABI library: it loads, exports every symbol include/sim.h
declares, and its host logic (circuit generator, gate-list text, cut planner,
copy-tree schedule, amplitude selection, argument checks) agrees with the
independent oracle implementation, bit for bit where the work is integer."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1802_06952_gb300 import build
    build.build()
    sim.lib()


def test_exports_match_header():
    hdr = open(os.path.join(ROOT, "include", "sim.h")).read()
    declared = set(re.findall(r"\b(sim_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(sim.EXPORTS)
    for name in declared:
        assert hasattr(sim.lib(), name), name


@pytest.mark.parametrize("R,C,d,seed", [(4, 4, 10, 0), (6, 5, 16, 0), (6, 5, 16, 3), (6, 7, 22, 0),
                                        (8, 8, 22, 0), (4, 2, 9, 5), (3, 5, 31, 77), (8, 7, 40, 2)])
def test_generator_text_equals_oracle(R, C, d, seed):
    c = sim.sim_build_circuit(R, C, d, seed)
    try:
        txt = sim.sim_circuit_text(c)
        ref = oc.to_text(R, C, d, seed, oc.generate(R, C, d, seed, R // 2))
        assert txt == ref
        n, depth, ng = sim.sim_circuit_info(c)
        assert (n, depth) == (R * C, d) and ng == len(ref.splitlines()) - 1
    finally:
        sim.sim_destroy_circuit(c)


@pytest.mark.parametrize("R,C,d,seed", [(6, 5, 16, 0), (6, 7, 22, 4), (8, 8, 22, 0)])
def test_t_in_pool_generator_equals_oracle(R, C, d, seed):
    """The T-in-pool gate rule: byte-equal gate lists from both generators; the same
    placement as the default rule (only gate names differ), and about a third of the
    gates after each qubit's first are T."""
    c = sim.sim_build_circuit(R, C, d, seed, 0, None, True)
    try:
        txt = sim.sim_circuit_text(c)
        gates = oc.generate(R, C, d, seed, R // 2, t_in_pool=True)
        assert txt == oc.to_text(R, C, d, seed, gates)
    finally:
        sim.sim_destroy_circuit(c)
    plain = oc.generate(R, C, d, seed, R // 2)
    assert [g[:1] + g[2:] for g in gates] == [g[:1] + g[2:] for g in plain]
    n = R * C
    firsts, later = set(), []
    for g in gates:
        if g[1] in ("X2", "Y2", "T") and g[0] >= 2:
            if g[2] in firsts:
                later.append(g[1])
            else:
                firsts.add(g[2])
                assert g[1] == "T"
    share = later.count("T") / len(later)
    assert abs(share - 1 / 3) < 4 * (2 / 9 / len(later)) ** 0.5 + 0.01


@pytest.mark.parametrize("R,C,d,seed", [(4, 4, 10, 0), (6, 5, 16, 1), (6, 7, 22, 0), (8, 8, 22, 0), (8, 7, 23, 0)])
def test_cut_list_equals_oracle(R, C, d, seed):
    gates, plan = oc.grid_cut(R, C, d, seed, R // 2)
    c = sim.sim_build_circuit(R, C, d, seed)
    p, ncut, copies, nu, nl = sim.sim_cut(c, R // 2)
    try:
        assert ncut == plan.c and copies == plan.copies and (nu, nl) == (plan.n_u, plan.n_l)
        cuts, ne = sim.sim_cut_list(p, ncut)
        assert cuts == [tuple(x) for x in plan.cuts]
        assert ne == plan.n_equivalent()
        for half in (0, 1):
            levels, fused, plain = sim.sim_plan_schedule(p, half)
            assert levels == len(plan.cuts_per_layer()) + 1
            assert 1 <= fused <= plain + levels
    finally:
        sim.sim_destroy_cut(p)
        sim.sim_destroy_circuit(c)


def test_explicit_gate_list_roundtrip():
    gates = oc.generate(4, 5, 12, 9)
    txt = oc.to_text(4, 5, 12, 9, gates)
    c = sim.sim_build_circuit(gate_list=txt)
    try:
        assert sim.sim_circuit_text(c) == txt
    finally:
        sim.sim_destroy_circuit(c)


@pytest.mark.parametrize("bad", [
    "circuit 2 2 3 0\n0 H 0\n0 H 0\n",          # qubit twice in a layer
    "circuit 2 2 3 0\n0 H 9\n",                 # qubit out of range
    "circuit 2 2 3 0\n1 H 0\n0 H 1\n",          # layers out of order
    "circuit 2 2 3 0\n0 Q 0\n",                 # unknown gate
    "0 H 0\n",                                  # missing header
    "circuit 2 2 3 0\n0 CZ 1 1\n",              # CZ on one qubit
])
def test_malformed_gate_lists_rejected(bad):
    with pytest.raises(sim.SimError) as e:
        sim.sim_build_circuit(gate_list=bad)
    assert e.value.code == sim.SIM_EINVAL and sim.sim_last_error()


def test_bad_shapes_and_cuts():
    with pytest.raises(sim.SimError):
        sim.sim_build_circuit(0, 4, 5, 0)
    with pytest.raises(sim.SimError):
        sim.sim_build_circuit(9, 8, 5, 0)        # 72 qubits
    c = sim.sim_build_circuit(4, 4, 5, 0)
    try:
        with pytest.raises(sim.SimError):
            sim.sim_cut(c, 4)                    # cut on the grid edge
    finally:
        sim.sim_destroy_circuit(c)
    c = sim.sim_build_circuit(2, 17, 3, 0)       # halves of 17 qubits are fine
    p = sim.sim_cut(c, 1)[0]
    sim.sim_destroy_cut(p)
    sim.sim_destroy_circuit(c)
    c = sim.sim_build_circuit(4, 11, 3, 0)       # a 33-qubit half is not
    try:
        with pytest.raises(sim.SimError) as e:
            sim.sim_cut(c, 3)
        assert e.value.code == sim.SIM_EUNSUPPORTED
    finally:
        sim.sim_destroy_circuit(c)


@pytest.mark.parametrize("R,C,d,b", [(4, 4, 10, 2), (6, 5, 16, 3), (6, 7, 22, 3), (8, 8, 22, 4)])
def test_plan_levels_cover_the_copy_bits(R, C, d, b):
    """Levels: root first, copy bits fixed in order up to c, passes adding up to the
    schedule's total; the branch layers are the layers holding cuts."""
    circ = sim.sim_build_circuit(R, C, d, 0, b)
    plan, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        cut_layers = sorted({t for (t, u, l) in sim.sim_cut_list(plan, c)[0]})
        for half in (0, 1):
            lv = sim.sim_plan_levels(plan, half)
            nlev, fused, plain = sim.sim_plan_schedule(plan, half)
            assert lv.shape == (nlev, 4) and lv[:, 3].sum() == fused
            assert lv[0, 0] == -1 and lv[0, 1] == 0 and lv[-1, 2] == c
            assert all(lv[j, 1] == lv[j - 1, 2] for j in range(1, nlev))
            assert list(lv[1:, 0]) == cut_layers[: nlev - 1]
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)



def test_sparse_qubits_of_the_last_levels():
    """The qubits the last copy-tree levels act on non-diagonally (the |Q| of the
    sparse leaf entries): none for the last level when the circuit ends with the
    last cut layer's slots (depth 16: layer 15 is the last), a few at depth 22 (the
    light cone of the layer-16 slots over layers 17-21); never fewer for more
    levels, never more than the half's qubits."""
    for (R, C, d, b), zero in (((6, 5, 16, 3), True), ((8, 8, 22, 4), False), ((6, 7, 22, 3), False)):
        circ = sim.sim_build_circuit(R, C, d, 0, b)
        plan, c, copies, nu, nl = sim.sim_cut(circ, b)
        try:
            for half, n in ((0, nu), (1, nl)):
                J = sim.sim_plan_levels(plan, half).shape[0]
                nq = [sim.sim_plan_sparse_qubits(plan, half, lv) for lv in range(1, J)]
                assert all(0 <= q <= n for q in nq)
                assert all(a <= b2 for a, b2 in zip(nq, nq[1:]))
                assert (nq[0] == 0) == zero
                if not zero:
                    assert nq[0] <= 10
                for bad in (0, J):
                    with pytest.raises(sim.SimError) as e:
                        sim.sim_plan_sparse_qubits(plan, half, bad)
                    assert e.value.code == sim.SIM_EINVAL
        finally:
            sim.sim_destroy_cut(plan)
            sim.sim_destroy_circuit(circ)
        with pytest.raises(sim.SimError):
            sim.sim_plan_sparse_qubits(None, 0, 1)


def test_sparse_depth_rule():
    """The trailing levels the evolve leaves unformed for a selection: the 64-qubit
    2^14-entry selection skips two levels (|Q| = 8 over levels 15 and 16, and
    2^14 * 2^8 <= 2^32 / 8); the 42-qubit one none (2^14 * 2^7 > 2^21 / 8) unless
    forced; never with mode -1 or a selection of every index."""
    cases = (((8, 8, 22, 4), 1 << 14, [2, 2], [2, 2]), ((6, 7, 22, 3), 1 << 14, [0, 0], [2, 2]))
    for (R, C, d, b), n_sel, auto, forced in cases:
        circ = sim.sim_build_circuit(R, C, d, 0, b)
        plan, c, copies, nu, nl = sim.sim_cut(circ, b)
        try:
            assert [sim.sim_plan_sparse_depth(plan, h, n_sel) for h in (0, 1)] == auto
            assert [sim.sim_plan_sparse_depth(plan, h, n_sel, 1) for h in (0, 1)] == forced
            assert [sim.sim_plan_sparse_depth(plan, h, n_sel, -1) for h in (0, 1)] == [0, 0]
            assert sim.sim_plan_sparse_depth(plan, 0, 1 << nu, 1) == 0
            for h, n in ((0, nu), (1, nl)):
                dd = sim.sim_plan_sparse_depth(plan, h, n_sel, 1)
                if dd:
                    assert sim.sim_plan_sparse_qubits(plan, h, dd) <= 10
            with pytest.raises(sim.SimError) as e:
                sim.sim_plan_sparse_depth(plan, 0, n_sel, 2)
            assert e.value.code == sim.SIM_EINVAL
        finally:
            sim.sim_destroy_cut(plan)
            sim.sim_destroy_circuit(circ)


@pytest.mark.parametrize("R,C,d,b,leaf_passes", [(6, 7, 22, 3, 1), (8, 8, 22, 4, 1)])
def test_copy_independent_ops_climb_the_tree(R, C, d, b, leaf_passes):
    """The cut slots are a level's only copy-dependent items and they are diagonal,
    so the ops that commute past them run in the parent level (Sec. 2.3.2's shared
    prefixes extended by commutation).  On the 42- and 64-qubit circuits the leaf
    level (2^c nodes per half) keeps one fused pass, and the work weighted by node
    count stays below the plain layer-by-layer tree's."""
    circ = sim.sim_build_circuit(R, C, d, 0, b)
    plan, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        for half in (0, 1):
            lv = sim.sim_plan_levels(plan, half)
            assert lv[-1, 3] == leaf_passes
            # node-passes of the full tree: passes x 2^(copy bits fixed by the level)
            weighted = int(sum(int(p) << int(bits) for bits, p in zip(lv[:, 2], lv[:, 3])))
            assert weighted <= (leaf_passes + 1) << c
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(circ)

@pytest.mark.parametrize("name", ["CX", "CT", "CY2"])
def test_controlled_gate_cuts_on_the_host(name):
    """Controlled X, T and Y^1/2 gates across the cut count as cuts (P_l on the
    control, U^l on the target, Supplementary A, Eq. 1); the gate list round-trips
    through the library's parser; the cut list equals the oracle's; a controlled
    gate inside one half is unsupported, and so are multi-part cuts of them."""
    from circuits import cx_cut_circuit
    R, C, b, depth, gates = cx_cut_circuit(1, name)
    txt = oc.to_text(R, C, depth, 0, gates)
    c = sim.sim_build_circuit(gate_list=txt)
    try:
        assert sim.sim_circuit_text(c) == txt
        plan, cc, copies, nu, nl = sim.sim_cut(c, b)
        ref = oc.CutPlan(R * C, b * C, gates)
        assert cc == ref.c and sim.sim_cut_list(plan, cc)[0] == [tuple(x) for x in ref.cuts]
        sim.sim_destroy_cut(plan)
    finally:
        sim.sim_destroy_circuit(c)
    bad = oc.to_text(4, 4, 3, 0, [(0, "H", 0), (1, name, 0, 1)])
    c = sim.sim_build_circuit(gate_list=bad)
    try:
        with pytest.raises(sim.SimError) as e:
            sim.sim_cut(c, 2)
        assert e.value.code == sim.SIM_EUNSUPPORTED
    finally:
        sim.sim_destroy_circuit(c)
    c = sim.sim_build_circuit(gate_list=txt)
    try:
        with pytest.raises(sim.SimError) as e:
            sim.sim_cut_multi(c, [1, 3])
        assert e.value.code == sim.SIM_EUNSUPPORTED
    finally:
        sim.sim_destroy_circuit(c)


def test_bad_batches_rejected_on_the_host():
    """sim_batch_create validates circuits and subset indices before any device work."""
    with pytest.raises(sim.SimError) as e:
        sim.sim_batch_create([(5, 4, 12, 0, 2), (0, 4, 12, 1, 2)])
    assert e.value.code == sim.SIM_EINVAL
    with pytest.raises(sim.SimError) as e:
        sim.sim_batch_create([(5, 4, 12, 0, 2)], subset_idx=np.array([[1, 2, 1 << 20]], dtype=np.uint64))
    assert e.value.code == sim.SIM_EINVAL and "subset" in sim.sim_last_error()
    with pytest.raises(sim.SimError) as e:
        sim.sim_batch_create([(5, 4, 12, 0, 5)])
    assert e.value.code == sim.SIM_EINVAL


def test_bad_copy_lists_rejected_on_the_host():
    """sim_evolve_halves_list validates its list before any device work."""
    c = sim.sim_build_circuit(4, 4, 10, 0)
    plan, cc, copies, nu, nl = sim.sim_cut(c, 2)
    try:
        for bad in ([], [0, 3, 3], [copies], [1, 2, copies + 5]):
            with pytest.raises(sim.SimError) as e:
                sim.sim_evolve_halves_list(plan, sim.SIM_C64, np.array(bad, dtype=np.uint64))
            assert e.value.code == sim.SIM_EINVAL and sim.sim_last_error()
        with pytest.raises(sim.SimError) as e:
            sim.sim_evolve_halves(plan, sim.SIM_C64, 3, 3)
        assert e.value.code == sim.SIM_EINVAL
    finally:
        sim.sim_destroy_cut(plan)
        sim.sim_destroy_circuit(c)


@pytest.mark.parametrize("nqu,nu,nql,nl,seed", [(15, 300, 15, 77, 0), (21, 1 << 10, 21, 1 << 10, 5),
                                                (4, 16, 4, 3, 1), (32, 5, 32, 5, 123)])
def test_select_equals_oracle(nqu, nu, nql, nl, seed):
    su, sl = sim.sim_select(nqu, nu, nql, nl, seed)
    ru, rl = oracle.select(nqu, nu, nql, nl, seed)
    assert np.array_equal(su, ru) and np.array_equal(sl, rl)


def test_cut_invariance_under_gate_order_text():
    # the planner numbers cuts by (layer, upper qubit), whatever order the list uses
    gates = oc.generate(4, 4, 10, 0)
    by_layer = {}
    for g in gates:
        by_layer.setdefault(g[0], []).append(g)
    shuffled = []
    for t in sorted(by_layer):
        shuffled += list(reversed(by_layer[t]))
    txt = oc.to_text(4, 4, 10, 0, shuffled)
    c = sim.sim_build_circuit(gate_list=txt)
    p, ncut, *_ = sim.sim_cut(c, 2)
    try:
        cuts, _ = sim.sim_cut_list(p, ncut)
        assert cuts == [tuple(x) for x in oc.CutPlan(16, 8, gates).cuts]
    finally:
        sim.sim_destroy_cut(p)
        sim.sim_destroy_circuit(c)


def _expected_output_phase_cuts(gates, n_u):
    """Cut CZs (upper < n_u <= lower) with no non-diagonal gate on either qubit at a
    later layer, from the oracle generator's gate list."""
    last = {}
    for g in gates:
        if g[1] not in ("T", "CZ"):
            for q in g[2:]:
                last[q] = max(last.get(q, -1), g[0])
    out, kept = [], []
    for g in gates:
        if g[1] == "CZ":
            a, b = min(g[2], g[3]), max(g[2], g[3])
            if a < n_u <= b:
                if last.get(a, -1) < g[0] and last.get(b, -1) < g[0]:
                    out.append((a, b))
                else:
                    kept.append((g[0], a, b))
    return out, kept


@pytest.mark.parametrize("R,C,d,seed,b", [(6, 5, 16, 0, 3), (6, 5, 16, 3, 3), (4, 4, 9, 0, 2), (4, 4, 10, 0, 2),
                                          (6, 7, 22, 0, 3), (5, 4, 15, 2, 2)])
def test_output_phase_cuts_on_the_host(R, C, d, seed, b):
    """sim_cut_ex(output_phase_cuts): which cut CZs leave the copy index (the rule
    recomputed from the oracle's generator), the remaining cut list in copy-bit order,
    and 2^c; without the option the plan is sim_cut's."""
    gates = oc.generate(R, C, d, seed, b)
    n_u = b * C
    want_out, want_kept = _expected_output_phase_cuts(gates, n_u)
    circ = sim.sim_build_circuit(R, C, d, seed, b)
    try:
        p0, c0, _, _, _ = sim.sim_cut(circ, b)
        p1, c1, copies1, _, _ = sim.sim_cut_ex(circ, b, output_phase_cuts=True)
        p2, c2, _, _, _ = sim.sim_cut_ex(circ, b, output_phase_cuts=False)
        try:
            assert c2 == c0 and sim.sim_cut_output_phases(p0) == [] and sim.sim_cut_output_phases(p2) == []
            assert sorted(sim.sim_cut_output_phases(p1)) == sorted(want_out)
            assert c1 == c0 - len(want_out) and copies1 == 1 << c1
            assert sim.sim_cut_list(p1, c1)[0] == sorted(want_kept)
        finally:
            for p in (p0, p1, p2):
                sim.sim_destroy_cut(p)
    finally:
        sim.sim_destroy_circuit(circ)
    # the 30-qubit workload: the three cuts of its last layer (15) leave, c = 8 -> 5
    if (R, C, d, b) == (6, 5, 16, 3):
        assert len(want_out) == 3 and c1 == 5


def test_output_phase_cuts_rejects_bad_option():
    import ctypes
    circ = sim.sim_build_circuit(4, 4, 9, 0, 2)
    try:
        o = sim.SimCutOpts(2)
        p = ctypes.c_void_p()
        rc = sim.lib().sim_cut_ex(circ, 2, ctypes.byref(o), ctypes.byref(p), None, None, None, None)
        assert rc == sim.SIM_EINVAL and not p.value
    finally:
        sim.sim_destroy_circuit(circ)


@pytest.mark.parametrize("R,C,d,rows", [(6, 3, 12, [2, 4]), (8, 8, 22, [3, 5]), (8, 2, 12, [2, 4, 6]),
                                        (8, 7, 10, [2, 5])])
def test_multi_part_plan_on_the_host(R, C, d, rows):
    """sim_cut_multi: parts and crossing counts against the oracle's multi-part plan."""
    circ = sim.sim_build_circuit(R, C, d, 0, rows[0])
    try:
        plan, t, cs, nq = sim.sim_cut_multi(circ, rows)
        sim.sim_destroy_multi(plan)
        mp = oc.MultiCutPlan(R, C, rows, oc.generate(R, C, d, 0, rows[0]))
        assert t == mp.t and nq == mp.nq and cs == [mp.c(j) for j in range(1, mp.t)]
    finally:
        sim.sim_destroy_circuit(circ)


def test_multi_part_plan_rejects_bad_rows_and_gates():
    circ = sim.sim_build_circuit(6, 3, 12, 1, 2)
    try:
        for rows in ([4, 2], [0, 3], [2, 6], [3, 3]):
            with pytest.raises(sim.SimError) as e:
                sim.sim_cut_multi(circ, rows)
            assert e.value.code == sim.SIM_EINVAL, rows
    finally:
        sim.sim_destroy_circuit(circ)
    from circuits import cx_cut_circuit
    R, C, b, depth, gates = cx_cut_circuit(0)
    circ = sim.sim_build_circuit(gate_list=oc.to_text(R, C, depth, 0, gates))
    try:
        with pytest.raises(sim.SimError) as e:
            sim.sim_cut_multi(circ, [1, 3])
        assert e.value.code == sim.SIM_EUNSUPPORTED
    finally:
        sim.sim_destroy_circuit(circ)


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No CPU fallback: with libsim.so absent, every entry point raises instead of
    computing anything, and the oracle is not reachable from the library package."""
    monkeypatch.setattr(sim, "_lib", None)
    monkeypatch.setattr(sim, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libsim.so"))
    with pytest.raises(RuntimeError):
        sim.lib()
    with pytest.raises(RuntimeError):
        sim.sim_build_circuit(4, 4, 10, 0, 2)
    for name in os.listdir(os.path.join(ROOT, "paper_1802_06952_gb300")):
        if name.endswith(".py"):
            text = open(os.path.join(ROOT, "paper_1802_06952_gb300", name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name
