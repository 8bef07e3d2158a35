"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* single gates against their mathematical definitions (scipy.linalg.sqrtm of X, Y);
* random small circuits against brute-force 2^n x 2^n Kronecker-product operators;
* closed forms: the H layer gives the uniform state; a circuit of H followed by
  only CZ and T layers has A(x) = 2^{-n/2} w^{m1(x)} (-1)^{m2(x)} (Section 2.4,
  Eqs. 4 and 6), at any size, including selections of 30- and 42-qubit circuits
  through the cut-and-sum;
* invariants: unit norm after every layer; cut-and-sum equals the uncut state
  (Section 2.1, Eq. 1; Supplementary A, Eq. 8); partial sums over copy subsets add up.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import circuit as oc

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Zm = np.diag([1, -1]).astype(complex)
H = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
T = np.diag([1, np.exp(1j * np.pi / 4)])
P0 = np.diag([1, 0]).astype(complex)
P1 = np.diag([0, 1]).astype(complex)
X2 = scipy.linalg.sqrtm(X)
Y2 = scipy.linalg.sqrtm(Y)
MATS = {"H": H, "X2": X2, "Y2": Y2, "T": T, "P0": P0, "P1": P1, "Z": Zm}


def full_operator(n, g):
    """Brute force: the 2^n x 2^n operator of one gate, qubit q = bit q of the index."""
    if g[1] == "CZ":
        d = np.ones(1 << n, dtype=complex)
        for x in range(1 << n):
            if (x >> g[2]) & 1 and (x >> g[3]) & 1:
                d[x] = -1
        return np.diag(d)
    op = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        op = np.kron(op, MATS[g[1]] if q == g[2] else np.eye(2))
    return op


def brute_state(n, gates):
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    for g in gates:
        psi = full_operator(n, g) @ psi
    return psi


def test_sqrt_gates_are_principal_roots():
    assert np.allclose(X2 @ X2, X, atol=1e-14)
    assert np.allclose(Y2 @ Y2, Y, atol=1e-14)
    for m in (H, X2, Y2, T):
        assert np.allclose(m.conj().T @ m, np.eye(2), atol=1e-14)
    # Eq. 1: CZ = P0 (x) I + P1 (x) Z  (first factor on the control qubit)
    cz = np.diag([1, 1, 1, -1]).astype(complex)
    assert np.array_equal(np.kron(P0, np.eye(2)) + np.kron(P1, Zm), cz)


@pytest.mark.parametrize("name", ["H", "X2", "Y2", "T", "P0", "P1", "Z"])
def test_single_gate_columns(name):
    # Apply the gate to each basis state of 3 qubits, on each qubit; compare with kron.
    n = 3
    for q in range(n):
        op = full_operator(n, (0, name, q))
        for x in range(1 << n):
            psi = np.zeros(1 << n, dtype=np.complex128)
            psi[x] = 1
            oracle.apply_gates(psi, n, [(0, name, q)])
            assert np.allclose(psi, op[:, x], atol=1e-15, rtol=0)


def random_gate_list(n, ngates, rng, with_cut_ops=True):
    names = ["H", "X2", "Y2", "T"] + (["CZ"] if n > 1 else []) + (["P0", "P1", "Z"] if with_cut_ops else [])
    gates = []
    for i in range(ngates):
        nm = names[rng.integers(len(names))]
        if nm == "CZ":
            a, b = rng.choice(n, size=2, replace=False)
            gates.append((i, "CZ", int(a), int(b)))
        else:
            gates.append((i, nm, int(rng.integers(n))))
    return gates


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_brute_force_kronecker(n):
    rng = np.random.default_rng(1000 + n)
    for _ in range(4):
        gates = random_gate_list(n, 40, rng)
        ref = brute_state(n, gates)
        got = oracle.statevector(n, gates)
        assert np.max(np.abs(got - ref)) <= 1e-13


def test_brute_force_grid_circuit():
    # A generated 4x2 grid circuit of depth 9 against the Kronecker products.
    gates = oc.generate(4, 2, 9, seed=5)
    assert np.max(np.abs(oracle.statevector(8, gates) - brute_state(8, gates))) <= 1e-13


def test_h_layer_uniform():
    for n in (1, 4, 12):
        psi = oracle.statevector(n, [(0, "H", q) for q in range(n)])
        assert np.max(np.abs(psi - 2.0 ** (-n / 2))) <= 1e-15


def test_unit_norm_each_layer():
    R, C, depth = 4, 4, 17
    gates = oc.generate(R, C, depth, seed=3)
    psi = np.zeros(1 << 16, dtype=np.complex128)
    psi[0] = 1
    for t in range(depth):
        oracle.apply_gates(psi, 16, [g for g in gates if g[0] == t])
        assert abs(np.vdot(psi, psi).real - 1.0) <= 1e-13


def omega_phase(m1, m2):
    return np.exp(1j * np.pi / 4 * m1) * (-1.0) ** m2


def diagonal_closed_form(n, xs, t_sets, cz_sets):
    """A(x) for H on all, then layers of T gates and CZ gates: 2^{-n/2} w^{m1} (-1)^{m2}."""
    out = np.empty(len(xs), dtype=complex)
    for i, x in enumerate(xs):
        x = int(x)
        m1 = sum((x >> q) & 1 for ts in t_sets for q in ts)
        m2 = sum(((x >> a) & 1) & ((x >> b) & 1) for cz in cz_sets for (a, b) in cz)
        out[i] = 2.0 ** (-n / 2) * omega_phase(m1, m2)
    return out


def diagonal_grid_circuit(R, C, depth, b):
    """H layer, then the CZ patterns of a grid, with a T on every qubit idle in odd layers."""
    n = R * C
    gates = [(0, "H", q) for q in range(n)]
    t_sets, cz_sets = [], []
    for t in range(1, depth):
        pairs = oc.pattern_couplers(R, C, b, oc.pattern_of_layer(t))
        busy = {q for p in pairs for q in p}
        cz_sets.append(pairs)
        gates += [(t, "CZ", a, c) for (a, c) in pairs]
        if t % 2 == 1:
            ts = [q for q in range(n) if q not in busy]
            t_sets.append(ts)
            gates += [(t, "T", q) for q in ts]
    return gates, t_sets, cz_sets


def test_closed_form_diagonal_full():
    R, C, depth, b = 4, 4, 12, 2
    gates, ts, cz = diagonal_grid_circuit(R, C, depth, b)
    psi = oracle.statevector(16, gates)
    xs = np.arange(1 << 16)
    ref = diagonal_closed_form(16, xs[::97], ts, cz)
    assert np.max(np.abs(psi[::97] - ref)) <= 1e-14
    # and through the cut: this circuit crosses the cut at layers 7 and 8 (c = 4)
    plan = oc.CutPlan(16, 8, gates)
    assert plan.c == 4
    amp = oracle.cut_amplitudes(plan).reshape(-1)
    assert np.max(np.abs(amp - psi)) <= 1e-14


@pytest.mark.parametrize("R,C,b,depth", [(6, 5, 3, 17), (6, 7, 3, 17)])
def test_closed_form_diagonal_large_selection(R, C, b, depth):
    """30 and 42 qubits: cut-and-sum on a few selected amplitudes vs the closed form."""
    n = R * C
    gates, ts, cz = diagonal_grid_circuit(R, C, depth, b)
    plan = oc.CutPlan(n, b * C, gates)
    rng = np.random.default_rng(7)
    su = np.sort(rng.choice(1 << plan.n_u, 3, replace=False)).astype(np.uint64)
    sl = np.sort(rng.choice(1 << plan.n_l, 2, replace=False)).astype(np.uint64)
    # the full sum over 2^c copies is too slow for a CPU test at c = 14; the
    # diagonal circuit only needs the copies whose projectors keep x_u, which is
    # exactly one copy per x_u-bit pattern.  Sum over all copies for c <= 8.
    if plan.c <= 8:
        amp = oracle.cut_amplitudes(plan, su, sl)
    else:
        amp = np.zeros((sl.size, su.size), dtype=np.complex128)
        for i, xu in enumerate(su):
            k = 0
            for m, (_t, h, _k) in enumerate(plan.cuts):
                k |= ((int(xu) >> h) & 1) << m
            part = oracle.cut_amplitudes(plan, su[i:i + 1], sl, k, k + 1)
            amp[:, i] = part[:, 0]
    xs = [int(xu) + (int(xl) << plan.n_u) for xl in sl for xu in su]
    ref = diagonal_closed_form(n, xs, ts, cz).reshape(sl.size, su.size)
    assert np.max(np.abs(amp - ref)) <= 1e-13 * 2.0 ** (-n / 2) * 64 + 1e-300


@pytest.mark.parametrize("R,C,depth,seed", [(4, 4, 10, 0), (4, 4, 17, 1), (4, 5, 16, 2), (6, 3, 17, 3)])
def test_cut_equals_uncut(R, C, depth, seed):
    b = R // 2
    gates, plan = oc.grid_cut(R, C, depth, seed, b)
    n = R * C
    psi = oracle.statevector(n, gates)
    amp = oracle.cut_amplitudes(plan).reshape(-1)
    assert plan.c > 0
    assert np.max(np.abs(amp - psi)) <= 1e-12 * np.max(np.abs(psi))


def test_partial_sums_add_up():
    gates, plan = oc.grid_cut(4, 4, 17, 4)
    full = oracle.cut_amplitudes(plan)
    mid = plan.copies // 3
    a = oracle.cut_amplitudes(plan, k_begin=0, k_end=mid)
    oracle.cut_amplitudes(plan, k_begin=mid, k_end=plan.copies, out=a)
    assert np.max(np.abs(a - full)) <= 1e-15


def test_half_state_matches_cut_sum_per_copy():
    gates, plan = oc.grid_cut(4, 4, 10, 0)
    for k in (0, 5, plan.copies - 1):
        u = oracle.half_state(plan, 0, k)
        lo = oracle.half_state(plan, 1, k)
        part = oracle.cut_amplitudes(plan, k_begin=k, k_end=k + 1)
        assert np.max(np.abs(part - np.outer(lo, u))) <= 1e-16
    # P_l projections keep only amplitudes whose cut bits equal l, right after
    # the last cut layer (for cuts of that layer; gates of later layers mix a projected qubit again)
    last = max(t for (t, _h, _k) in plan.cuts)
    plan8 = oc.CutPlan(16, 8, [g for g in gates if g[0] <= last])
    for k in range(plan8.copies):
        u = oracle.half_state(plan8, 0, k)
        idx = np.arange(u.size)
        for m, (t_m, h, _k2) in enumerate(plan8.cuts):
            if t_m != last:  # single-qubit gates of later layers act on earlier cut qubits
                continue
            assert np.all(u[((idx >> h) & 1) != ((k >> m) & 1)] == 0)
