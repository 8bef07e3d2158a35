"""Pins of the oracle's controlled-X gate and controlled-X cuts (Supplementary A,
Eq. 1 with U = X: CX = P0 (x) I + P1 (x) X), against brute-force Kronecker
products and the uncut state vector."""
import numpy as np

import oracle
from oracle import circuit as oc
from circuits import cx_cut_circuit

I2 = np.eye(2)
X = np.array([[0, 1], [1, 0]], dtype=complex)
P0 = np.diag([1.0, 0.0])
P1 = np.diag([0.0, 1.0])


def op_on(n, q, m):
    """2^n x 2^n operator of a single-qubit matrix m on qubit q (little endian:
    qubit q is bit q of the index, so it is the q-th factor from the right)."""
    out = np.eye(1)
    for p in reversed(range(n)):
        out = np.kron(out, m if p == q else I2)
    return out


def cx_matrix(n, qc, qt):
    return op_on(n, qc, P0) + op_on(n, qc, P1) @ op_on(n, qt, X)


def test_cx_decomposition_identity():
    # CX on (control 0, target 1) as a 4 x 4 matrix: |c t> -> |c, t xor c>
    m = np.zeros((4, 4))
    for i in range(4):
        c, t = i & 1, (i >> 1) & 1
        m[c | ((t ^ c) << 1), i] = 1
    assert np.array_equal(cx_matrix(2, 0, 1), m)
    assert np.array_equal(cx_matrix(2, 1, 0) @ cx_matrix(2, 1, 0), np.eye(4))


def test_cx_against_kronecker_products():
    n = 5
    rng = np.random.default_rng(3)
    gates = [(0, "H", q) for q in range(n)]
    u = np.eye(1 << n, dtype=complex)
    for g in gates:
        u = op_on(n, g[2], np.array([[1, 1], [1, -1]]) / np.sqrt(2)) @ u
    for t in range(1, 9):
        qc, qt = (int(v) for v in rng.choice(n, 2, replace=False))
        gates.append((t, "CX", qc, qt))
        u = cx_matrix(n, qc, qt) @ u
        q = int(rng.integers(n))
        gates.append((t, "T", q))
        u = op_on(n, q, np.diag([1, (1 + 1j) / np.sqrt(2)])) @ u
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[0] = 1
    assert np.max(np.abs(oracle.statevector(n, gates) - u @ psi0)) < 1e-13


def test_cut_equals_uncut_with_controlled_x_cuts():
    for seed in (0, 1, 2):
        R, C, b, depth, gates = cx_cut_circuit(seed)
        n, n_u = R * C, b * C
        plan = oc.CutPlan(n, n_u, gates)
        n_cx = sum(1 for g in gates if g[1] == "CX")
        n_cz_cross = sum(1 for g in gates if g[1] == "CZ" and min(g[2], g[3]) < n_u <= max(g[2], g[3]))
        assert n_cx > 0 and plan.c == n_cx + n_cz_cross
        assert any(g[1] == "CUTX" for g in plan.lower) and any(g[1] == "CUTX" for g in plan.upper)
        ref = oracle.statevector(n, gates).reshape(1 << (n - n_u), 1 << n_u)
        got = oracle.cut_amplitudes(plan)
        assert np.max(np.abs(got - ref)) < 1e-12
