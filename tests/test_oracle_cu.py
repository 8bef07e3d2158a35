"""Pins of the oracle's controlled T and controlled Y^1/2 gates and of their cuts
(Supplementary A, Eq. 1: CU = P0 (x) I + P1 (x) U with U = T or Y^1/2), against
brute-force Kronecker products built from scipy's matrix square root and the
uncut state vector.  Also the identities the library's fused sweeps use to write
U^l with copy-independent gates around a diagonal slot."""
import numpy as np
import pytest
from scipy.linalg import sqrtm

import oracle
from oracle import circuit as oc
from circuits import cx_cut_circuit

I2 = np.eye(2)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
P0 = np.diag([1.0, 0.0])
P1 = np.diag([0.0, 1.0])
T = np.diag([1.0, np.exp(1j * np.pi / 4)])
S = np.diag([1.0, 1j])
X2 = sqrtm(X)
Y2 = sqrtm(Y)
U_OF = {"CT": T, "CY2": Y2}


def op_on(n, q, m):
    """2^n x 2^n operator of a single-qubit matrix m on qubit q (qubit q = bit q)."""
    out = np.eye(1)
    for p in reversed(range(n)):
        out = np.kron(out, m if p == q else I2)
    return out


def cu_matrix(n, qc, qt, u):
    return op_on(n, qc, P0) + op_on(n, qc, P1) @ op_on(n, qt, u)


def test_principal_square_roots():
    # the gate set's Y^1/2 is the principal square root the oracle hard-codes
    assert np.allclose(Y2 @ Y2, Y) and np.allclose(Y2, 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]]))


@pytest.mark.parametrize("name", ["CT", "CY2"])
def test_controlled_u_against_kronecker_products(name):
    n = 5
    rng = np.random.default_rng(7 if name == "CT" else 8)
    gates = [(0, "H", q) for q in range(n)]
    u = np.eye(1 << n, dtype=complex)
    for g in gates:
        u = op_on(n, g[2], np.array([[1, 1], [1, -1]]) / np.sqrt(2)) @ u
    for t in range(1, 10):
        qc, qt = (int(v) for v in rng.choice(n, 2, replace=False))
        gates.append((t, name, qc, qt))
        u = cu_matrix(n, qc, qt, U_OF[name]) @ u
        q = int(rng.integers(n))
        if q not in (qc, qt):
            gates.append((t, "X2", q))
            u = op_on(n, q, X2) @ u
    psi0 = np.zeros(1 << n, dtype=complex)
    psi0[0] = 1
    assert np.max(np.abs(oracle.statevector(n, gates) - u @ psi0)) < 1e-13


@pytest.mark.parametrize("name", ["CT", "CY2"])
def test_cut_equals_uncut_with_controlled_u_cuts(name):
    for seed in (0, 1, 2):
        R, C, b, depth, gates = cx_cut_circuit(seed, name)
        n, n_u = R * C, b * C
        plan = oc.CutPlan(n, n_u, gates)
        n_cu = sum(1 for g in gates if g[1] == name)
        n_cz_cross = sum(1 for g in gates if g[1] == "CZ" and min(g[2], g[3]) < n_u <= max(g[2], g[3]))
        assert n_cu > 0 and plan.c == n_cu + n_cz_cross
        assert any(g[1] == "CUTU" for g in plan.lower) and any(g[1] == "CUTU" for g in plan.upper)
        ref = oracle.statevector(n, gates).reshape(1 << (n - n_u), 1 << n_u)
        got = oracle.cut_amplitudes(plan)
        assert np.max(np.abs(got - ref)) < 1e-12
        # the copy with every bit set carries U on every cut target, copy 0 none
        u_name = oc.CONTROLLED_U[name]
        k = plan.copies - 1
        n_tgt = sum(1 for h in (0, 1) for g in (plan.upper, plan.lower)[h] if g[1] == "CUTU")
        assert sum(1 for h in (0, 1) for g in plan.half_gates(h, k) if g[1] == u_name) >= n_tgt
        assert sum(1 for h in (0, 1) for g in plan.half_gates(h, 0) if g[1] == u_name) == \
            sum(1 for h in (0, 1) for g in (plan.upper, plan.lower)[h] if g[1] == u_name)


def test_text_round_trip_of_controlled_gates():
    R, C, b, depth, gates = cx_cut_circuit(1, "CY2")
    txt = oc.to_text(R, C, depth, 0, gates)
    assert oc.parse_text(txt)[4] == gates


def test_fused_sweep_identities():
    """The library writes U^l with copy-independent gates of its fused kinds around
    one diagonal copy slot w^{b l x_t} on the target (w = e^{i pi/4}):
    T^l = diag(1, w^l) (b = 1); (Y^1/2)^l = X^1/2 X^1/2 X^1/2 diag(1, i^l) X^1/2
    (b = 2), since (X^1/2)^3 = X^-1/2 and X^-1/2 S X^1/2 = Y^1/2."""
    w = np.exp(1j * np.pi / 4)
    for l in (0, 1):
        assert np.allclose(np.linalg.matrix_power(T, l), np.diag([1, w ** l]))
        slot = np.diag([1, w ** (2 * l)])
        assert np.allclose(X2 @ X2 @ X2 @ slot @ X2, np.linalg.matrix_power(Y2, l))
