"""FP64 CPU oracle for the cut-CZ partition scheme of arXiv 1802.06952.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_1802_06952_gb300``),
and the library never imports it.

Contents
  circuit.py  random grid circuit generator, canonical gate-list text, cut plan
              (Supplementary A, Eqs. 3-8; Section 2.1, Eq. 1), multi-part cut
              plan (Section 3, Fig. 3)
  oracle.c    plain FP64 state-vector evolution (Supplementary A, Eq. 4) and the
              cut-and-sum reconstruction (Supplementary A, Eq. 8)
  this file   ctypes binding, the amplitude selection draw, the FP64
              statistics of Section 3 (Eq. 7), and Born-rule sampling of
              measurement outcomes with the cross-entropy statistics

Parity status: every function here is pinned by tests under ``tests/`` that do
not call the oracle to make their expected values (brute-force Kronecker
products, closed forms, counts printed in the paper, invariants).
"""
import ctypes
import math
import os
import subprocess

import numpy as np

from . import circuit  # noqa: F401
from .circuit import SplitMix64, CutPlan, MultiCutPlan, generate, grid_cut, to_text, parse_text  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

CODES = {"H": 0, "X2": 1, "Y2": 2, "T": 3, "CZ": 4, "P0": 5, "P1": 6, "Z": 7, "CX": 8, "X": 9, "CT": 10, "CY2": 11}


def build(force=False):
    """Compile oracle.c into liboracle.so with gcc (OpenMP, -O2, portable flags)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _SO + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_SO + ".tmp", _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i32p = ctypes.POINTER(ctypes.c_int32)
        dp = ctypes.POINTER(ctypes.c_double)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.or_evolve.argtypes = [ctypes.c_int, i32p, ctypes.c_int, dp, ctypes.c_int]
        L.or_evolve.restype = None
        L.or_cut_sum.argtypes = [ctypes.c_int, i32p, ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
                                 ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_int64, u64p,
                                 ctypes.c_int64, ctypes.c_int, dp]
        L.or_cut_sum.restype = ctypes.c_int
        L.or_half_state.argtypes = [ctypes.c_int, i32p, ctypes.c_int, ctypes.c_uint64, dp]
        L.or_half_state.restype = ctypes.c_int
        L.or_num_threads.argtypes = []
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads():
    return lib().or_num_threads()


def _encode(gates):
    """Gate tuples -> int32 [ngates, 3] {code, q1, q2}; cut slots -> codes -1 / -2 / -3."""
    rows = []
    for g in gates:
        name = g[1]
        if name in ("CZ", "CX", "CT", "CY2"):
            rows.append((CODES[name], g[2], g[3]))
        elif name == "CUTU":
            rows.append((-100 - CODES[g[4]], g[3], g[2]))
        elif name == "CUTP":
            rows.append((-1, g[3], g[2]))
        elif name == "CUTZ":
            rows.append((-2, g[3], g[2]))
        elif name == "CUTX":
            rows.append((-3, g[3], g[2]))
        else:
            rows.append((CODES[name], g[2], 0))
    a = np.asarray(rows if rows else np.zeros((0, 3)), dtype=np.int32).reshape(-1, 3)
    return np.ascontiguousarray(a)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def statevector(n, gates):
    """Uncut state U_{d-1}...U_0 |0...0> (Supplementary A, Eq. 4), gate by gate, FP64."""
    ops = _encode(gates)
    psi = np.zeros(1 << n, dtype=np.complex128)
    lib().or_evolve(n, _ptr(ops, ctypes.c_int32), ops.shape[0], _ptr(psi, ctypes.c_double), 1)
    return psi


def apply_gates(psi, n, gates):
    """Apply a gate list to an existing complex128 state in place (no re-init)."""
    ops = _encode(gates)
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == (1 << n)
    lib().or_evolve(n, _ptr(ops, ctypes.c_int32), ops.shape[0], _ptr(psi, ctypes.c_double), 0)
    return psi


def half_state(plan, half, k):
    """Half-state of copy k: half 0 = upper, half 1 = lower, each with its cut slots."""
    n_h = plan.n_u if half == 0 else plan.n_l
    tmpl = _encode(plan.upper if half == 0 else plan.lower)
    psi = np.zeros(1 << n_h, dtype=np.complex128)
    rc = lib().or_half_state(n_h, _ptr(tmpl, ctypes.c_int32), tmpl.shape[0], k,
                             _ptr(psi, ctypes.c_double))
    assert rc == 0
    return psi


def cut_amplitudes(plan, sel_u=None, sel_l=None, k_begin=0, k_end=None, out=None):
    """Section 2.1 / Supplementary A, Eq. 8: A(x_u, x_l) = sum_k U_k[x_u] L_k[x_l].

    Returns a complex128 array [len(sel_l), len(sel_u)] (row = lower index); with no
    selection it is the full vector in index order x = x_u + 2^{n_u} x_l.  A copy
    range gives the partial sum over those copies; ``out`` accumulates into an
    existing array.
    """
    if sel_u is None:
        sel_u = np.arange(1 << plan.n_u, dtype=np.uint64)
    if sel_l is None:
        sel_l = np.arange(1 << plan.n_l, dtype=np.uint64)
    sel_u = np.ascontiguousarray(sel_u, dtype=np.uint64)
    sel_l = np.ascontiguousarray(sel_l, dtype=np.uint64)
    if k_end is None:
        k_end = plan.copies
    acc = 1
    if out is None:
        out = np.zeros((sel_l.size, sel_u.size), dtype=np.complex128)
        acc = 0
    up = _encode(plan.upper)
    lo = _encode(plan.lower)
    rc = lib().or_cut_sum(plan.n_u, _ptr(up, ctypes.c_int32), up.shape[0],
                          plan.n_l, _ptr(lo, ctypes.c_int32), lo.shape[0],
                          k_begin, k_end, _ptr(sel_u, ctypes.c_uint64), sel_u.size,
                          _ptr(sel_l, ctypes.c_uint64), sel_l.size, acc,
                          _ptr(out, ctypes.c_double))
    assert rc == 0
    return out


def part_state(plan, p, k):
    """State of part p of a MultiCutPlan for its copy index k (FP64)."""
    n_p = plan.nq[p]
    tmpl = _encode(plan.parts[p])
    psi = np.zeros(1 << n_p, dtype=np.complex128)
    rc = lib().or_half_state(n_p, _ptr(tmpl, ctypes.c_int32), tmpl.shape[0], k, _ptr(psi, ctypes.c_double))
    assert rc == 0
    return psi


def multi_cut_amplitudes(plan, sels=None):
    """Section 3 / Fig. 3 multi-part cut-and-sum:
        A(x_0, ..., x_{t-1}) = sum over l_1 .. l_{t-1} of  prod_p  S_p[l_p, l_{p+1}][x_p]
    with S_p the state of part p for boundary values l_p (above) and l_{p+1}
    (below).  sels[p] selects indices of part p (None: all).  Returns complex128
    [n_{t-1}, ..., n_0] (row-major; with no selection the full vector in index
    order x = x_0 + 2^{q_0} x_1 + ...).  The sum over the boundary bits is one
    numpy einsum over the part tensors."""
    t = plan.t
    sels = sels or [None] * t
    tensors = []
    for p in range(t):
        n_above = 1 << plan.c(p) if p > 0 else 1
        n_below = 1 << plan.c(p + 1) if p < t - 1 else 1
        sel = np.arange(1 << plan.nq[p]) if sels[p] is None else np.asarray(sels[p], dtype=np.int64)
        S = np.zeros((n_above, n_below, sel.size), dtype=np.complex128)
        for la in range(n_above):
            for lb in range(n_below):
                S[la, lb] = part_state(plan, p, plan.part_index(p, la, lb))[sel]
        tensors.append(S)
    # einsum subscripts: boundary j -> letter b_j, part p's index -> letter x_p
    letters = "abcdefghijklmnopqrstuvwxyz"
    bl = [None] + [letters[j] for j in range(1, t)]
    xl = [letters[13 + p].upper() for p in range(t)]
    terms, ops = [], []
    for p in range(t):
        above = bl[p] if p > 0 else "y"
        below = bl[p + 1] if p < t - 1 else "z"
        T = tensors[p]
        if p == 0:
            T = T[0]
            terms.append(below + xl[p])
        elif p == t - 1:
            T = T[:, 0]
            terms.append(above + xl[p])
        else:
            terms.append(above + below + xl[p])
        ops.append(T)
    out = "".join(reversed(xl))
    return np.einsum(",".join(terms) + "->" + out, *ops, optimize=True)


def floyd_select(rng, universe, count):
    """Floyd's algorithm: `count` distinct values of [0, universe), sorted ascending.

    For j = universe-count .. universe-1: t = draw mod (j+1); insert t unless it is
    already chosen, else insert j.  One splitmix64 draw per j.
    """
    if count >= universe:
        return np.arange(universe, dtype=np.uint64)
    chosen = set()
    for j in range(universe - count, universe):
        t = rng.next() % (j + 1)
        chosen.add(j if t in chosen else t)
    return np.array(sorted(chosen), dtype=np.uint64)


def select(n_u_qubits, n_sel_u, n_l_qubits, n_sel_l, seed):
    """The amplitude selection of Section 3 ("sampling" of components): distinct
    upper bitstrings first, then distinct lower ones, from one splitmix64(seed)."""
    rng = SplitMix64(seed)
    su = floyd_select(rng, 1 << n_u_qubits, n_sel_u)
    sl = floyd_select(rng, 1 << n_l_qubits, n_sel_l)
    return su, sl


KS_BINS = 4096


def gumbel_cdf(z):
    """CDF of Eq. 7 with alpha = 1: the integral of exp(z - e^z) is 1 - exp(-e^z)."""
    return 1.0 - np.exp(-np.exp(z))


def stats(amps, n_qubits):
    """Section 3 statistics over a block of amplitudes, FP64:
    [sum |A|^2, mean w, mean ln w over w > 0, binned KS distance to Eq. 7],
    with w = 2^n |A|^2 and z = ln w.

    Eq. 7 (alpha = 1) has the CDF F(z) = 1 - exp(-e^z) = 1 - exp(-w), so u = F(z)
    is uniform on [0, 1) if z follows Eq. 7.  The KS distance is taken between the
    empirical CDF of u and the uniform CDF at the KS_BINS equal bin edges of u.
    Returns (stats, histogram of u).
    """
    a = np.asarray(amps).astype(np.complex128).ravel()
    p = a.real * a.real + a.imag * a.imag
    w = p * math.ldexp(1.0, n_qubits)
    norm = float(p.sum())
    mean_w = float(w.mean())
    pos = w > 0
    mean_ln = float(np.log(w[pos]).mean()) if pos.any() else float("-inf")
    u = -np.expm1(-w)
    idx = np.minimum(np.floor(u * KS_BINS), KS_BINS - 1).astype(np.int64)
    hist = np.bincount(idx, minlength=KS_BINS)
    return np.array([norm, mean_w, mean_ln, ks_from_hist(hist)]), hist


def ks_from_hist(hist):
    """max_b |G(u_b) - u_b| at the bin edges u_b = (b + 1) / KS_BINS."""
    hist = np.asarray(hist, dtype=np.float64)
    tot = hist.sum()
    if tot == 0:
        return 0.0
    edges = np.arange(1, KS_BINS + 1) / KS_BINS
    emp = np.cumsum(hist) / tot
    return float(np.max(np.abs(emp - edges)))


# ---------------------------------------------------------------------------
# Measurement outcomes (Section 3: "measurement outcomes of the full vector space
# can be extracted"): Born-rule samples of a block of amplitudes, and the
# cross-entropy statistics of the samples against the distribution of Eq. 7.
# ---------------------------------------------------------------------------
EULER_GAMMA = 0.57721566490153286061


def splitmix64_at(seed, counters):
    """Outputs c of the splitmix64 stream seeded with `seed` (c = 0 is the first
    output): state_c = seed + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64, then the
    published finaliser (shifts 30, 27, 31; multipliers 0xBF58476D1CE4E5B9,
    0x94D049BB133111EB), vectorised over the counters."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def born_proposals(seed, count, c_begin, c_end):
    """Proposal c of the rejection sampler: index i_c = r_{2c} mod count and
    uniform u_c = (r_{2c+1} >> 11) * 2^-53 in [0, 1), from the counter-based
    splitmix64 stream r seeded with `seed`."""
    c = np.arange(c_begin, c_end, dtype=np.uint64)
    r_i = splitmix64_at(seed, np.uint64(2) * c)
    r_u = splitmix64_at(seed, np.uint64(2) * c + np.uint64(1))
    i = r_i % np.uint64(count)
    u = (r_u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return i, u


def born_sample(amps, seed, n_samples, max_proposals, batch=1 << 20):
    """Born-rule samples over a block of amplitudes by rejection sampling: with
    p = |A|^2 in FP64 and p_max its largest value over the block, proposal c (see
    born_proposals) is accepted when u_c * p_max < p_{i_c}.  Accepted i follow
    p / sum(p) over the block (the Born rule restricted to the block).
    Returns (indices, proposal ordinals, p_max) of the first n_samples accepted
    proposals among the first max_proposals."""
    a = np.asarray(amps).astype(np.complex128).ravel()
    p = a.real * a.real + a.imag * a.imag
    pmax = float(p.max())
    idx, ords = [], []
    got = 0
    c0 = 0
    while got < n_samples and c0 < max_proposals:
        c1 = min(max_proposals, c0 + batch)
        i, u = born_proposals(seed, p.size, c0, c1)
        acc = np.nonzero(u * pmax < p[i.astype(np.int64)])[0]
        take = acc[: n_samples - got]
        idx.append(i[take])
        ords.append(take.astype(np.uint64) + np.uint64(c0))
        got += take.size
        c0 = c1
    idx = np.concatenate(idx) if idx else np.zeros(0, np.uint64)
    ords = np.concatenate(ords) if ords else np.zeros(0, np.uint64)
    return idx, ords, pmax


def cross_entropy(p_samples, n_qubits):
    """Cross-entropy statistics of samples x_s with probabilities p(x_s), w = 2^n p:
    linear  mean(w) - 1
    log     mean(ln w) + gamma
    Under Eq. 7 (alpha = 1, w exponentially distributed) a sample drawn by the
    Born rule has w with density w e^{-w}, so E[w] = 2 and E[ln w] = 1 - gamma
    (both statistics 1); a uniform sample has E[w] = 1 and E[ln w] = -gamma (both
    0)."""
    w = np.asarray(p_samples, dtype=np.float64) * math.ldexp(1.0, n_qubits)
    return float(w.mean() - 1.0), float(np.log(w).mean() + EULER_GAMMA)
