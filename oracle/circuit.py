"""Oracle-side random grid circuit generator, canonical gate-list text, and cut plan.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It is written independently of the library's own C++
generator and planner; the two are compared by gate-list text equality.

Circuit model (Supplementary A, Eq. 3 and the text around it): a circuit is a
sequence of layers G_t = (V_t, E_t) on the qubits of an R x C grid; every edge
of E_t is a CZ, no qubit is in two edges of one layer, and single-qubit gates
sit on qubits that are not in an edge.  Qubit q = r*C + c (row r, column c).

Readings taken where the paper is silent (its circuit figures are lost):

* Layer 0 is H on every qubit.  Layer t >= 1 uses CZ pattern p(t) = ((t-1) mod 8) + 1.
* Patterns 1-4 are horizontal couplers (r,c)-(r,c+1) whose (r mod 2, c mod 2) is
  (0,0), (1,1), (0,1), (1,0).  Patterns 5-8 are vertical couplers (r,c)-(r+1,c):
  5: r != b-1 (mod 2), r+c even; 6: r != b-1 (mod 2), r+c odd;
  7: r == b-1 (mod 2), r+c even; 8: r == b-1 (mod 2), r+c odd.
  So the couplers that cross rows b-1 | b appear only in patterns 7 and 8, as
  Supplementary A states (cuts only in layers 8a+7 and 8a+8).
* A qubit gets a single-qubit gate at layer t >= 2 iff it was in a CZ at t-1 and
  is not in a CZ at t.  Its first such gate after H is T; later ones are X^1/2 or
  Y^1/2, one splitmix64 draw each in (layer, qubit) ascending order, Y^1/2 when the
  draw's top bit is 1.  Nothing is placed at t = 1.
"""

MASK64 = (1 << 64) - 1

GATE_NAMES = ("H", "X2", "Y2", "T", "CZ")


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014; constants as published by Vigna)."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def pattern_of_layer(t):
    return ((t - 1) % 8) + 1


def pattern_couplers(R, C, b, p):
    """Couplers (q1, q2), q1 < q2, of CZ pattern p on an R x C grid cut above row b."""
    out = []
    if p <= 4:
        want = {1: (0, 0), 2: (1, 1), 3: (0, 1), 4: (1, 0)}[p]
        for r in range(R):
            for c in range(C - 1):
                if (r % 2, c % 2) == want:
                    out.append((r * C + c, r * C + c + 1))
    else:
        same_parity_as_cut = p in (7, 8)
        want_even = p in (5, 7)
        for r in range(R - 1):
            for c in range(C):
                row_ok = ((r % 2) == ((b - 1) % 2)) == same_parity_as_cut
                par_ok = ((r + c) % 2 == 0) == want_even
                if row_ok and par_ok:
                    out.append((r * C + c, (r + 1) * C + c))
    return out


def generate(R, C, depth, seed, b=None, t_in_pool=False):
    """Gate list [(t, name, q) or (t, 'CZ', q1, q2)] of a random grid circuit.

    ``b`` is the cut row used to place patterns 5-8; by default b = R // 2.
    Gates within a layer are ordered by their first qubit.  A qubit gets a gate
    in layer t >= 2 when it was in a CZ at t - 1 and is not at t: its first such
    gate is T; later ones are X2 / Y2 by the top bit of the next splitmix64
    output, or with ``t_in_pool`` uniform over X2, Y2, T by (output >> 32) mod 3
    (a variant nearer the paper's T share; the paper does not print its rule).
    """
    if b is None:
        b = R // 2
    n = R * C
    rng = SplitMix64(seed)
    gates = []
    had_first = [False] * n
    prev_in_cz = [False] * n
    for t in range(depth):
        layer = []
        if t == 0:
            for q in range(n):
                layer.append((0, "H", q))
        else:
            pairs = pattern_couplers(R, C, b, pattern_of_layer(t))
            in_cz = [False] * n
            for (q1, q2) in pairs:
                in_cz[q1] = in_cz[q2] = True
                layer.append((t, "CZ", q1, q2))
            if t >= 2:
                for q in range(n):
                    if prev_in_cz[q] and not in_cz[q]:
                        if not had_first[q]:
                            had_first[q] = True
                            layer.append((t, "T", q))
                        else:
                            r = rng.next()
                            if t_in_pool:
                                name = ("X2", "Y2", "T")[(r >> 32) % 3]
                            else:
                                name = "Y2" if (r >> 63) & 1 else "X2"
                            layer.append((t, name, q))
            prev_in_cz = in_cz
        layer.sort(key=lambda g: g[2])
        gates.extend(layer)
    return gates


def to_text(R, C, depth, seed, gates):
    """Canonical gate-list text: a header line, then one 't NAME q [q2]' line per gate."""
    lines = ["circuit %d %d %d %d" % (R, C, depth, seed)]
    for g in gates:
        lines.append(" ".join(str(v) for v in g))
    return "\n".join(lines) + "\n"


def parse_text(text):
    """Inverse of to_text: returns (R, C, depth, seed, gates)."""
    rows = [ln.split() for ln in text.splitlines() if ln.strip() and not ln.startswith("#")]
    head = rows[0]
    assert head[0] == "circuit"
    R, C, depth, seed = (int(v) for v in head[1:5])
    gates = []
    for f in rows[1:]:
        t, name = int(f[0]), f[1]
        if name in TWO_QUBIT:
            gates.append((t, name, int(f[2]), int(f[3])))
        else:
            gates.append((t, name, int(f[2])))
    return R, C, depth, seed, gates


# two-qubit gates of the gate lists; the controlled ones map to their U
TWO_QUBIT = ("CZ", "CX", "CT", "CY2")
CONTROLLED_U = {"CT": "T", "CY2": "Y2"}


class CutPlan:
    """Section 2.1 / Supplementary A, Eqs. 6-8: split the qubits into an upper half
    (0 .. n_u-1) and a lower half (n_u .. n-1).  Every CZ with one endpoint in each
    half (the set E_int of its layer) is replaced by P_l on the upper endpoint and
    Q_l in {I, Z} on the lower endpoint, l being one bit l_m of the copy index.
    A controlled X across the cut (Supplementary A, Eq. 1 with U = X) is replaced
    by P_l on its control and X^l on its target, whichever half each is in; a
    controlled T or Y^1/2 (Eq. 1 with U = T or Y^1/2) likewise by P_l on its
    control and U^l on its target (slot ('CUTU', m, q, U)).
    Bits are numbered by (layer, upper qubit) ascending; copy k = sum_m l_m 2^m.
    """

    def __init__(self, n, n_u, gates):
        self.n, self.n_u, self.n_l = n, n_u, n - n_u
        self.cuts = []          # (t, h, k) with h upper, k lower (global indices)
        self.upper = []         # gates on upper qubits; cut slots as ('CUTP', m, h)
        self.lower = []         # gates on lower qubits (re-indexed); ('CUTZ', m, k-n_u)
        cz_cross = []
        for g in gates:
            if g[1] in TWO_QUBIT:
                a, c2 = min(g[2], g[3]), max(g[2], g[3])
                if a < n_u <= c2:
                    cz_cross.append((g[0], a, c2))
        cz_cross.sort()
        index = {cz: m for m, cz in enumerate(cz_cross)}
        self.cuts = cz_cross
        for g in gates:
            t = g[0]
            if g[1] == "CZ":
                a, c2 = min(g[2], g[3]), max(g[2], g[3])
                if c2 < n_u:
                    self.upper.append((t, "CZ", a, c2))
                elif a >= n_u:
                    self.lower.append((t, "CZ", a - n_u, c2 - n_u))
                else:
                    m = index[(t, a, c2)]
                    self.upper.append((t, "CUTP", m, a))
                    self.lower.append((t, "CUTZ", m, c2 - n_u))
            elif g[1] == "CX":
                qc, qt = g[2], g[3]
                if qc < n_u and qt < n_u:
                    self.upper.append(g)
                elif qc >= n_u and qt >= n_u:
                    self.lower.append((t, "CX", qc - n_u, qt - n_u))
                else:
                    m = index[(t, min(qc, qt), max(qc, qt))]
                    if qc < n_u:
                        self.upper.append((t, "CUTP", m, qc))
                        self.lower.append((t, "CUTX", m, qt - n_u))
                    else:
                        self.upper.append((t, "CUTX", m, qt))
                        self.lower.append((t, "CUTP", m, qc - n_u))
            elif g[1] in CONTROLLED_U:
                qc, qt = g[2], g[3]
                u = CONTROLLED_U[g[1]]
                if qc < n_u and qt < n_u:
                    self.upper.append(g)
                elif qc >= n_u and qt >= n_u:
                    self.lower.append((t, g[1], qc - n_u, qt - n_u))
                else:
                    m = index[(t, min(qc, qt), max(qc, qt))]
                    if qc < n_u:
                        self.upper.append((t, "CUTP", m, qc))
                        self.lower.append((t, "CUTU", m, qt - n_u, u))
                    else:
                        self.upper.append((t, "CUTU", m, qt, u))
                        self.lower.append((t, "CUTP", m, qc - n_u))
            else:
                q = g[2]
                if q < n_u:
                    self.upper.append(g)
                else:
                    self.lower.append((t, g[1], q - n_u))

    @property
    def c(self):
        return len(self.cuts)

    @property
    def copies(self):
        return 1 << self.c

    def n_equivalent(self):
        """Section 3: N_e = qubits per half-circuit + log2(number of half-circuits)."""
        return max(self.n_u, self.n_l) + self.c + 1

    def half_gates(self, half, k):
        """Concrete gate list of half 0 (upper) or 1 (lower) for copy k."""
        src = self.upper if half == 0 else self.lower
        out = []
        for g in src:
            if g[1] == "CUTP":
                bit = (k >> g[2]) & 1
                out.append((g[0], "P1" if bit else "P0", g[3]))
            elif g[1] == "CUTZ":
                bit = (k >> g[2]) & 1
                if bit:
                    out.append((g[0], "Z", g[3]))
            elif g[1] == "CUTX":
                bit = (k >> g[2]) & 1
                if bit:
                    out.append((g[0], "X", g[3]))
            elif g[1] == "CUTU":
                bit = (k >> g[2]) & 1
                if bit:
                    out.append((g[0], g[4], g[3]))
            else:
                out.append(g)
        return out

    def cuts_per_layer(self):
        per = {}
        for (t, _h, _k) in self.cuts:
            per[t] = per.get(t, 0) + 1
        return dict(sorted(per.items()))


def grid_cut(R, C, depth, seed, b=None, t_in_pool=False):
    """Generate a grid circuit and cut it between rows b-1 and b (default R // 2)."""
    if b is None:
        b = R // 2
    gates = generate(R, C, depth, seed, b, t_in_pool)
    return gates, CutPlan(R * C, b * C, gates)


class MultiCutPlan:
    """Section 3 / Fig. 3: the grid split into t row bands (parts) at the cut rows
    r_1 < ... < r_{t-1}.  Every CZ across a band boundary is rewritten by Eq. 1: P_l
    on its upper qubit, Z^l on its lower qubit, l one bit of the copy index, so the
    circuit is the sum over all boundary bits of products of t part circuits.

    Boundary j (between parts j-1 and j) has c_j cut CZs, numbered by (layer, upper
    qubit) ascending; its bits form l_j in [0, 2^{c_j}).  Part p carries the Z^l
    slots of boundary p (above it) and the P_l slots of boundary p+1 (below it).
    Its own copy index numbers its slots by (layer, upper qubit) ascending, so
    part_index() maps (l_p, l_{p+1}) to the part's copy index.  Parts are indexed
    from the top; qubit q of part p is global qubit q + offset[p].
    """

    def __init__(self, R, C, cut_rows, gates):
        rows = [0] + list(cut_rows) + [R]
        assert all(rows[i] < rows[i + 1] for i in range(len(rows) - 1)), "cut rows must increase inside the grid"
        self.R, self.C = R, C
        self.t = len(rows) - 1
        self.offset = [r * C for r in rows[:-1]]
        self.nq = [(rows[i + 1] - rows[i]) * C for i in range(self.t)]
        part_of = {}
        for p in range(self.t):
            for q in range(self.offset[p], self.offset[p] + self.nq[p]):
                part_of[q] = p
        # cut CZs per boundary j = 1 .. t-1 (index 0 unused)
        self.cuts = [[] for _ in range(self.t)]
        for g in gates:
            if g[1] == "CZ":
                a, b = min(g[2], g[3]), max(g[2], g[3])
                pa, pb = part_of[a], part_of[b]
                assert pb - pa <= 1, "a CZ may cross one boundary at most"
                if pa != pb:
                    self.cuts[pb].append((g[0], a, b))
            elif g[1] not in GATE_NAMES:
                raise ValueError("multi-part cuts take H, X2, Y2, T and CZ gates")
        for j in range(1, self.t):
            self.cuts[j].sort()
        bidx = {}
        for j in range(1, self.t):
            for i, cz in enumerate(self.cuts[j]):
                bidx[cz] = (j, i)
        # each part's slots in (layer, upper qubit) order: (t, upper, boundary, bit in boundary)
        slots = [[] for _ in range(self.t)]
        for j in range(1, self.t):
            for i, (tt, a, b) in enumerate(self.cuts[j]):
                slots[j - 1].append((tt, a, j, i))
                slots[j].append((tt, a, j, i))
        self.local = []          # per part: {(boundary, bit): local bit}
        for p in range(self.t):
            slots[p].sort()
            self.local.append({(s[2], s[3]): m for m, s in enumerate(slots[p])})
        self.parts = [[] for _ in range(self.t)]
        for g in gates:
            tt = g[0]
            if g[1] == "CZ":
                a, b = min(g[2], g[3]), max(g[2], g[3])
                pa, pb = part_of[a], part_of[b]
                if pa == pb:
                    o = self.offset[pa]
                    self.parts[pa].append((tt, "CZ", a - o, b - o))
                else:
                    j, i = bidx[(tt, a, b)]
                    self.parts[pa].append((tt, "CUTP", self.local[pa][(j, i)], a - self.offset[pa]))
                    self.parts[pb].append((tt, "CUTZ", self.local[pb][(j, i)], b - self.offset[pb]))
            else:
                p = part_of[g[2]]
                self.parts[p].append((tt, g[1], g[2] - self.offset[p]))

    def c(self, j):
        """Cut CZs across boundary j (1 .. t-1)."""
        return len(self.cuts[j])

    @property
    def c_total(self):
        return sum(len(self.cuts[j]) for j in range(1, self.t))

    def part_bits(self, p):
        return len(self.local[p])

    def part_index(self, p, l_above, l_below):
        """Part p's copy index for boundary values l_p = l_above and l_{p+1} = l_below."""
        k = 0
        for (j, i), m in self.local[p].items():
            v = l_above if j == p else l_below
            k |= ((v >> i) & 1) << m
        return k
