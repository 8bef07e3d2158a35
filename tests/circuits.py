"""Explicit test circuits shared by several test files (plain gate lists)."""
import numpy as np

from oracle import circuit as oc


def cx_cut_circuit(seed, name="CX"):
    """4x4 grid: H layer, CZ patterns, random single-qubit gates, and controlled
    gates (name: CX, CT or CY2) across the cut (rows 1 | 2) in both directions."""
    R, C, b, depth = 4, 4, 2, 10
    base = oc.generate(R, C, depth, seed, b)
    rng = np.random.default_rng(seed)
    gates = list(base)
    busy = {}
    for g in base:
        for q in g[2:]:
            busy.setdefault(g[0], set()).add(q)
    extra = []
    for t in range(2, depth):
        free = [q for q in range(R * C) if q not in busy.get(t, set())]
        up = [q for q in free if q < b * C]
        lo = [q for q in free if q >= b * C]
        if up and lo:
            qa, qb = int(rng.choice(up)), int(rng.choice(lo))
            extra.append((t, name, qa, qb) if t % 2 else (t, name, qb, qa))
            busy.setdefault(t, set()).update((qa, qb))
    gates = sorted(gates + extra, key=lambda g: (g[0], g[2]))
    return R, C, b, depth, gates


def with_cross_controlled(R, C, depth, seed, b, rng, names=("CX", "CT", "CY2"), p=0.5, max_cuts=12):
    """The generated circuit plus, in each layer t >= 2 with probability p, one
    controlled gate (name drawn from names) between a free qubit of the upper half
    (rows < b) and a free qubit of the lower half, in a random direction, as long as
    the cut stays at max_cuts copy bits or fewer."""
    base = oc.generate(R, C, depth, seed, b)
    room = max_cuts - oc.CutPlan(R * C, b * C, base).c
    busy = {}
    for g in base:
        for q in g[2:]:
            busy.setdefault(g[0], set()).add(q)
    extra = []
    for t in range(2, depth):
        if rng.random() >= p or len(extra) >= room:
            continue
        free = [q for q in range(R * C) if q not in busy.get(t, set())]
        up = [q for q in free if q < b * C]
        lo = [q for q in free if q >= b * C]
        if up and lo:
            qa, qb = int(rng.choice(up)), int(rng.choice(lo))
            name = names[int(rng.integers(len(names)))]
            extra.append((t, name, qa, qb) if rng.random() < 0.5 else (t, name, qb, qa))
            busy.setdefault(t, set()).update((qa, qb))
    return sorted(base + extra, key=lambda g: (g[0], g[2]))
