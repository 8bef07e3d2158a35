"""GPU parity on explicit copy lists and at the 42- and 64-qubit sizes, through the
C-ABI.

  copy lists     sim_evolve_halves_list against the oracle's sum over the same copies
  42 qubits      6x7 grid, depth 22, c = 14 (16384 copies of two 21-qubit halves):
                 a copy subset against the oracle's partial cut-and-sum, and a
                 diagonal circuit over all 16384 copies against its closed form
  64 qubits      8x8 grid, depth 22, c = 16 (65536 copies of two 32-qubit halves):
                 a seeded copy, complex64 sweeps + split contraction against the
                 plain complex128 GPU path + FP64 contraction on the same copy
"""
import numpy as np
import pytest

import oracle
from oracle import circuit as oc
import paper_1802_06952_gb300 as sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-5
TOL_PLAIN = 1e-12


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06952_gb300 import build
    build.build()
    sim.lib()
    torch.cuda.set_device(0)
    yield
    sim.sim_release_cache()


def rel_err(got, ref):
    scale = float(np.max(np.abs(ref)))
    diff = float(np.max(np.abs(got - ref)))
    return diff if scale == 0 else diff / scale


def contract(h, contraction, M, N):
    dt = torch.complex128 if contraction == sim.SIM_FP64_PLAIN else torch.complex64
    out = torch.zeros((M, N), dtype=dt, device="cuda")
    sim.sim_amplitudes(h, contraction, False, out)
    sim.sim_status()
    return out


class Plan:
    def __init__(self, R, C, d, seed, b, gate_list=None):
        self.circ = sim.sim_build_circuit(R, C, d, seed, b, gate_list)
        self.plan, self.c, self.copies, self.nu, self.nl = sim.sim_cut(self.circ, b)
        self.halves = []

    def keep(self, h):
        self.halves.append(h)
        return h

    def close(self):
        for h in self.halves:
            sim.sim_destroy_halves(h)
        sim.sim_destroy_cut(self.plan)
        sim.sim_destroy_circuit(self.circ)
        sim.sim_release_cache()


def test_copy_list_matches_oracle():
    """An explicit, unordered list of copies: the contraction is the oracle's sum over
    exactly those copies, and each listed leaf is the oracle's half-state."""
    R, C, d, seed, b = 4, 5, 16, 2, 2
    gates, oplan = oc.grid_cut(R, C, d, seed, b)
    rng = np.random.default_rng(11)
    copies = rng.permutation(oplan.copies)[:11].astype(np.uint64)
    su = np.sort(rng.permutation(1 << oplan.n_u)[:40]).astype(np.uint64)
    sl = np.sort(rng.permutation(1 << oplan.n_l)[:36]).astype(np.uint64)
    ref = sum(oracle.cut_amplitudes(oplan, su, sl, int(k), int(k) + 1) for k in copies)
    p = Plan(R, C, d, seed, b)
    try:
        h = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C64, copies, su, sl))
        assert rel_err(contract(h, sim.SIM_SPLIT_FP16, sl.size, su.size).cpu().numpy(), ref) <= TOL_SPLIT
        hp = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C128_PLAIN, copies, su, sl))
        assert rel_err(contract(hp, sim.SIM_FP64_PLAIN, sl.size, su.size).cpu().numpy(), ref) <= TOL_PLAIN
        # full leaves of one listed copy against the oracle's half-states
        hf = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C64, copies[3:6]))
        k = int(copies[4])
        for half, nq in ((0, oplan.n_u), (1, oplan.n_l)):
            want = oracle.half_state(oplan, half, k)
            buf = torch.zeros(1 << nq, dtype=torch.complex64, device="cuda")
            sim.sim_halves_leaf(hf, half, k, buf)
            assert rel_err(buf.cpu().numpy(), want) <= 1e-5
        with pytest.raises(sim.SimError):
            sim.sim_halves_leaf(hf, 0, int(copies[0]), buf)
    finally:
        p.close()


def test_config3_42q_copy_subsets():
    """42 qubits (6x7, depth 22, c = 14), the configured 2^14 x 2^14 selection: a copy
    range and a seeded copy list, each on an 8 x 8 block of sampled amplitudes
    against the oracle's partial cut-and-sum over the same copies."""
    R, C, d, seed, b = 6, 7, 22, 0, 3
    gates, oplan = oc.grid_cut(R, C, d, seed, b)
    assert oplan.c == 14 and oplan.n_u == oplan.n_l == 21
    su, sl = sim.sim_select(21, 1 << 14, 21, 1 << 14, 0)
    iu = np.arange(5, 1 << 14, 2039)[:8]
    il = np.arange(9, 1 << 14, 2029)[:8]
    lst, _ = sim.sim_select(14, 8, 1, 1, 3)
    p = Plan(R, C, d, seed, b)
    try:
        for kind, arg in (("range", (100, 116)), ("list", lst)):
            if kind == "range":
                h = p.keep(sim.sim_evolve_halves(p.plan, sim.SIM_C64, arg[0], arg[1], su, sl))
                ref = oracle.cut_amplitudes(oplan, su[iu], sl[il], arg[0], arg[1])
            else:
                h = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C64, arg, su, sl))
                ref = sum(oracle.cut_amplitudes(oplan, su[iu], sl[il], int(k), int(k) + 1) for k in arg)
            # 16 copies in the range take split-bf16; the 8-copy list takes split-fp16
            # (split-bf16 is offered from 16 copies on)
            out = contract(h, sim.SIM_SPLIT_BF16 if kind == "range" else sim.SIM_SPLIT_FP16, sl.size, su.size)
            got = out[torch.from_numpy(il).cuda()][:, torch.from_numpy(iu).cuda()].cpu().numpy()
            assert rel_err(got, ref) <= TOL_SPLIT, kind
            del out
            sim.sim_destroy_halves(p.halves.pop())
    finally:
        p.close()


def diag_circuit_text(R, C, depth, b):
    """H layer, CZ patterns, T on the idle qubits of odd layers: A(x) is
    2^{-n/2} w^{m1(x)} (-1)^{m2(x)} (Eqs. 4, 6)."""
    n = R * C
    gates = [(0, "H", q) for q in range(n)]
    tsets, czsets = [], []
    for t in range(1, depth):
        pairs = oc.pattern_couplers(R, C, b, oc.pattern_of_layer(t))
        busy = {q for pr in pairs for q in pr}
        czsets.append(pairs)
        layer = [(t, "CZ", a, c) for (a, c) in pairs]
        if t % 2 == 1:
            ts = [q for q in range(n) if q not in busy]
            tsets.append(ts)
            layer += [(t, "T", q) for q in ts]
        layer.sort(key=lambda g: g[2])
        gates += layer
    return oc.to_text(R, C, depth, 0, gates), tsets, czsets


def test_config3_42q_diagonal_closed_form_all_copies():
    """A diagonal 42-qubit circuit with 14 cut CZs: the contraction over all 16384
    copies on a 512 x 512 selection against the closed form (no oracle involved);
    this pins the sum over the full copy index."""
    R, C, b, depth = 6, 7, 3, 22
    txt, ts, cz = diag_circuit_text(R, C, depth, b)
    p = Plan(R, C, depth, 0, b, gate_list=txt)
    try:
        assert p.c == 14
        su, sl = sim.sim_select(21, 512, 21, 512, 7)
        h = p.keep(sim.sim_evolve_halves(p.plan, sim.SIM_C64, 0, p.copies, su, sl))
        got = contract(h, sim.SIM_SPLIT_BF16, sl.size, su.size).cpu().numpy()
        x = (sl[:, None] << np.uint64(21)) | su[None, :]
        bit = lambda q: ((x >> np.uint64(q)) & np.uint64(1)).astype(np.int64)
        m1 = sum(bit(q) for s in ts for q in s)
        m2 = sum(bit(a) & bit(c) for pr in cz for (a, c) in pr)
        ref = 2.0 ** -21 * np.exp(1j * np.pi / 4 * m1) * (-1.0) ** m2
        assert rel_err(got, ref) <= TOL_SPLIT
    finally:
        p.close()


def test_config4_64q_seeded_copy_vs_plain_fp64():
    """64 qubits (8x8, depth 22, cut between rows 3 and 4, c = 16): one copy drawn with
    splitmix64(0), 1024 x 1024 selected entries of its two 32-qubit leaves.

    A single copy's contraction is the outer product U_k (x) L_k, so its error is the
    two leaves' errors plus the split rounding, with no averaging over copies.  The
    checks separate them: each complex64 leaf against the plain complex128 GPU path
    (<= 1e-5 of the leaf's largest entry), the split-fp16 contraction against the
    FP64 outer product of its own leaves, within the split's per-product bound: hi +
    lo leaves a residual of 2^-22 of each operand (10 fp16 mantissa bits) and lo*lo
    is dropped, 3 * 2^-22 in all (FP64 plain <= 1e-12).  Split-bf16, whose
    per-product bound 3 * 2^-16 is above 1e-5, is refused for one copy."""
    R, C, d, seed, b = 8, 8, 22, 0, 4
    p = Plan(R, C, d, seed, b)
    try:
        assert p.c == 16 and p.nu == p.nl == 32
        copies, _ = sim.sim_select(16, 1, 1, 1, 0)
        su, sl = sim.sim_select(32, 1024, 32, 1024, 1)

        def leaves_of(h, dt):
            out = []
            for half, n in ((0, su.size), (1, sl.size)):
                buf = torch.zeros(n, dtype=dt, device="cuda")
                sim.sim_halves_leaf(h, half, int(copies[0]), buf)
                out.append(buf.cpu().numpy().astype(np.complex128))
            return out

        h = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C64, copies, su, sl))
        lu, ll = leaves_of(h, torch.complex64)
        outer = ll[:, None] * lu[None, :]
        assert rel_err(contract(h, sim.SIM_SPLIT_FP16, sl.size, su.size).cpu().numpy(), outer) <= 3 * 2.0 ** -22
        with pytest.raises(sim.SimError) as ei:
            contract(h, sim.SIM_SPLIT_BF16, sl.size, su.size)
        assert ei.value.code == sim.SIM_EUNSUPPORTED
        sim.sim_destroy_halves(p.halves.pop())
        sim.sim_release_cache()
        hp = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C128_PLAIN, copies, su, sl))
        pu, pl = leaves_of(hp, torch.complex128)
        for got, want in ((lu, pu), (ll, pl)):
            assert np.max(np.abs(want)) > 0
            assert rel_err(got, want) <= TOL_SPLIT
        ref = contract(hp, sim.SIM_FP64_PLAIN, sl.size, su.size).cpu().numpy()
        assert rel_err(ref, pl[:, None] * pu[None, :]) <= TOL_PLAIN
    finally:
        p.close()


@pytest.mark.parametrize("R,C,d,seed,b,with_oracle", [(4, 4, 10, 0, 2, True), (6, 5, 16, 1, 3, True),
                                                      (6, 8, 16, 2, 3, False)])
def test_host_levels_match_device_levels(R, C, d, seed, b, with_oracle):
    """Copy-tree level buffers in pinned host memory (sim_opts.host_levels), read and
    written by the sweep kernels over the host link: the same leaves, bit for bit, as
    with device-resident levels (same kernels, same order), and the oracle's
    amplitudes on a selection (where it runs in seconds).  The 6x8 case has
    24-qubit halves (128 MB states)."""
    gates, oplan = oc.grid_cut(R, C, d, seed, b)
    rng = np.random.default_rng(seed)
    su = np.sort(rng.permutation(1 << oplan.n_u)[:48]).astype(np.uint64)
    sl = np.sort(rng.permutation(1 << oplan.n_l)[:40]).astype(np.uint64)
    p = Plan(R, C, d, seed, b)
    try:
        ks = np.arange(min(p.copies, 32), dtype=np.uint64)
        hd = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C64, ks, su, sl))
        hh = p.keep(sim.sim_evolve_halves_list(p.plan, sim.SIM_C64, ks, su, sl, opts={"host_levels": 1}))
        for half, n in ((0, su.size), (1, sl.size)):
            for k in (int(ks[0]), int(ks[-1])):
                a = torch.zeros(n, dtype=torch.complex64, device="cuda")
                bb = torch.zeros(n, dtype=torch.complex64, device="cuda")
                sim.sim_halves_leaf(hd, half, k, a)
                sim.sim_halves_leaf(hh, half, k, bb)
                assert torch.equal(a, bb)
        if with_oracle:
            got = contract(hh, sim.SIM_SPLIT_FP16, sl.size, su.size).cpu().numpy()
            ref = sum(oracle.cut_amplitudes(oplan, su, sl, int(k), int(k) + 1) for k in ks)
            assert rel_err(got, ref) <= TOL_SPLIT
    finally:
        p.close()
