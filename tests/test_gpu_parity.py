"""GPU parity of libsim against the FP64 oracle, through the C-ABI.

Tolerances (max|da| / max|a| over the compared amplitudes):
  complex64 halves + split bf16 / fp16 contraction   <= 1e-5
  complex128 plain halves + FP64 contraction         <= 1e-12
  half-state fidelity of complex64 leaves            >= 1 - 1e-6
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
    """max|got - ref| / max|ref|; a reference that is exactly zero (a partial copy sum
    the projectors cancel) needs an exactly zero result."""
    scale = np.max(np.abs(ref))
    diff = float(np.max(np.abs(got - ref)))
    if scale == 0:
        return diff
    return diff / float(scale)


class Run:
    """Circuit + cut + evolved halves for one test; destroyed at exit."""

    def __init__(self, R, C, d, seed, b=None, gate_list=None, n=None):
        b = b or R // 2
        self.circ = sim.sim_build_circuit(R, C, d, seed, b, gate_list)
        self.plan, self.c, self.copies, self.nu, self.nl = sim.sim_cut(self.circ, b)
        self.halves = []

    def evolve(self, precision, k0=0, k1=None, sel_u=None, sel_l=None, opts=None):
        h = sim.sim_evolve_halves(self.plan, precision, k0, self.copies if k1 is None else k1, sel_u, sel_l, opts)
        self.halves.append(h)
        return h

    def close(self):
        for h in self.halves:
            sim.sim_destroy_halves(h)
        sim.sim_destroy_cut(self.plan)
        sim.sim_destroy_circuit(self.circ)


def amplitudes(h, contraction, M, N, accumulate=False, out=None):
    dt = torch.complex128 if contraction == sim.SIM_FP64_PLAIN else torch.complex64
    if out is None:
        out = torch.zeros((M, N), dtype=dt, device="cuda")
    sim.sim_amplitudes(h, contraction, accumulate, out)
    sim.sim_status()
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_config0_16q_plain_fp64(seed):
    """4x4 grid, depth 10, c = 4: complex128 plain path, all 2^16 amplitudes."""
    gates, plan = oc.grid_cut(4, 4, 10, seed, 2)
    ref = oracle.statevector(16, gates).reshape(1 << 8, 1 << 8)
    r = Run(4, 4, 10, seed)
    try:
        assert r.c == 4
        h = r.evolve(sim.SIM_C128_PLAIN)
        got = amplitudes(h, sim.SIM_FP64_PLAIN, 256, 256).cpu().numpy()
        assert rel_err(got, ref) <= TOL_PLAIN
    finally:
        r.close()


@pytest.mark.parametrize("contraction", [sim.SIM_SPLIT_BF16, sim.SIM_SPLIT_FP16, sim.SIM_FP64_PLAIN])
def test_config0_16q_c64(contraction):
    gates, plan = oc.grid_cut(4, 4, 10, 0, 2)
    ref = oracle.statevector(16, gates).reshape(256, 256)
    r = Run(4, 4, 10, 0)
    try:
        h = r.evolve(sim.SIM_C64)
        got = amplitudes(h, contraction, 256, 256).cpu().numpy()
        assert rel_err(got, ref) <= TOL_SPLIT
    finally:
        r.close()


def test_leaf_half_states_fidelity():
    gates, plan = oc.grid_cut(6, 4, 17, 2, 3)
    r = Run(6, 4, 17, 2, 3)
    try:
        h = r.evolve(sim.SIM_C64)
        hp = r.evolve(sim.SIM_C128_PLAIN)
        for k in (0, 1, 37, r.copies - 1):
            for half, nq in ((0, r.nu), (1, r.nl)):
                ref = oracle.half_state(plan, half, k)
                buf = torch.zeros(1 << nq, dtype=torch.complex64, device="cuda")
                sim.sim_halves_leaf(h, half, k, buf)
                got = buf.cpu().numpy().astype(np.complex128)
                nr, ng = np.vdot(ref, ref).real, np.vdot(got, got).real
                if nr == 0:
                    assert ng == 0
                    continue
                fid = abs(np.vdot(ref, got)) ** 2 / (nr * ng)
                assert fid >= 1 - 1e-6
                assert np.max(np.abs(got - ref)) <= 1e-6 * max(np.max(np.abs(ref)), 1e-30) * 10
                bp = torch.zeros(1 << nq, dtype=torch.complex128, device="cuda")
                sim.sim_halves_leaf(hp, half, k, bp)
                assert np.max(np.abs(bp.cpu().numpy() - ref)) <= 1e-14
    finally:
        r.close()


@pytest.mark.parametrize("R,C,d,seed,nsu,nsl,k0,k1", [
    (4, 5, 16, 0, 300, 77, 0, None),      # ragged selections, all copies
    (4, 5, 16, 1, 1, 1, 3, 16),           # single amplitude, copy subrange
    (6, 4, 17, 3, 129, 257, 5, 18),       # tile edges +-1, 13 copies
    (6, 4, 17, 3, 130, 257, 0, None),     # CTA-pair tiles with ragged rows and columns
    (4, 4, 10, 2, 256, 256, 0, None),     # "selection" of every index, shuffled order
])
def test_selection_and_copy_ranges(R, C, d, seed, nsu, nsl, k0, k1):
    gates, plan = oc.grid_cut(R, C, d, seed, R // 2)
    rng = np.random.default_rng(seed + 100)
    su = rng.permutation(1 << plan.n_u)[:nsu].astype(np.uint64)
    sl = rng.permutation(1 << plan.n_l)[:nsl].astype(np.uint64)
    k1v = plan.copies if k1 is None else k1
    ref = oracle.cut_amplitudes(plan, su, sl, k0, k1v)
    r = Run(R, C, d, seed)
    try:
        h = r.evolve(sim.SIM_C64, k0, k1v, su, sl)
        # split-bf16 is offered from 16 copies on; fewer take the fp16 split
        split = sim.SIM_SPLIT_BF16 if k1v - k0 >= 16 else sim.SIM_SPLIT_FP16
        got = amplitudes(h, split, nsl, nsu).cpu().numpy()
        assert rel_err(got, ref) <= TOL_SPLIT
        hp = r.evolve(sim.SIM_C128_PLAIN, k0, k1v, su, sl)
        gotp = amplitudes(hp, sim.SIM_FP64_PLAIN, nsl, nsu).cpu().numpy()
        assert rel_err(gotp, ref) <= TOL_PLAIN
    finally:
        r.close()


def test_accumulate_over_copy_batches():
    gates, plan = oc.grid_cut(4, 5, 16, 4, 2)
    ref = oracle.cut_amplitudes(plan)
    r = Run(4, 5, 16, 4)
    try:
        out = torch.zeros((1 << plan.n_l, 1 << plan.n_u), dtype=torch.complex64, device="cuda")
        bounds = [0, 5, 6, 40, plan.copies]
        for a, b in zip(bounds[:-1], bounds[1:]):
            h = r.evolve(sim.SIM_C64, a, b)
            sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, True, out)
        sim.sim_status()
        assert rel_err(out.cpu().numpy(), ref) <= TOL_SPLIT
    finally:
        r.close()


def test_many_copies_chunked_accumulation():
    """c = 12 (4096 copies of 12-qubit halves): the contraction accumulates 256 copies
    per tensor-memory run and adds the runs in fp32; a 300-copy range (one full and
    one partial run) is added into an existing output."""
    R, C, d, seed, b = 4, 6, 23, 8, 2
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    assert plan.c == 12
    rng = np.random.default_rng(4)
    su = np.unique(rng.integers(0, 1 << plan.n_u, 700)).astype(np.uint64)
    sl = np.unique(rng.integers(0, 1 << plan.n_l, 500)).astype(np.uint64)
    ref = oracle.cut_amplitudes(plan, su, sl)
    r = Run(R, C, d, seed, b)
    try:
        for kind in (sim.SIM_SPLIT_BF16, sim.SIM_SPLIT_FP16):
            h = r.evolve(sim.SIM_C64, 0, None, su, sl)
            got = amplitudes(h, kind, sl.size, su.size).cpu().numpy()
            assert rel_err(got, ref) <= TOL_SPLIT
        part = oracle.cut_amplitudes(plan, su, sl, 1000, 1300)
        out = torch.from_numpy(ref.astype(np.complex64)).cuda()
        h = r.evolve(sim.SIM_C64, 1000, 1300, su, sl)
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, True, out)
        sim.sim_status()
        assert rel_err(out.cpu().numpy(), ref + part) <= TOL_SPLIT
    finally:
        r.close()


def test_stats_fused_with_chunked_and_accumulated_contraction():
    """Statistics fused into the contraction when the final amplitudes are formed by
    a read-modify-write: 4096 copies (16 tensor-memory runs of 256 copies), and a
    second copy batch added into an existing output."""
    R, C, d, seed, b = 4, 6, 23, 8, 2
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    rng = np.random.default_rng(5)
    su = np.unique(rng.integers(0, 1 << plan.n_u, 800)).astype(np.uint64)
    su = su[: su.size & ~1]  # an even count: 16-byte output rows (CTA-pair kernel)
    sl = np.unique(rng.integers(0, 1 << plan.n_l, 600)).astype(np.uint64)
    nq = plan.n_u + plan.n_l
    ref = oracle.cut_amplitudes(plan, su, sl)
    st_ref, hist_ref = oracle.stats(ref, nq)
    n = ref.size
    r = Run(R, C, d, seed, b)
    try:
        out = torch.zeros((sl.size, su.size), dtype=torch.complex64, device="cuda")
        h = r.evolve(sim.SIM_C64, 0, None, su, sl)
        results = [sim.sim_amplitudes_stats(h, sim.SIM_SPLIT_BF16, False, out, want_hist=True)]
        assert rel_err(out.cpu().numpy(), ref) <= TOL_SPLIT
        out.zero_()
        h = r.evolve(sim.SIM_C64, 0, 1000, su, sl)
        sim.sim_amplitudes(h, sim.SIM_SPLIT_BF16, False, out)
        h = r.evolve(sim.SIM_C64, 1000, None, su, sl)
        results.append(sim.sim_amplitudes_stats(h, sim.SIM_SPLIT_BF16, True, out, want_hist=True))
        assert rel_err(out.cpu().numpy(), ref) <= TOL_SPLIT
        for st, hist in results:
            assert abs(st[0] - st_ref[0]) <= 1e-5 * st_ref[0]
            assert abs(st[1] - st_ref[1]) <= 1e-5 * st_ref[1]
            assert abs(st[2] - st_ref[2]) < 1e-4
            assert hist.sum() == hist_ref.sum() == n
            assert np.abs(hist.astype(np.int64) - hist_ref.astype(np.int64)).sum() <= n // 50
    finally:
        r.close()


def test_host_output_buffer():
    gates, plan = oc.grid_cut(4, 4, 10, 0, 2)
    ref = oracle.statevector(16, gates).reshape(256, 256)
    r = Run(4, 4, 10, 0)
    try:
        h = r.evolve(sim.SIM_C64)
        host = torch.zeros((256, 256), dtype=torch.complex64).pin_memory()
        sim.sim_amplitudes(h, sim.SIM_SPLIT_BF16, False, host)
        assert rel_err(host.numpy(), ref) <= TOL_SPLIT
        pageable = torch.zeros((256, 256), dtype=torch.complex64)
        sim.sim_amplitudes(h, sim.SIM_SPLIT_BF16, False, pageable)
        assert np.array_equal(pageable.numpy(), host.numpy())
    finally:
        r.close()


def test_host_output_written_in_place_and_staged():
    """Host output (pinned or pageable, overwritten or accumulated, full or ragged
    selections) goes through the device staging copy and gives the device route's
    bits."""
    R, C, d, seed, b = 4, 5, 16, 3, 2
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    full = oracle.statevector(R * C, gates).reshape(1 << plan.n_l, 1 << plan.n_u)
    r = Run(R, C, d, seed, b)
    try:
        h = r.evolve(sim.SIM_C64)
        shape = (1 << r.nl, 1 << r.nu)
        dev = torch.zeros(shape, dtype=torch.complex64, device="cuda")
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, dev)
        sim.sim_status()
        want = dev.cpu().numpy()
        assert rel_err(want, full) <= TOL_SPLIT
        pinned = torch.zeros(shape, dtype=torch.complex64).pin_memory()
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, pinned)
        assert np.array_equal(pinned.numpy(), want)
        # accumulate: the block is read back from the host first
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, True, pinned)
        assert rel_err(pinned.numpy(), 2 * full) <= TOL_SPLIT
        pageable = torch.zeros(shape, dtype=torch.complex64)
        sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, False, pageable)
        assert np.array_equal(pageable.numpy(), want)
        # ragged selection (n_u not a multiple of 4)
        su = np.sort(np.random.default_rng(5).choice(1 << r.nu, 301, replace=False)).astype(np.uint64)
        sl = np.arange(0, 1 << r.nl, 3, dtype=np.uint64)
        hs = r.evolve(sim.SIM_C64, sel_u=su, sel_l=sl)
        dsel = torch.zeros((sl.size, su.size), dtype=torch.complex64, device="cuda")
        sim.sim_amplitudes(hs, sim.SIM_SPLIT_FP16, False, dsel)
        psel = torch.zeros((sl.size, su.size), dtype=torch.complex64).pin_memory()
        sim.sim_amplitudes(hs, sim.SIM_SPLIT_FP16, False, psel)
        assert np.array_equal(psel.numpy(), dsel.cpu().numpy())
        assert rel_err(psel.numpy(), full[np.ix_(sl.astype(np.int64), su.astype(np.int64))]) <= TOL_SPLIT
    finally:
        r.close()


def diag_circuit_text(R, C, depth, b):
    """H layer, CZ patterns, T on idle qubits of odd layers (closed form of Eqs. 4, 6)."""
    n = R * C
    gates = [(0, "H", q) for q in range(n)]
    tsets, czsets = [], []
    for t in range(1, depth):
        pairs = oc.pattern_couplers(R, C, b, oc.pattern_of_layer(t))
        busy = {q for p in pairs for q in p}
        czsets.append(pairs)
        layer = [(t, "CZ", a, c) for (a, c) in pairs]
        if t % 2 == 1:
            ts = [q for q in range(n) if q not in busy]
            tsets.append(ts)
            layer += [(t, "T", q) for q in ts]
        layer.sort(key=lambda g: g[2])
        gates += layer
    return oc.to_text(R, C, depth, 0, gates), tsets, czsets


def test_diagonal_closed_form_30q():
    """All 2^30 amplitudes of a diagonal 30-qubit circuit with 10 cut CZs against
    2^{-15} w^{m1(x)} (-1)^{m2(x)} at sampled x (no oracle involved)."""
    R, C, b, depth = 6, 5, 3, 17
    txt, ts, cz = diag_circuit_text(R, C, depth, b)
    r = Run(R, C, depth, 0, b, gate_list=txt)
    try:
        assert r.c == 10
        h = r.evolve(sim.SIM_C64)
        out = amplitudes(h, sim.SIM_SPLIT_BF16, 1 << 15, 1 << 15)
        rng = np.random.default_rng(3)
        xs = rng.integers(0, 1 << 30, size=4096)
        got = out.reshape(-1)[torch.from_numpy(xs).cuda()].cpu().numpy()
        tm = sum(1 << q for s in ts for q in s)
        m1 = np.array([sum((int(x) >> q) & 1 for s in ts for q in s) for x in xs])
        m2 = np.array([sum(((int(x) >> a) & 1) & ((int(x) >> c) & 1) for p in cz for (a, c) in p) for x in xs])
        ref = 2.0 ** -15 * np.exp(1j * np.pi / 4 * m1) * (-1.0) ** m2
        assert tm > 0
        assert rel_err(got, ref) <= TOL_SPLIT
    finally:
        r.close()


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_config1_30q_split_bf16_sampled(seed):
    """6x5 grid (30 qubits), depth 16, c = 8: the full 32768 x 256 x 32768 contraction,
    checked on 4096 sampled amplitudes against the oracle's cut-and-sum."""
    gates, plan = oc.grid_cut(6, 5, 16, seed, 3)
    assert plan.c == 8
    rng = np.random.default_rng(seed)
    su = np.unique(rng.integers(0, 1 << 15, size=64)).astype(np.uint64)
    sl = np.unique(rng.integers(0, 1 << 15, size=64)).astype(np.uint64)
    ref = oracle.cut_amplitudes(plan, su, sl)
    r = Run(6, 5, 16, seed, 3)
    try:
        h = r.evolve(sim.SIM_C64)
        out = amplitudes(h, sim.SIM_SPLIT_BF16, 1 << 15, 1 << 15)
        got = out[torch.from_numpy(sl.astype(np.int64)).cuda()][:, torch.from_numpy(su.astype(np.int64)).cuda()]
        assert rel_err(got.cpu().numpy(), ref) <= TOL_SPLIT
        st = sim.sim_stats(out, 0, 1 << 30, 30)
        assert abs(st[0] - 1.0) < 1e-4      # unit norm of the full state
        del out
        torch.cuda.empty_cache()
    finally:
        r.close()


def test_config1_30q_plain_fp64_sampled():
    gates, plan = oc.grid_cut(6, 5, 16, 0, 3)
    rng = np.random.default_rng(11)
    su = np.unique(rng.integers(0, 1 << 15, size=48)).astype(np.uint64)
    sl = np.unique(rng.integers(0, 1 << 15, size=48)).astype(np.uint64)
    ref = oracle.cut_amplitudes(plan, su, sl)
    r = Run(6, 5, 16, 0, 3)
    try:
        h = r.evolve(sim.SIM_C128_PLAIN, 0, None, su, sl)
        got = amplitudes(h, sim.SIM_FP64_PLAIN, sl.size, su.size).cpu().numpy()
        assert rel_err(got, ref) <= TOL_PLAIN
    finally:
        r.close()


def test_stats_match_oracle():
    gates, plan = oc.grid_cut(4, 5, 16, 7, 2)
    ref = oracle.cut_amplitudes(plan)
    st_ref, hist_ref = oracle.stats(ref, 20)
    r = Run(4, 5, 16, 7)
    try:
        h = r.evolve(sim.SIM_C64)
        out = amplitudes(h, sim.SIM_SPLIT_BF16, 1 << plan.n_l, 1 << plan.n_u)
        n = 1 << 20
        # GPU statistics of the GPU amplitudes vs oracle statistics of the oracle's:
        # the amplitudes differ by the split-contraction error, which moves entries
        # that sit near a bin edge, so the histograms agree up to a share of entries
        for st, hist in (sim.sim_stats(out, 0, n, 20, want_hist=True),
                         sim.sim_amplitudes_stats(h, sim.SIM_SPLIT_BF16, False, out, want_hist=True)):
            assert abs(st[0] - st_ref[0]) < 1e-5 and abs(st[1] - st_ref[1]) < 1e-5
            assert abs(st[2] - st_ref[2]) < 1e-4
            assert abs(st[3] - st_ref[3]) < 1e-3
            assert hist.sum() == hist_ref.sum() == n
            assert np.abs(hist.astype(np.int64) - hist_ref.astype(np.int64)).sum() <= n // 50
        # the same complex64 block on both sides: only the fp32 bin decision (GPU)
        # against the FP64 one (oracle) differs, for entries within ~1e-7 of an edge
        ref64 = ref.astype(np.complex64)
        st_c, hist_c = oracle.stats(ref64, 20)
        st_g, hist_g = sim.sim_stats(torch.from_numpy(ref64).cuda(), 0, n, 20, want_hist=True)
        assert np.abs(hist_g.astype(np.int64) - hist_c.astype(np.int64)).sum() <= n // 250
        assert abs(st_g[0] - st_c[0]) < 1e-6 and abs(st_g[2] - st_c[2]) < 1e-5 and abs(st_g[3] - st_c[3]) < 2e-4
        # complex128 input: FP64 throughout, bins decided in FP64 on both sides
        st2, hist2 = sim.sim_stats(torch.from_numpy(ref).cuda(), 1, n, 20, want_hist=True)
        assert np.allclose(st2[:3], st_ref[:3], rtol=1e-12, atol=1e-12)
        assert np.abs(hist2.astype(np.int64) - hist_ref.astype(np.int64)).sum() <= 8
        assert abs(st2[3] - st_ref[3]) < 1e-5
    finally:
        r.close()


def test_sample_entry_point():
    r = Run(6, 5, 16, 2, 3)
    try:
        out = torch.zeros((200, 300), dtype=torch.complex64, device="cuda")
        su, sl, st = sim.sim_sample(r.plan, 300, 200, 9, out, r.nu, r.nl)
        ru, rl = oracle.select(r.nu, 300, r.nl, 200, 9)
        assert np.array_equal(su, ru) and np.array_equal(sl, rl)
        gates, plan = oc.grid_cut(6, 5, 16, 2, 3)
        ref = oracle.cut_amplitudes(plan, su, sl)
        assert rel_err(out.cpu().numpy(), ref) <= TOL_SPLIT
        st_ref, _ = oracle.stats(ref, 30)
        assert abs(st[1] - st_ref[1]) < 1e-4 * max(1, st_ref[1])
    finally:
        r.close()


@pytest.mark.parametrize("R,C,d,seed,b", [(6, 4, 17, 5, 3), (4, 6, 23, 8, 2)])
def test_fuse_widths_and_sweep_kernels_agree(R, C, d, seed, b):
    """Staged (shared-memory) and register-blocked sweeps, fuse widths 4..13: the
    register-blocked kernel runs for 8 <= k <= 13 (rank 0-4 lane gates by shuffle,
    5-7 warp gates through smem, 8+ register gates), the staged one otherwise."""
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    ref = oracle.cut_amplitudes(plan)
    # pass orders: 0 dependency-aware formation (the default), 1 in order
    for fq, kern, order in ((4, 0, 0), (7, 0, 0), (8, 0, 0), (9, 0, 0), (10, 1, 0), (10, 2, 0), (12, 1, 0),
                            (12, 2, 0), (13, 0, 0), (4, 0, 1), (9, 0, 1), (10, 2, 1), (13, 0, 1)):
        r = Run(R, C, d, seed, b)
        try:
            h = r.evolve(sim.SIM_C64, opts={"fuse_qubits": fq, "sweep_threads": 128, "sweep_kernel": kern,
                                            "pass_order": order})
            got = amplitudes(h, sim.SIM_SPLIT_FP16, 1 << plan.n_l, 1 << plan.n_u).cpu().numpy()
            assert rel_err(got, ref) <= TOL_SPLIT, (fq, kern, order)
            for k in (0, plan.copies - 1):
                for half, nq in ((0, plan.n_u), (1, plan.n_l)):
                    buf = torch.zeros(1 << nq, dtype=torch.complex64, device="cuda")
                    sim.sim_halves_leaf(h, half, k, buf)
                    hs = oracle.half_state(plan, half, k)
                    # a leaf can be exactly zero (two projectors on one cut qubit with
                    # opposite bits): the floor is the state's natural scale 2^{-n/2}
                    scale = max(np.max(np.abs(hs)), 2.0 ** (-nq / 2))
                    assert np.max(np.abs(buf.cpu().numpy() - hs)) <= 1e-5 * scale, (fq, kern, order)
        finally:
            r.close()


def test_gpu_argument_errors():
    r = Run(4, 4, 10, 0)
    try:
        with pytest.raises(sim.SimError) as e:
            r.evolve(sim.SIM_C64, opts={"pass_order": 2})
        assert e.value.code == sim.SIM_EINVAL
        with pytest.raises(sim.SimError) as e:
            r.evolve(sim.SIM_C64, 5, 5)
        assert e.value.code == sim.SIM_EINVAL
        with pytest.raises(sim.SimError):
            r.evolve(sim.SIM_C64, 0, 17)
        with pytest.raises(sim.SimError):
            r.evolve(sim.SIM_C64, 0, 16, np.array([256], dtype=np.uint64), None)
        h = r.evolve(sim.SIM_C128_PLAIN)
        out = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
        with pytest.raises(sim.SimError):
            sim.sim_amplitudes(h, sim.SIM_SPLIT_BF16, False, out)
        sim.sim_status()
    finally:
        r.close()


def test_t_in_pool_rule_circuit():
    """A circuit of the T-in-pool gate rule (T also after a qubit's first gate, folded
    into that layer's combined diagonal): full 20-qubit vector vs the oracle."""
    R, C, d, seed, b = 4, 5, 18, 3, 2
    gates, plan = oc.grid_cut(R, C, d, seed, b, t_in_pool=True)
    assert sum(1 for g in gates if g[1] == "T") > R * C
    ref = oracle.statevector(R * C, gates).reshape(1 << plan.n_l, 1 << plan.n_u)
    circ = sim.sim_build_circuit(R, C, d, seed, b, None, True)
    cp, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        for prec, kind, tol in ((sim.SIM_C64, sim.SIM_SPLIT_BF16, TOL_SPLIT),
                                (sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, TOL_PLAIN)):
            h = sim.sim_evolve_halves(cp, prec, 0, copies)
            got = amplitudes(h, kind, 1 << nl, 1 << nu).cpu().numpy()
            sim.sim_destroy_halves(h)
            assert rel_err(got, ref) <= tol
    finally:
        sim.sim_destroy_cut(cp)
        sim.sim_destroy_circuit(circ)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_controlled_x_cuts(seed):
    """Controlled X gates across the cut (Supplementary A, Eq. 1 with U = X: P_l on
    the control, X^l on the target, in either half): the full 16-qubit vector of the
    split path, the plain FP64 path, both sweep kernels and a copy list, against the
    oracle's uncut state vector."""
    from circuits import cx_cut_circuit
    R, C, b, depth, gates = cx_cut_circuit(seed)
    n, n_u = R * C, b * C
    ref = oracle.statevector(n, gates).reshape(1 << (n - n_u), 1 << n_u)
    circ = sim.sim_build_circuit(gate_list=oc.to_text(R, C, depth, 0, gates))
    cp, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        runs = [(sim.SIM_C64, sim.SIM_SPLIT_BF16, TOL_SPLIT, {"sweep_kernel": 2}),
                (sim.SIM_C64, sim.SIM_SPLIT_FP16, TOL_SPLIT, {"sweep_kernel": 1, "fuse_qubits": 5}),
                (sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, TOL_PLAIN, None)]
        for prec, kind, tol, opts in runs:
            h = sim.sim_evolve_halves(cp, prec, 0, copies, None, None, opts)
            got = amplitudes(h, kind, 1 << nl, 1 << nu).cpu().numpy()
            sim.sim_destroy_halves(h)
            assert rel_err(got, ref) <= tol, (prec, kind)
        # a copy list: the oracle's partial sum over those three copies.  A sum of
        # three outer products has no averaging to bring the bf16 split's per-product
        # error (3 * 2^-16) below 1e-5, so split-bf16 is refused and split-fp16 holds
        # the plain 1e-5.
        gplan = oc.CutPlan(n, n_u, gates)
        lst = np.array([copies - 1, 0, copies // 2 + 1], dtype=np.uint64)
        part = sum(oracle.cut_amplitudes(gplan, None, None, int(k), int(k) + 1) for k in lst)
        h = sim.sim_evolve_halves_list(cp, sim.SIM_C64, lst)
        with pytest.raises(sim.SimError) as ei:
            amplitudes(h, sim.SIM_SPLIT_BF16, 1 << nl, 1 << nu)
        assert ei.value.code == sim.SIM_EUNSUPPORTED
        got = amplitudes(h, sim.SIM_SPLIT_FP16, 1 << nl, 1 << nu).cpu().numpy()
        sim.sim_destroy_halves(h)
        assert rel_err(got, part) <= TOL_SPLIT
        h = sim.sim_evolve_halves_list(cp, sim.SIM_C128_PLAIN, lst)
        got = amplitudes(h, sim.SIM_FP64_PLAIN, 1 << nl, 1 << nu).cpu().numpy()
        sim.sim_destroy_halves(h)
        assert rel_err(got, part) <= TOL_PLAIN
    finally:
        sim.sim_destroy_cut(cp)
        sim.sim_destroy_circuit(circ)


@pytest.mark.parametrize("name,seed", [("CT", 0), ("CT", 1), ("CY2", 0), ("CY2", 2)])
def test_controlled_u_cuts(name, seed):
    """Controlled T (diagonal U) and controlled Y^1/2 (non-diagonal U) across the cut
    (Supplementary A, Eq. 1: P_l on the control, U^l on the target, in either half).
    The fused sweeps write U^l as copy-independent gates around a phase slot
    w^{b l x} (T^l: b = 1; (Y^1/2)^l = (X^1/2)^3 S^l X^1/2: b = 2); the plain path
    applies U in the copies with l = 1.  Full 16-qubit vectors through both sweep
    kernels and the plain FP64 path, and a copy list, against the oracle."""
    from circuits import cx_cut_circuit
    R, C, b, depth, gates = cx_cut_circuit(seed, name)
    n, n_u = R * C, b * C
    ref = oracle.statevector(n, gates).reshape(1 << (n - n_u), 1 << n_u)
    circ = sim.sim_build_circuit(gate_list=oc.to_text(R, C, depth, 0, gates))
    cp, c, copies, nu, nl = sim.sim_cut(circ, b)
    try:
        assert copies >= 16
        runs = [(sim.SIM_C64, sim.SIM_SPLIT_BF16, TOL_SPLIT, {"sweep_kernel": 2}),
                (sim.SIM_C64, sim.SIM_SPLIT_FP16, TOL_SPLIT, {"sweep_kernel": 2, "fuse_qubits": 8}),
                (sim.SIM_C64, sim.SIM_SPLIT_FP16, TOL_SPLIT, {"sweep_kernel": 1, "fuse_qubits": 5}),
                (sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, TOL_PLAIN, None)]
        for prec, kind, tol, opts in runs:
            h = sim.sim_evolve_halves(cp, prec, 0, copies, None, None, opts)
            got = amplitudes(h, kind, 1 << nl, 1 << nu).cpu().numpy()
            sim.sim_destroy_halves(h)
            assert rel_err(got, ref) <= tol, (prec, kind, opts)
        gplan = oc.CutPlan(n, n_u, gates)
        lst = np.array([copies - 1, 0, copies // 2 + 1], dtype=np.uint64)
        part = sum(oracle.cut_amplitudes(gplan, None, None, int(k), int(k) + 1) for k in lst)
        for prec, kind, tol in ((sim.SIM_C64, sim.SIM_SPLIT_FP16, TOL_SPLIT),
                                (sim.SIM_C128_PLAIN, sim.SIM_FP64_PLAIN, TOL_PLAIN)):
            h = sim.sim_evolve_halves_list(cp, prec, lst)
            got = amplitudes(h, kind, 1 << nl, 1 << nu).cpu().numpy()
            sim.sim_destroy_halves(h)
            assert rel_err(got, part) <= tol, (prec, kind)
    finally:
        sim.sim_destroy_cut(cp)
        sim.sim_destroy_circuit(circ)


class PhaseRun(Run):
    """Run whose cut applies the last cut layers as output signs (sim_cut_ex)."""

    def __init__(self, R, C, d, seed, b):
        self.circ = sim.sim_build_circuit(R, C, d, seed, b)
        self.plan, self.c, self.copies, self.nu, self.nl = sim.sim_cut_ex(self.circ, b, output_phase_cuts=True)
        self.halves = []


def test_output_phase_cuts_full_vector():
    """4x4 grid, depth 9: the two cut CZs of the last layer become output signs
    (c = 4 -> 2).  The rewrite is exact, so every contraction path gives the uncut
    state vector: split fp16 (CTA-pair kernel, sign in the epilogue) and FP64 plain
    (separate sign pass).  Four copies are too few for split-bf16, which is refused."""
    gates = oc.generate(4, 4, 9, 0, 2)
    ref = oracle.statevector(16, gates).reshape(256, 256)
    r = PhaseRun(4, 4, 9, 0, 2)
    try:
        assert r.c == 2 and len(sim.sim_cut_output_phases(r.plan)) == 2
        h = r.evolve(sim.SIM_C64)
        with pytest.raises(sim.SimError) as ei:
            amplitudes(h, sim.SIM_SPLIT_BF16, 256, 256)
        assert ei.value.code == sim.SIM_EUNSUPPORTED
        assert rel_err(amplitudes(h, sim.SIM_SPLIT_FP16, 256, 256).cpu().numpy(), ref) <= TOL_SPLIT
        hp = r.evolve(sim.SIM_C128_PLAIN)
        assert rel_err(amplitudes(hp, sim.SIM_FP64_PLAIN, 256, 256).cpu().numpy(), ref) <= TOL_PLAIN
    finally:
        r.close()


@pytest.mark.parametrize("nsu", [256, 255])
def test_output_phase_cuts_accumulate_and_selections(nsu):
    """Selections (255 upper indices: the single-CTA kernel with separate sign passes;
    256: the CTA-pair kernel) and accumulation over copy batches: each batch's part
    gets the sign, the earlier sum keeps its own."""
    R, C, d, seed, b = 6, 4, 16, 3, 3
    gates, plan = oc.grid_cut(R, C, d, seed, b)
    rng = np.random.default_rng(nsu)
    su = np.sort(rng.permutation(1 << plan.n_u)[:nsu]).astype(np.uint64)
    sl = np.sort(rng.permutation(1 << plan.n_l)[:200]).astype(np.uint64)
    ref = oracle.cut_amplitudes(plan, su, sl)
    r = PhaseRun(R, C, d, seed, b)
    try:
        assert r.c < plan.c
        out = torch.zeros((sl.size, su.size), dtype=torch.complex64, device="cuda")
        outp = torch.zeros((sl.size, su.size), dtype=torch.complex128, device="cuda")
        bounds = [0, 1, r.copies // 2, r.copies]
        for a, bnd in zip(bounds[:-1], bounds[1:]):
            h = r.evolve(sim.SIM_C64, a, bnd, su, sl)
            sim.sim_amplitudes(h, sim.SIM_SPLIT_FP16, True, out)
            hp = r.evolve(sim.SIM_C128_PLAIN, a, bnd, su, sl)
            sim.sim_amplitudes(hp, sim.SIM_FP64_PLAIN, True, outp)
        sim.sim_status()
        assert rel_err(out.cpu().numpy(), ref) <= TOL_SPLIT
        assert rel_err(outp.cpu().numpy(), ref) <= TOL_PLAIN
    finally:
        r.close()


def test_output_phase_cuts_30q_sampled():
    """The 30-qubit workload (6x5, depth 16) with its last cut layer as output signs:
    c = 8 -> 5 (32 copies), the full 2^30 vector against the oracle's cut-and-sum on
    sampled amplitudes, and the statistics fused into the same contraction."""
    gates, plan = oc.grid_cut(6, 5, 16, 1, 3)
    rng = np.random.default_rng(5)
    su = np.unique(rng.integers(0, 1 << 15, size=64)).astype(np.uint64)
    sl = np.unique(rng.integers(0, 1 << 15, size=64)).astype(np.uint64)
    ref = oracle.cut_amplitudes(plan, su, sl)
    r = PhaseRun(6, 5, 16, 1, 3)
    try:
        assert r.c == 5
        h = r.evolve(sim.SIM_C64)
        out = torch.empty((1 << 15, 1 << 15), dtype=torch.complex64, device="cuda")
        st = sim.sim_amplitudes_stats(h, sim.SIM_SPLIT_BF16, False, out)
        got = out[torch.from_numpy(sl.astype(np.int64)).cuda()][:, torch.from_numpy(su.astype(np.int64)).cuda()]
        assert rel_err(got.cpu().numpy(), ref) <= TOL_SPLIT
        assert abs(st[0] - 1.0) < 1e-4
        del out
        torch.cuda.empty_cache()
    finally:
        r.close()


def test_bounded_wait_reports_timeout_and_context_survives():
    """The bounded mbarrier wait of the contraction kernels, run on a barrier that
    nothing arrives on: it gives up after 100 ms, the host reads SIM_ETIMEOUT, the
    status word is clear afterwards, and the next contraction is correct."""
    import time
    t0 = time.perf_counter()
    rc = sim.sim_selftest_wait(100)
    dt = time.perf_counter() - t0
    assert rc == sim.SIM_ETIMEOUT
    assert 0.09 <= dt < 5.0
    sim.sim_status()  # raises unless the status word is clear
    gates, plan = oc.grid_cut(4, 4, 10, 0, 2)
    ref = oracle.statevector(16, gates).reshape(256, 256)
    r = Run(4, 4, 10, 0)
    try:
        h = r.evolve(sim.SIM_C64)
        assert rel_err(amplitudes(h, sim.SIM_SPLIT_BF16, 256, 256).cpu().numpy(), ref) <= TOL_SPLIT
    finally:
        r.close()
    with pytest.raises(sim.SimError):
        sim._check(sim.sim_selftest_wait(0))
