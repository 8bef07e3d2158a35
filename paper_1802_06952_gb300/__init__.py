"""Python binding of libsim, the GB300 (sm_103a) implementation of the cut-CZ
partition scheme of arXiv 1802.06952 (Section 2.1, Eq. 1; Supplementary A, Eqs. 6-8).

Argument marshalling only: every step of the computation runs in libsim.so
(CUDA kernels and the C++ host logic behind include/sim.h).  The functions keep
the C names.  Device buffers are torch tensors (their data_ptr is passed through)
and streams are torch.cuda.Stream objects or raw cudaStream_t integers.  If the
shared library is missing, importing works but every call raises: there is no
fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsim.so")

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ETIMEOUT, SIM_EUNSUPPORTED = range(6)
SIM_C64, SIM_C128_PLAIN = 0, 1
SIM_SPLIT_BF16, SIM_SPLIT_FP16, SIM_FP64_PLAIN = 0, 1, 2
SIM_KS_BINS = 4096
(SIM_PHASE_SWEEP, SIM_PHASE_GATHER, SIM_PHASE_PLAIN, SIM_PHASE_PACK, SIM_PHASE_CONTRACT,
 SIM_PHASE_FP64_GEMM, SIM_PHASE_STATS) = range(7)
SIM_NUM_PHASES = 7
PHASE_NAMES = ("sweep", "gather", "plain", "pack", "contract", "fp64_gemm", "stats")

# every symbol include/sim.h declares
EXPORTS = (
    "sim_build_circuit", "sim_circuit_info", "sim_circuit_text", "sim_cut", "sim_cut_list",
    "sim_plan_schedule", "sim_evolve_halves", "sim_halves_leaf", "sim_amplitudes", "sim_stats",
    "sim_select", "sim_sample", "sim_status", "sim_release_cache", "sim_destroy_circuit",
    "sim_destroy_cut", "sim_destroy_halves", "sim_last_error", "sim_version",
    "sim_profile_enable", "sim_profile_read", "sim_amplitudes_noalloc", "sim_amplitudes_stats",
    "sim_evolve_halves_list", "sim_plan_levels", "sim_batch_create", "sim_batch_run", "sim_batch_results",
    "sim_batch_info", "sim_destroy_batch", "sim_born_sample", "sim_cut_ex", "sim_cut_output_phases",
    "sim_cut_multi", "sim_multi_amplitudes", "sim_destroy_multi", "sim_selftest_wait", "sim_plan_sparse_qubits", "sim_plan_sparse_depth",
)
SIM_NOALLOC_SCRATCH_BYTES = 32 << 20


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libsim error %d: %s" % (code, msg))
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int), ("cols", ctypes.c_int), ("depth", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("cut_row", ctypes.c_int), ("gate_list", ctypes.c_char_p),
                ("rule_t_in_pool", ctypes.c_int)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("contraction", ctypes.c_int), ("autotune", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class SimCutOpts(ctypes.Structure):
    _fields_ = [("output_phase_cuts", ctypes.c_int), ("reserved", ctypes.c_int * 7)]


class SimOpts(ctypes.Structure):
    _fields_ = [("fuse_qubits", ctypes.c_int), ("sweep_threads", ctypes.c_int),
                ("gemm_group_m", ctypes.c_int), ("sweep_kernel", ctypes.c_int), ("pass_order", ctypes.c_int),
                ("host_levels", ctypes.c_int), ("sparse_leaves", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


_lib = None


def lib():
    """Load libsim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsim.so is not built; run paper_1802_06952_gb300/build.py "
                           "(or __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, u64p, i32p = ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "sim_build_circuit": (ctypes.c_int, [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]),
        "sim_circuit_info": (ctypes.c_int, [vp, ip, ip, ip]),
        "sim_circuit_text": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "sim_cut": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ip, u64p, ip, ip]),
        "sim_cut_ex": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(SimCutOpts), ctypes.POINTER(vp), ip, u64p,
                                      ip, ip]),
        "sim_cut_output_phases": (ctypes.c_int, [vp, i32p, ctypes.c_int, ip]),
        "sim_cut_list": (ctypes.c_int, [vp, i32p, ip]),
        "sim_cut_multi": (ctypes.c_int, [vp, ctypes.c_int, ip, ctypes.POINTER(vp), ip, ip, ip]),
        "sim_multi_amplitudes": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(u64p), u64p, vp,
                                                ctypes.POINTER(SimOpts), vp]),
        "sim_destroy_multi": (None, [vp]),
        "sim_selftest_wait": (ctypes.c_int, [ctypes.c_int, vp]),
        "sim_plan_schedule": (ctypes.c_int, [vp, ctypes.c_int, ip, ip, ip]),
        "sim_plan_levels": (ctypes.c_int, [vp, ctypes.c_int, i32p, ctypes.c_int, ip]),
        "sim_plan_sparse_qubits": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip]),
        "sim_plan_sparse_depth": (ctypes.c_int, [vp, ctypes.c_int, u64, ctypes.c_int, ip]),
        "sim_evolve_halves": (ctypes.c_int, [vp, ctypes.c_int, u64, u64, u64p, u64, u64p, u64,
                                             ctypes.POINTER(SimOpts), vp, ctypes.POINTER(vp)]),
        "sim_evolve_halves_list": (ctypes.c_int, [vp, ctypes.c_int, u64p, u64, u64p, u64, u64p, u64,
                                                  ctypes.POINTER(SimOpts), vp, ctypes.POINTER(vp)]),
        "sim_halves_leaf": (ctypes.c_int, [vp, ctypes.c_int, u64, vp, vp]),
        "sim_batch_create": (ctypes.c_int, [ctypes.POINTER(_Desc), ctypes.c_int, u64p, u64, ctypes.POINTER(BatchOpts),
                                            vp, ctypes.POINTER(vp)]),
        "sim_batch_run": (ctypes.c_int, [vp, vp]),
        "sim_batch_results": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), vp]),
        "sim_batch_info": (ctypes.c_int, [vp, ctypes.c_int, i32p, ctypes.POINTER(ctypes.c_double)]),
        "sim_destroy_batch": (None, [vp]),
        "sim_born_sample": (ctypes.c_int, [vp, u64, ctypes.c_int, u64, u64, u64, u64p, u64p,
                                           ctypes.POINTER(ctypes.c_double), u64p, vp]),
        "sim_amplitudes": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp]),
        "sim_stats": (ctypes.c_int, [vp, ctypes.c_int, u64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     u64p, vp]),
        "sim_select": (ctypes.c_int, [ctypes.c_int, u64, ctypes.c_int, u64, u64, u64p, u64p]),
        "sim_sample": (ctypes.c_int, [vp, u64, u64, u64, u64p, u64p, vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(SimOpts), vp]),
        "sim_status": (ctypes.c_int, [vp]),
        "sim_release_cache": (ctypes.c_int, []),
        "sim_destroy_circuit": (None, [vp]),
        "sim_destroy_cut": (None, [vp]),
        "sim_destroy_halves": (None, [vp]),
        "sim_last_error": (ctypes.c_char_p, []),
        "sim_profile_enable": (ctypes.c_int, [ctypes.c_int]),
        "sim_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), u64p, u64p, u64p, ctypes.c_int]),
        "sim_version": (ctypes.c_int, []),
        "sim_amplitudes_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp]),
        "sim_amplitudes_stats": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double),
                                                u64p, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != SIM_OK:
        raise SimError(rc, lib().sim_last_error().decode())


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    return t if isinstance(t, int) else t.data_ptr()


def _u64(a):
    if a is None:
        return None, 0
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.size


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, SimOpts):
        return ctypes.byref(opts)
    o = SimOpts()
    for k, v in opts.items():
        setattr(o, k, v)
    return ctypes.byref(o)


# ---------------------------------------------------------------------------
# C-ABI names
# ---------------------------------------------------------------------------
def sim_build_circuit(rows=0, cols=0, depth=0, seed=0, cut_row=0, gate_list=None, t_in_pool=False):
    d = _Desc(rows, cols, depth, seed, cut_row, gate_list.encode() if gate_list else None, int(t_in_pool))
    h = ctypes.c_void_p()
    _check(lib().sim_build_circuit(ctypes.byref(d), ctypes.byref(h)))
    return h.value


def sim_circuit_info(circ):
    n, d, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sim_circuit_info(circ, ctypes.byref(n), ctypes.byref(d), ctypes.byref(g)))
    return n.value, d.value, g.value


def sim_circuit_text(circ):
    ln = ctypes.c_size_t()
    _check(lib().sim_circuit_text(circ, None, 0, ctypes.byref(ln)))
    buf = ctypes.create_string_buffer(ln.value + 1)
    _check(lib().sim_circuit_text(circ, buf, ln.value + 1, ctypes.byref(ln)))
    return buf.value.decode()


def sim_cut(circ, cut_row=0):
    """Returns (plan, c, copies, n_upper, n_lower)."""
    p = ctypes.c_void_p()
    c, nu, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    copies = ctypes.c_uint64()
    _check(lib().sim_cut(circ, cut_row, ctypes.byref(p), ctypes.byref(c), ctypes.byref(copies),
                         ctypes.byref(nu), ctypes.byref(nl)))
    return p.value, c.value, copies.value, nu.value, nl.value


def sim_cut_ex(circ, cut_row=0, output_phase_cuts=False):
    """sim_cut with options; returns (plan, c, copies, n_upper, n_lower)."""
    o = SimCutOpts(int(output_phase_cuts))
    p = ctypes.c_void_p()
    c, nu, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    copies = ctypes.c_uint64()
    _check(lib().sim_cut_ex(circ, cut_row, ctypes.byref(o), ctypes.byref(p), ctypes.byref(c), ctypes.byref(copies),
                            ctypes.byref(nu), ctypes.byref(nl)))
    return p.value, c.value, copies.value, nu.value, nl.value


def sim_cut_output_phases(plan):
    """Output-sign cuts of a plan: list of (upper qubit, lower qubit)."""
    n = ctypes.c_int()
    _check(lib().sim_cut_output_phases(plan, None, 0, ctypes.byref(n)))
    arr = (ctypes.c_int32 * max(2 * n.value, 1))()
    _check(lib().sim_cut_output_phases(plan, arr, n.value, ctypes.byref(n)))
    return [tuple(arr[2 * i:2 * i + 2]) for i in range(n.value)]


def sim_cut_multi(circ, cut_rows):
    """Multi-part cut at the given rows; returns (plan, t, [c_j per boundary], [qubits per part])."""
    rows = (ctypes.c_int * len(cut_rows))(*cut_rows)
    p = ctypes.c_void_p()
    t = ctypes.c_int()
    cs = (ctypes.c_int * len(cut_rows))()
    nq = (ctypes.c_int * (len(cut_rows) + 1))()
    _check(lib().sim_cut_multi(circ, len(cut_rows), rows, ctypes.byref(p), ctypes.byref(t), cs, nq))
    return p.value, t.value, list(cs), list(nq)


def sim_multi_amplitudes(plan, precision, contraction, out, sels=None, opts=None, stream=None):
    """Amplitudes of a multi-part cut into the device tensor out ([n_{t-1}] ... [n_0]);
    sels: list with one array (or None) per part."""
    P = ctypes.POINTER(ctypes.c_uint64)
    arr, ptrs, ns = None, None, None
    keep = []
    if sels is not None:
        ptrs = (P * len(sels))()
        ns = (ctypes.c_uint64 * len(sels))()
        for i, sel in enumerate(sels):
            if sel is None:
                ptrs[i] = P()
                ns[i] = 0
            else:
                a = np.ascontiguousarray(sel, dtype=np.uint64)
                keep.append(a)
                ptrs[i] = a.ctypes.data_as(P)
                ns[i] = a.size
    _check(lib().sim_multi_amplitudes(plan, precision, contraction, ptrs, ns, _ptr(out), _opts(opts),
                                      _stream(stream)))


def sim_selftest_wait(limit_ms=100, stream=None):
    """Health check of the bounded device waits; returns the status code
    (SIM_ETIMEOUT when the machinery works)."""
    return lib().sim_selftest_wait(limit_ms, _stream(stream))


def sim_destroy_multi(plan):
    lib().sim_destroy_multi(plan)


def sim_cut_list(plan, c):
    """Returns (cuts [(layer, upper qubit, lower qubit)], N_e)."""
    arr = (ctypes.c_int32 * max(3 * c, 1))()
    ne = ctypes.c_int()
    _check(lib().sim_cut_list(plan, arr, ctypes.byref(ne)))
    return [tuple(arr[3 * m:3 * m + 3]) for m in range(c)], ne.value


def sim_plan_schedule(plan, half):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sim_plan_schedule(plan, half, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sim_plan_sparse_depth(plan, half, n_sel, mode=0):
    d = ctypes.c_int()
    _check(lib().sim_plan_sparse_depth(plan, half, int(n_sel), int(mode), ctypes.byref(d)))
    return d.value


def sim_plan_sparse_qubits(plan, half, levels):
    n = ctypes.c_int()
    _check(lib().sim_plan_sparse_qubits(plan, half, levels, ctypes.byref(n)))
    return n.value


def sim_plan_levels(plan, half):
    """Copy-tree levels of one half: array of rows (branch layer, copy bits before,
    copy bits after, fused passes)."""
    n = ctypes.c_int()
    _check(lib().sim_plan_levels(plan, half, None, 0, ctypes.byref(n)))
    out = np.zeros(4 * n.value, dtype=np.int32)
    _check(lib().sim_plan_levels(plan, half, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                                 ctypes.byref(n)))
    return out.reshape(-1, 4)


def sim_evolve_halves(plan, precision, copy_begin, copy_end, sel_u=None, sel_l=None, opts=None, stream=None):
    su, nu = _u64(sel_u)
    sl, nl = _u64(sel_l)
    P = ctypes.POINTER(ctypes.c_uint64)
    h = ctypes.c_void_p()
    _check(lib().sim_evolve_halves(plan, precision, copy_begin, copy_end,
                                   su.ctypes.data_as(P) if su is not None else None, nu,
                                   sl.ctypes.data_as(P) if sl is not None else None, nl,
                                   _opts(opts), _stream(stream), ctypes.byref(h)))
    return h.value


def sim_evolve_halves_list(plan, precision, copies, sel_u=None, sel_l=None, opts=None, stream=None):
    """sim_evolve_halves over an explicit list of distinct copy indices (leaf rows in
    list order)."""
    cp, ncp = _u64(copies)
    su, nu = _u64(sel_u)
    sl, nl = _u64(sel_l)
    P = ctypes.POINTER(ctypes.c_uint64)
    h = ctypes.c_void_p()
    _check(lib().sim_evolve_halves_list(plan, precision, cp.ctypes.data_as(P) if cp is not None else None, ncp,
                                        su.ctypes.data_as(P) if su is not None else None, nu,
                                        sl.ctypes.data_as(P) if sl is not None else None, nl,
                                        _opts(opts), _stream(stream), ctypes.byref(h)))
    return h.value


def sim_batch_create(descs, subset_idx=None, contraction=0, autotune=False, use_graph=False, stream=None):
    """descs: list of (rows, cols, depth, seed, cut_row), optionally extended by
    (gate_list text or None, t_in_pool); subset_idx: uint64 array [n_circuits, S] of
    flat amplitude indices (or None)."""
    n = len(descs)
    keep = []

    def desc(t):
        r, c, d, s, b = t[:5]
        gl = t[5] if len(t) > 5 else None
        tp = int(t[6]) if len(t) > 6 else 0
        if gl is not None:
            gl = gl.encode()
            keep.append(gl)
        return _Desc(r, c, d, s, b, gl, tp)

    arr = (_Desc * n)(*[desc(t) for t in descs])
    S = 0
    ptr = None
    if subset_idx is not None:
        subset_idx = np.ascontiguousarray(subset_idx, dtype=np.uint64)
        assert subset_idx.shape[0] == n
        S = subset_idx.shape[1]
        ptr = subset_idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    o = BatchOpts(contraction, int(autotune), int(use_graph), (ctypes.c_int * 5)())
    h = ctypes.c_void_p()
    _check(lib().sim_batch_create(arr, n, ptr, S, ctypes.byref(o), _stream(stream), ctypes.byref(h)))
    return h.value


def sim_batch_run(batch, stream=None):
    _check(lib().sim_batch_run(batch, _stream(stream)))


def sim_batch_results(batch, n_circuits, subset_n):
    """(stats [n, 4], subset amplitudes [n, subset_n] complex64); call after the
    run's stream has been synchronised."""
    st = np.zeros((n_circuits, 4), dtype=np.float64)
    sub = np.zeros((n_circuits, subset_n), dtype=np.complex64)
    _check(lib().sim_batch_results(batch, st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   sub.ctypes.data_as(ctypes.c_void_p) if subset_n else None))
    return st, sub


def sim_batch_info(batch, i):
    """({n, c, fuse, gemm kernel (0 pair, 1 single), raster group}, tuned ms)."""
    info = np.zeros(5, dtype=np.int32)
    ms = ctypes.c_double()
    _check(lib().sim_batch_info(batch, i, info.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(ms)))
    return dict(zip(("n", "c", "fuse", "single_cta", "group"), (int(x) for x in info))), ms.value


def sim_born_sample(amps, n_qubits, seed, n_samples, max_proposals, stream=None):
    """Born-rule samples of a device block of complex64 amplitudes (torch tensor or
    pointer with amps.numel()): returns (indices, proposal ordinals, xeb) where xeb =
    [linear, log, 2^n p_max]."""
    count = amps.numel()
    idx = np.zeros(n_samples, dtype=np.uint64)
    ords = np.zeros(n_samples, dtype=np.uint64)
    xeb = (ctypes.c_double * 3)()
    n = ctypes.c_uint64()
    P = ctypes.POINTER(ctypes.c_uint64)
    _check(lib().sim_born_sample(_ptr(amps), count, n_qubits, seed, n_samples, max_proposals,
                                 idx.ctypes.data_as(P), ords.ctypes.data_as(P), xeb, ctypes.byref(n),
                                 _stream(stream)))
    return idx[: n.value], ords[: n.value], np.array(xeb[:], dtype=np.float64)


def sim_destroy_batch(batch):
    lib().sim_destroy_batch(batch)


def sim_halves_leaf(halves, half, copy, out, stream=None):
    _check(lib().sim_halves_leaf(halves, half, copy, _ptr(out), _stream(stream)))


def sim_amplitudes(halves, contraction, accumulate, out, stream=None):
    """out: torch tensor (device or host) or a raw pointer."""
    _check(lib().sim_amplitudes(halves, contraction, int(accumulate), _ptr(out), _stream(stream)))


def sim_amplitudes_noalloc(halves, contraction, accumulate, out, stream=None):
    """The split contraction without library allocation: its scratch is a fixed
    SIM_NOALLOC_SCRATCH_BYTES device array; out must be device memory.  Returns
    after the work has finished."""
    _check(lib().sim_amplitudes_noalloc(halves, contraction, int(accumulate), _ptr(out), _stream(stream)))


def sim_amplitudes_stats(halves, contraction, accumulate, out, stream=None, want_hist=False):
    """sim_amplitudes into device memory plus the statistics of the written block
    (fused into the split contraction's epilogue).  Returns stats (and the histogram)."""
    st = (ctypes.c_double * 4)()
    hist = np.zeros(SIM_KS_BINS, dtype=np.uint64) if want_hist else None
    _check(lib().sim_amplitudes_stats(halves, contraction, int(accumulate), _ptr(out), st,
                                      hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if want_hist else None,
                                      _stream(stream)))
    out_st = np.array(st[:], dtype=np.float64)
    return (out_st, hist) if want_hist else out_st


def sim_stats(amps, is_c128, count, n_qubits, stream=None, want_hist=False):
    st = (ctypes.c_double * 4)()
    hist = np.zeros(SIM_KS_BINS, dtype=np.uint64) if want_hist else None
    _check(lib().sim_stats(_ptr(amps), int(is_c128), count, n_qubits, st,
                           hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if want_hist else None,
                           _stream(stream)))
    out = np.array(st[:], dtype=np.float64)
    return (out, hist) if want_hist else out


def sim_select(nq_u, n_u, nq_l, n_l, seed):
    cu = min(n_u, 1 << nq_u)
    cl = min(n_l, 1 << nq_l)
    su = np.zeros(cu, dtype=np.uint64)
    sl = np.zeros(cl, dtype=np.uint64)
    P = ctypes.POINTER(ctypes.c_uint64)
    _check(lib().sim_select(nq_u, n_u, nq_l, n_l, seed, su.ctypes.data_as(P), sl.ctypes.data_as(P)))
    return su, sl


def sim_sample(plan, n_u, n_l, seed, amps_out, nq_u, nq_l, opts=None, stream=None):
    cu = min(n_u, 1 << nq_u)
    cl = min(n_l, 1 << nq_l)
    su = np.zeros(cu, dtype=np.uint64)
    sl = np.zeros(cl, dtype=np.uint64)
    st = (ctypes.c_double * 4)()
    P = ctypes.POINTER(ctypes.c_uint64)
    _check(lib().sim_sample(plan, n_u, n_l, seed, su.ctypes.data_as(P), sl.ctypes.data_as(P), _ptr(amps_out),
                            st, _opts(opts), _stream(stream)))
    return su, sl, np.array(st[:])


def sim_status(stream=None):
    _check(lib().sim_status(_stream(stream)))


def sim_release_cache():
    _check(lib().sim_release_cache())


def sim_destroy_circuit(c):
    lib().sim_destroy_circuit(c)


def sim_destroy_cut(p):
    lib().sim_destroy_cut(p)


def sim_destroy_halves(h):
    lib().sim_destroy_halves(h)


def sim_profile_enable(on):
    _check(lib().sim_profile_enable(int(on)))


def sim_profile_read(reset=True):
    """Returns {"ms": [...], "instances": [...], "launches": [...], "h2d": B, "d2h": B} per phase."""
    ms = (ctypes.c_double * SIM_NUM_PHASES)()
    inst = (ctypes.c_uint64 * SIM_NUM_PHASES)()
    la = (ctypes.c_uint64 * SIM_NUM_PHASES)()
    by = (ctypes.c_uint64 * 2)()
    _check(lib().sim_profile_read(ms, inst, la, by, int(reset)))
    return {"ms": list(ms), "instances": list(inst), "launches": list(la), "h2d": by[0], "d2h": by[1]}


def sim_last_error():
    return lib().sim_last_error().decode()


def sim_version():
    return lib().sim_version()
