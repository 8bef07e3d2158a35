/*
 * libsim: GB300 (sm_103a) implementation of the cut-CZ partition scheme of
 * "64-qubit quantum circuit simulation" (Chen, Zhou, Xue, Yang, Guo, Guo;
 * arXiv 1802.06952).
 *
 * Every CZ that crosses the cut between the upper and lower half of a grid is
 * rewritten as P0 (x) I + P1 (x) Z (Section 2.1, Eq. 1), which turns the circuit
 * into 2^c copies of two unentangled half-circuits (Supplementary A, Eqs. 6-8).
 * The library evolves the half-circuit state vectors on the GPU and rebuilds
 * amplitudes as the complex contraction over the copy index
 *     A(x_u, x_l) = sum_k U_k[x_u] * L_k[x_l]          (Supplementary A, Eq. 8).
 *
 * Conventions
 *   - Qubit q of an R x C grid is row q / C, column q % C.  The cut lies between
 *     rows b-1 and b: the upper half holds qubits 0 .. b*C-1, the lower half the
 *     rest.  A full index is x = x_u + 2^{n_u} * x_l and qubit q is bit q.
 *   - Copy k = sum_m l_m 2^m, the cut CZs m numbered by (layer, upper qubit).
 *     Copy k applies P_{l_m} to the upper endpoint and Z^{l_m} to the lower one.
 *   - Amplitude blocks are row-major [n_sel_l][n_sel_u]:
 *       out[i_l * n_sel_u + i_u] = A(sel_u[i_u], sel_l[i_l]).
 *     Without a selection this is the full state vector in index order.
 *
 * Errors: every function returns SIM_OK or an error code and never throws or
 * aborts.  sim_last_error() gives a description of the last error raised on the
 * calling thread.  Functions taking a stream only enqueue work on it; device-side
 * failures (a wait that gave up) are reported by sim_status().
 *
 * Ownership: handles and the device buffers they hold belong to the library and
 * are released by the matching sim_destroy_* call.  Selection and output buffers
 * belong to the caller.  Streams are cudaStream_t values passed as void*; NULL is
 * the legacy default stream.
 */
#ifndef LIBSIM_SIM_H
#define LIBSIM_SIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
  SIM_OK = 0,
  SIM_EINVAL = 1,        /* invalid argument */
  SIM_ENOMEM = 2,        /* host or device allocation failed */
  SIM_ECUDA = 3,         /* a CUDA runtime or driver call failed */
  SIM_ETIMEOUT = 4,      /* a device-side wait gave up (see sim_status) */
  SIM_EUNSUPPORTED = 5   /* request outside what the library handles */
};

/* Half-state precision for sim_evolve_halves. */
enum {
  SIM_C64 = 0,        /* complex64 states, fused multi-gate sweeps, shared prefixes */
  SIM_C128_PLAIN = 1  /* complex128 states, one pass per non-diagonal gate plus one
                         combined diagonal pass per layer (Section 2.4), every copy
                         evolved on its own (Section 2.3.1) */
};

/* Contraction for sim_amplitudes. */
enum {
  SIM_SPLIT_BF16 = 0,  /* 3-term split bf16 products on tcgen05, fp32 accumulation */
  SIM_SPLIT_FP16 = 1,  /* 3-term split fp16 (power-of-two pre-scaled) on tcgen05 */
  SIM_FP64_PLAIN = 2   /* complex128 products and sums on CUDA cores */
};

typedef struct sim_circuit_s* sim_circuit;
typedef struct sim_cut_s* sim_cut_plan;
typedef struct sim_halves_s* sim_halves;
typedef struct sim_multi_s* sim_multi_plan;

/* Circuit description for sim_build_circuit.
 *   rows, cols   grid shape R x C (R*C <= 64)
 *   depth        number of layers; layer 0 is H on every qubit, layer t >= 1 uses
 *                CZ pattern ((t-1) mod 8) + 1 (Supplementary A, Eq. 3 circuit model)
 *   seed         splitmix64 seed of the X^1/2 / Y^1/2 draws
 *   cut_row      b, the row the CZ patterns 7 and 8 straddle (0 => rows / 2)
 *   gate_list    optional canonical gate-list text ("circuit R C depth seed" then
 *                one "t NAME q [q2]" line per gate, NAME in H X2 Y2 T CZ CX CT CY2;
 *                the controlled X, T and Y^1/2 gates are "t CX control target"
 *                etc.); when not NULL it replaces the generator.
 *   rule_t_in_pool  0: a qubit's first gate after H is T and later ones are X^1/2
 *                or Y^1/2 (top bit of the next splitmix64 output); 1: later ones are
 *                uniform over {X^1/2, Y^1/2, T} ((output >> 32) mod 3), a variant
 *                nearer the T share the paper reports (Sec. 3, Fig. 4); its exact
 *                rule is not printed in the paper. */
typedef struct {
  int rows, cols, depth;
  uint64_t seed;
  int cut_row;
  const char* gate_list;
  int rule_t_in_pool;
} sim_circuit_desc;

/* Tuning knobs; pass NULL for defaults.  Zero fields mean "choose automatically".
 *   fuse_qubits    local qubits staged per thread block in a fused sweep (4..13;
 *                  default 13)
 *   sweep_threads  threads per block of the staged sweep (64..256, multiple of 32)
 *   gemm_group_m   m-blocks per raster group of the persistent contraction
 *   sweep_kernel   1: staged shared-memory sweep; 0 or 2: register-blocked sweep
 *                  wherever the pass allows it (8 <= k <= 13), staged otherwise
 *   pass_order     0: dependency-aware pass formation (a gate whose qubit does not
 *                  fit is left for a later pass, together with everything that
 *                  depends on it, and the pass goes on with the rest; fewer passes);
 *                  1: in order (a pass ends at the first gate that does not fit)
 *   host_levels    1: the copy-tree level buffers of the complex64 sweeps (the
 *                  half-states a level keeps for its children, Section 2.3.2, and
 *                  the states it works on) live in pinned host memory, which the
 *                  sweep kernels read and write over NVLink-C2C; their chunk budget
 *                  is a quarter of the available host memory.  For halves whose
 *                  levels do not fit in device memory; each pass then runs at the
 *                  host link's bandwidth.  The leaves stay in device memory, and
 *                  the results are those of device-resident levels.
 *   sparse_leaves  selected entries of the complex64 leaves (a selection, not all
 *                  indices) computed from an ancestor's state instead of from
 *                  whole leaf states (Section 2.3.1: only the selected entries are
 *                  needed).  The ops of the last d copy-tree levels act
 *                  non-diagonally on a set Q of qubits (sim_plan_sparse_qubits); an
 *                  entry then needs the 2^|Q| entries of its ancestor d levels up
 *                  that agree with it outside Q, and those d levels are never
 *                  formed.  d is the largest value below the number of levels with
 *                  |Q| <= 10 and (0, the default) n_sel * 2^|Q| <= 2^n / 8, or
 *                  (1) |Q| <= 10 alone; -1: never.  Same results up to rounding
 *                  order. */
typedef struct {
  int fuse_qubits;
  int sweep_threads;
  int gemm_group_m;
  int sweep_kernel;
  int pass_order;
  int host_levels;
  int sparse_leaves;
  int reserved[1];
} sim_opts;

/* Build a circuit (Supplementary A, Eq. 3 circuit model; gate rules of the random
 * grid circuits the paper simulates, Section 3).  Host only.
 * Returns SIM_EINVAL for bad shapes or a malformed gate list. */
int sim_build_circuit(const sim_circuit_desc* desc, sim_circuit* out);

/* Number of qubits, layers and gates of a circuit.  Host only. */
int sim_circuit_info(sim_circuit circ, int* n_qubits, int* depth, int* n_gates);

/* Canonical gate-list text of the circuit (same format as desc->gate_list).
 * Writes at most cap bytes including the terminating NUL; *len_out receives the
 * full length without the NUL (call with cap = 0 to size the buffer).  Host only. */
int sim_circuit_text(sim_circuit circ, char* buf, size_t cap, size_t* len_out);

/* Cut the circuit between rows cut_row-1 and cut_row (Section 2.1; Supplementary A,
 * Eqs. 6-8): find E_int, number the cut CZs, split the gates into two half-circuits,
 * build the copy tree (one level per layer holding cuts) and the fused pass
 * schedule.  A controlled gate across the cut (explicit gate lists: controlled X,
 * controlled T, controlled Y^1/2) is cut the same way, Supplementary A, Eq. 1 with
 * U = X, T or Y^1/2: P_l on the control and U^l on the target, whichever half each
 * is in.  The fused complex64 sweeps write U^l with copy-independent gates around
 * one diagonal slot w^{b l x} on the target (w = e^{i pi/4}): X^l = H Z^l H (b = 4),
 * T^l (b = 1), (Y^1/2)^l = X^1/2 X^1/2 X^1/2 S^l X^1/2 (b = 2, in time order); the
 * plain complex128 path applies U in the copies with l = 1.  Outputs (any may be
 * NULL): c, 2^c, qubits per half.  Host only.  SIM_EUNSUPPORTED if a controlled
 * gate lies inside one half, a half exceeds 32 qubits or c exceeds 40. */
int sim_cut(sim_circuit circ, int cut_row, sim_cut_plan* out, int* c_out,
            uint64_t* copies_out, int* n_upper_out, int* n_lower_out);

/* Options of sim_cut_ex; a zero field keeps sim_cut's behaviour.
 *   output_phase_cuts  1: a cut CZ at layer t with no non-diagonal gate (X^1/2,
 *                      Y^1/2, H, controlled X) on either of its qubits after t
 *                      commutes with every later gate, so it is applied to the final
 *                      amplitudes as the sign (-1)^{x_h x_k} instead of being split
 *                      by Supplementary A, Eq. 1 into two copies: 2^c shrinks by 2
 *                      per such cut.  The amplitudes are the same; the leaves of
 *                      sim_halves_leaf then lack those CZs.  At most 32 cuts
 *                      become signs (in copy-bit order); further ones stay copy
 *                      bits.  (Not in the paper: an exact rewrite of the last cut
 *                      layers.) */
typedef struct {
  int output_phase_cuts;
  int reserved[7];
} sim_cut_opts;

/* sim_cut with options (opts may be NULL).  Same outputs and errors as sim_cut;
 * SIM_EINVAL for an unknown option value. */
int sim_cut_ex(sim_circuit circ, int cut_row, const sim_cut_opts* opts, sim_cut_plan* out, int* c_out,
               uint64_t* copies_out, int* n_upper_out, int* n_lower_out);

/* The output-sign cuts of a plan (sim_cut_ex with output_phase_cuts) as int32 pairs
 * {upper qubit, lower qubit}: every amplitude A(x) is multiplied by
 * (-1)^{sum over pairs of x_h x_k}.  Writes at most cap pairs; *n_out receives
 * their number.  Host only. */
int sim_cut_output_phases(sim_cut_plan plan, int32_t* pairs_out, int cap, int* n_out);

/* Multi-part cut (Section 3, Fig. 3): the grid is cut between rows r-1 and r for
 * every r of cut_rows (strictly increasing, inside the grid), giving t = n_cut_rows
 * + 1 row bands (parts, numbered from the top).  Every CZ across a boundary is
 * rewritten by Eq. 1: P_l on its upper qubit, Z^l on its lower one, one copy bit
 * l each; the amplitude is the sum over all boundary bits of the products of the
 * t part states.  Outputs (any may be NULL): t, the cut CZs per boundary
 * (c_out[j-1] for boundary j, n_cut_rows values) and the qubits per part (nq_out,
 * t values).  Host only.  SIM_EUNSUPPORTED if the circuit holds a controlled gate, a
 * part exceeds 32 qubits or its copy bits exceed 40. */
int sim_cut_multi(sim_circuit circ, int n_cut_rows, const int* cut_rows, sim_multi_plan* out, int* parts_out,
                  int* c_out, int* nq_out);

/* Amplitudes of a multi-part cut for the selected indices of every part: sels[p]
 * is a host array of nsel[p] distinct indices < 2^{nq[p]} (sels == NULL or
 * sels[p] == NULL: all of them in order).  Every part is evolved for each of its
 * 2^{c_p + c_{p+1}} copies (the copy tree of Section 2.3.2 over its own cut
 * layers; SIM_EUNSUPPORTED above 2^24), then the parts are contracted boundary by
 * boundary from the top, each step one contraction over that boundary's copy bits.
 *   precision, contraction   SIM_C64 with SIM_SPLIT_FP16 (complex64 out; keeps the
 *                            chained contractions within 1e-5) or SIM_SPLIT_BF16 (two
 *                            parts with at least 16 copies only: chained bf16
 *                            roundings add up past 1e-5, so three or more parts
 *                            return SIM_EUNSUPPORTED), or SIM_C128_PLAIN with
 *                            SIM_FP64_PLAIN (complex128)
 *   out_dev                  caller-owned device array [n_{t-1}] ... [n_0], row-major
 *                            (x_0 fastest); with no selection the full vector in
 *                            index order
 * Device memory: all parts' leaves, plus after part p the partial product of
 * 2^{c_{p+1}} n_p ... n_0 values.  Returns when the work has finished.
 * SIM_ENOMEM if it does not fit. */
int sim_multi_amplitudes(sim_multi_plan plan, int precision, int contraction, const uint64_t* const* sels,
                         const uint64_t* nsel, void* out_dev, const sim_opts* opts, void* stream);

void sim_destroy_multi(sim_multi_plan plan);

/* Health check of the bounded device waits.  One thread waits, with the helper
 * every contraction kernel uses for its mbarrier waits, on a fresh shared-memory
 * barrier that nothing arrives on.  It gives up after limit_ms (1 .. 10000),
 * records the timeout in the device status word and returns.  The GPU is not
 * faulted and the context stays usable.  The call waits for the stream and returns
 * what sim_status then reports: SIM_ETIMEOUT when the machinery works (the expected
 * result), after which the status word is clear again.  SIM_EINVAL for a limit
 * outside the range. */
int sim_selftest_wait(int limit_ms, void* stream);

/* The cut list as int32 triples {layer, upper qubit, lower qubit}, ordered by copy
 * bit m (3*c values).  *n_equiv_out (may be NULL) receives N_e of Section 3:
 * qubits per half + log2(number of half-circuits).  Host only. */
int sim_cut_list(sim_cut_plan plan, int32_t* cuts_out, int* n_equiv_out);

/* Fused-pass schedule summary of one half (0 upper, 1 lower) for complex64 sweeps:
 * number of copy-tree levels, number of fused passes summed over levels, and the
 * number of plain passes the Section 2.4 scheme would need for one copy (one per
 * non-diagonal gate plus one per layer holding diagonal gates).  Host only. */
/* Per copy-tree level of one half (0 upper, 1 lower): four int32 values
 * {branch layer (-1 for the root), copy bits fixed before the level, copy bits
 * fixed after it, fused passes of the level}.  A level is run once per distinct
 * value of its fixed copy bits among the evolved copies (Section 2.3.2), so the
 * work of any copy set follows from this table (Eq. (2) with n_i the passes of a
 * level and m its node count).  Writes at most cap levels; *n_levels receives the
 * number of levels.  Host only. */
int sim_plan_levels(sim_cut_plan plan, int half, int32_t* out, int cap, int* n_levels);

/* Number of qubits on which the ops of a half's last `levels` copy-tree levels act
 * non-diagonally (0 when they apply only diagonal terms): the |Q| of
 * sim_opts.sparse_leaves, whose selected leaf entries are each computed from 2^|Q|
 * entries of their ancestor `levels` levels up (Section 2.3.1; Supplementary A,
 * Eq. 1: the cut slots are diagonal).  1 <= levels < number of levels
 * (sim_plan_levels), else SIM_EINVAL.  Host only. */
int sim_plan_sparse_qubits(sim_cut_plan plan, int half, int levels, int* nq_out);

/* The number of trailing copy-tree levels of a half that sim_evolve_halves leaves
 * unformed for a selection of n_sel entries of that half under sim_opts.sparse_leaves
 * = mode (0, 1 or -1; see sim_opts): the largest d below the number of levels with
 * |Q| <= 10 (sim_plan_sparse_qubits) and, for mode 0, n_sel * 2^|Q| <= 2^n / 8; 0
 * when none qualifies, mode is -1 or n_sel covers the whole half.  Host only. */
int sim_plan_sparse_depth(sim_cut_plan plan, int half, uint64_t n_sel, int mode, int* depth_out);

int sim_plan_schedule(sim_cut_plan plan, int half, int* levels, int* fused_passes,
                      int* plain_passes);

/* Evolve both half-circuits of copies [copy_begin, copy_end) on the GPU
 * (Supplementary A, Eqs. 4-5 per half; diagonal gates combined per Section 2.4).
 *   precision    SIM_C64 or SIM_C128_PLAIN
 *   sel_u, n_u   host array of n_u distinct upper indices < 2^{n_upper}, or NULL
 *                for all of them in order (n_u is then ignored)
 *   sel_l, n_l   the same for the lower half
 *   stream       cudaStream_t on which the work is enqueued
 * The returned handle keeps, for every copy in the range, the selected entries of
 * both leaf half-states (complex64 or complex128) for sim_amplitudes.
 * SIM_ENOMEM if the device cannot hold them; SIM_EUNSUPPORTED for more than 2^26
 * copies in one call (evolve copy ranges and accumulate their contractions). */
int sim_evolve_halves(sim_cut_plan plan, int precision, uint64_t copy_begin,
                      uint64_t copy_end, const uint64_t* sel_u, uint64_t n_u,
                      const uint64_t* sel_l, uint64_t n_l, const sim_opts* opts,
                      void* stream, sim_halves* out);

/* sim_evolve_halves for an explicit list of copies instead of a range: the copy
 * tree is built over the listed copies only, so copies whose cut bits share a
 * prefix share the evolution of that prefix (Section 2.3.2).  The paper evaluates
 * the partitions independently (Supplementary B); a list lets a caller time a
 * seeded sample of them and extrapolate with Eq. (2).
 *   copies, n_copies  host array of n_copies distinct copy indices < 2^c, in the
 *                     order of the leaf rows (sim_amplitudes sums over all of them)
 * SIM_EINVAL for an empty list, an index >= 2^c or a repeated index; otherwise as
 * sim_evolve_halves. */
int sim_evolve_halves_list(sim_cut_plan plan, int precision, const uint64_t* copies,
                           uint64_t n_copies, const uint64_t* sel_u, uint64_t n_u,
                           const uint64_t* sel_l, uint64_t n_l, const sim_opts* opts,
                           void* stream, sim_halves* out);

/* Copy the selected entries of one leaf half-state (half 0 upper, 1 lower) of copy
 * `copy` (an absolute copy index among the evolved copies) into out_dev, a device
 * buffer of n_sel elements of the halves' precision (complex64 or complex128). */
int sim_halves_leaf(sim_halves h, int half, uint64_t copy, void* out_dev, void* stream);

/* Contract the halves over the copy index (Supplementary A, Eq. 8):
 *   out[i_l * n_u + i_u] (+)= sum_k U_k[sel_u[i_u]] * L_k[sel_l[i_l]]
 *   contraction  SIM_SPLIT_BF16 / SIM_SPLIT_FP16 (complex64 halves, complex64 out)
 *                or SIM_FP64_PLAIN (complex64 or complex128 halves, complex128 out)
 *   accumulate   0: overwrite out; 1: add into out (sums over copy batches)
 *   out          caller-owned buffer of n_l * n_u complex values, device memory or
 *                host memory (a host buffer is filled through a device staging
 *                buffer; the call then returns after the copy has finished).
 * Accuracy of the split contractions: each product U_k L_k is off by at most
 * 3 * 2^-(2p+2) |U_k| |L_k| (p = 7 mantissa bits for bf16, 10 for fp16) plus the
 * fp32 accumulation.  SIM_SPLIT_FP16 (2^-22 per product) keeps max|dA| / max|A|
 * within 1e-5 for any number of copies.  The bf16 bound (4.6e-5 for one product)
 * is averaged below 1e-5 only by summing many copies, so SIM_SPLIT_BF16 is
 * refused with SIM_EUNSUPPORTED when the halves hold fewer than 16 copies
 * (whatever accumulate says: accumulate copy batches with SIM_SPLIT_FP16). */
int sim_amplitudes(sim_halves h, int contraction, int accumulate, void* out, void* stream);

/* sim_amplitudes without allocation: the same split-precision tensor-core
 * contraction (SIM_SPLIT_BF16 or SIM_SPLIT_FP16 only) for callers that cannot let
 * the library allocate device memory while they run: an application whose device
 * memory already belongs to its own allocator, or a latency-bound loop that cannot
 * afford cudaMalloc / cudaFree (they can block the host and synchronise the
 * device).  The paper has no counterpart; this is a deployment variant.
 *   h, contraction, accumulate   as for sim_amplitudes (the same split-bf16 rule)
 *   out_dev   caller-owned DEVICE buffer of n_l * n_u complex64 values on the
 *             current device (a buffer of another device returns SIM_EINVAL)
 * Scratch: a fixed device array of SIM_NOALLOC_SCRATCH_BYTES inside the library
 * (the two split copies of both operands, 4 * (n_l + 2 n_u) * kpad bytes with
 * kpad = 2K rounded up to 64, plus 1 KiB).  Larger requests return SIM_EINVAL
 * with the number of bytes they would need.
 * When the array comes into being: it belongs to the library's CUDA module, which
 * the runtime loads into a device's context lazily by default, at this function's
 * first call on that device (the call that looks up the array's device address
 * with cudaGetSymbolAddress, with that device current).  That first call
 * therefore reserves the SIM_NOALLOC_SCRATCH_BYTES of device memory itself: make
 * it before the application's allocator takes the device's memory.  Under
 * CUDA_MODULE_LOADING=EAGER every context that loads the library holds the array
 * from the start, whether or not this function is called.  Every GPU that holds
 * the array keeps it until the process exits.
 * All calls share the array and it keeps the previous call's contents: calls whose
 * work can overlap on the GPU (other streams, other host threads) race on it and
 * must be serialised by the caller.  Every call synchronises the stream and reads
 * a status word back from the device, so it cannot be called while the stream is
 * being captured into a CUDA graph.  It returns SIM_ETIMEOUT if a bounded device
 * wait gave up.  It never calls cudaMalloc, cudaFree or an allocating library
 * routine. */
#define SIM_NOALLOC_SCRATCH_BYTES (32u << 20)
int sim_amplitudes_noalloc(sim_halves h, int contraction, int accumulate, void* out_dev,
                           void* stream);

/* Statistics of an amplitude block (Section 3, Eq. 7 with alpha = 1), summed in
 * FP64.  With w = 2^n |A|^2 and z = ln w, Eq. 7 is the density exp(z - e^z) whose
 * CDF is F(z) = 1 - exp(-w); u = F(z) is uniform on [0, 1) under that law.
 * stats_out = {sum |A|^2, mean w, mean ln w over entries with w > 0,
 * KS distance max_b |G(u_b) - u_b| between the empirical CDF G of u and the
 * uniform CDF at the SIM_KS_BINS bin edges u_b = (b+1) / SIM_KS_BINS}.
 * amps is device memory, complex64 (is_c128 = 0; per-entry work in fp32) or
 * complex128 (is_c128 = 1; FP64 throughout).  hist_out (may be NULL) receives the
 * SIM_KS_BINS counts of u.  Synchronises the stream. */
#define SIM_KS_BINS 4096
int sim_stats(const void* amps, int is_c128, uint64_t count, int n_qubits,
              double stats_out[4], uint64_t* hist_out, void* stream);

/* sim_amplitudes followed by the statistics of sim_stats over the n_l * n_u values
 * it wrote (the accumulated values when accumulate = 1), with n the circuit's qubit
 * count.  For the split contractions the statistics are computed inside the
 * contraction's epilogue from the fp32 results, so the amplitudes are not read
 * back from memory.  out must be device memory.  Synchronises the stream. */
int sim_amplitudes_stats(sim_halves h, int contraction, int accumulate, void* out_dev,
                         double stats_out[4], uint64_t* hist_out, void* stream);

/* Draw the amplitude selection used by sim_sample (Section 3: "sampling" of state
 * components): n_u distinct upper indices of [0, 2^{nq_u}), then n_l distinct lower
 * indices of [0, 2^{nq_l}), each set by Floyd's algorithm from one splitmix64(seed)
 * stream (draw t = next() mod (j+1)) and sorted ascending.  n >= 2^nq gives all
 * indices.  Host only; outputs are caller-owned host arrays. */
int sim_select(int nq_u, uint64_t n_u, int nq_l, uint64_t n_l, uint64_t seed,
               uint64_t* sel_u_out, uint64_t* sel_l_out);

/* Selection + evolution + split-fp16 contraction + statistics in one call:
 * draws the selection (sim_select), evolves all copies in complex64, writes the
 * [n_l][n_u] complex64 block to amps_dev_out (caller-owned device memory) and the
 * statistics to stats_out (may be NULL).  Synchronises the stream. */
int sim_sample(sim_cut_plan plan, uint64_t n_u, uint64_t n_l, uint64_t seed,
               uint64_t* sel_u_out, uint64_t* sel_l_out, void* amps_dev_out,
               double stats_out[4], const sim_opts* opts, void* stream);

/* Synchronise the stream and report device-side failures recorded since the last
 * call: SIM_ETIMEOUT if a kernel's bounded wait gave up, SIM_ECUDA on a CUDA error. */
int sim_status(void* stream);

/* Release cached device memory held by the library's pool. */
int sim_release_cache(void);

/* Phase profiler.  While enabled, every library call that launches kernels records
 * a CUDA event pair around each phase on the stream it launches on, and counts the
 * kernels it launches and the bytes it copies between host and device.
 * sim_profile_read synchronises the recorded events and returns, per phase, the
 * summed device milliseconds, the number of phase instances (event pairs) and the
 * number of kernel launches; bytes_out (may be NULL) receives {host->device,
 * device->host} bytes.  reset != 0 clears all counters afterwards. */
enum {
  SIM_PHASE_SWEEP = 0,     /* fused complex64 gate sweeps of the copy tree */
  SIM_PHASE_GATHER = 1,    /* selection gather of leaf states */
  SIM_PHASE_PLAIN = 2,     /* plain complex128 per-gate passes */
  SIM_PHASE_PACK = 3,      /* split-pack of the contraction operands */
  SIM_PHASE_CONTRACT = 4,  /* tcgen05 split contraction */
  SIM_PHASE_FP64_GEMM = 5, /* plain FP64 contraction */
  SIM_PHASE_STATS = 6,     /* FP64 statistics */
  SIM_NUM_PHASES = 7
};
int sim_profile_enable(int on);
int sim_profile_read(double* ms_out, uint64_t* instances_out, uint64_t* launches_out,
                     uint64_t* bytes_out, int reset);

/* Born-rule samples of measurement outcomes (Section 3: measurement outcomes of the
 * full vector space) from a block of amplitudes, by rejection sampling with a
 * measured bound, and their cross-entropy statistics against Eq. 7.
 *   amps_dev       device array of count complex64 amplitudes (for example the
 *                  output of sim_amplitudes; with no selection its flat index is
 *                  the bitstring x = x_u + 2^{n_u} x_l)
 *   n_qubits       n of w = 2^n |A|^2
 *   seed           proposal c draws i_c = r_{2c} mod count and u_c =
 *                  (r_{2c+1} >> 11) 2^-53 from the counter-based splitmix64 stream r
 *                  of the seed (output c: state seed + (c+1) 0x9E3779B97F4A7C15,
 *                  then the published finaliser); it is accepted when
 *                  u_c p_max < p_{i_c}, p = |A|^2 in FP64, p_max the block's maximum
 *   n_samples      samples wanted; max_proposals caps the proposals drawn
 *   idx_out        host array of n_samples: the accepted indices, in proposal order
 *   ordinal_out    host array of n_samples (or NULL): the proposal number c of each
 *   xeb_out        {mean w - 1, mean ln w + Euler's gamma, 2^n p_max}: both
 *                  statistics are 1 for Born samples of Eq. 7 (alpha = 1) and 0 for
 *                  uniform samples
 *   n_out          samples produced (fewer than n_samples if max_proposals ran out)
 * The accepted indices follow p / sum(p) over the block.  Returns after the work
 * has finished.  SIM_EINVAL for empty or NULL arguments. */
int sim_born_sample(const void* amps_dev, uint64_t count, int n_qubits, uint64_t seed, uint64_t n_samples,
                    uint64_t max_proposals, uint64_t* idx_out, uint64_t* ordinal_out, double xeb_out[3],
                    uint64_t* n_out, void* stream);

/* ---- Batches of circuits ------------------------------------------------------
 * Many circuits of different sizes and cuts, each evaluated in full (all copies,
 * all 2^n amplitudes) into one output buffer that the circuits reuse in turn.  The
 * paper evaluates one circuit at a time; a batch keeps the GPU busy across many
 * small ones: everything is planned and allocated at creation, so a run is a pure
 * sequence of kernel launches that can be captured once into a CUDA graph. */
typedef struct sim_batch_s* sim_batch;

/* Batch options (NULL: defaults; zero fields mean the default).
 *   contraction  SIM_SPLIT_BF16 (default; refused with SIM_EUNSUPPORTED at
 *                creation if a circuit has fewer than 16 copies) or SIM_SPLIT_FP16
 *   autotune     0: fixed choices (fused-pass width 13, CTA-pair contraction with
 *                raster groups of 32); 1: for each circuit shape (rows, cols, cut
 *                row, cut CZs c), time fuse widths 10..13 and three contraction tile
 *                variants on its first circuit and keep the fastest
 *   use_graph    1: the second sim_batch_run captures the batch into a CUDA graph
 *                (the first one runs uncaptured and initialises every kernel);
 *                later runs launch the graph */
typedef struct {
  int contraction;
  int autotune;
  int use_graph;
  int reserved[5];
} sim_batch_opts;

/* Build, cut and schedule every circuit (host), autotune if asked (device work on
 * stream, which is synchronised), allocate the buffers for the largest circuit and
 * upload the op and node tables.
 *   descs, n_circuits  circuit descriptions (sim_build_circuit); cut_row 0 means
 *                      the middle row
 *   subset_idx         host array [n_circuits][subset_n] of flat amplitude indices
 *                      x = x_u + 2^{n_u} x_l (< 2^n of that circuit), or NULL when
 *                      subset_n is 0; each run gathers those amplitudes
 * SIM_EINVAL on a bad description or index; SIM_ENOMEM if the buffers do not fit;
 * SIM_EUNSUPPORTED for circuits above 34 qubits (full vectors). */
int sim_batch_create(const sim_circuit_desc* descs, int n_circuits, const uint64_t* subset_idx,
                     uint64_t subset_n, const sim_batch_opts* opts, void* stream, sim_batch* out);

/* Enqueue one evaluation of the whole batch on stream: per circuit the sweeps of
 * both halves, the split-pack, the tensor-core contraction into the shared output
 * buffer with the statistics fused into it, and the subset gather.  No host
 * synchronisation and no allocation; the batch's buffers are reused, so runs must
 * not overlap. */
int sim_batch_run(sim_batch b, void* stream);

/* After a run has finished (the caller synchronises its stream), per circuit i:
 * stats_out[4i .. 4i+3] = {sum |A|^2, mean 2^n |A|^2, mean ln 2^n |A|^2, KS
 * distance to Eq. 7} over all 2^n amplitudes, and subset_out[i * subset_n + j] =
 * A_i(subset_idx[i][j]) as complex64 (host memory).  Either may be NULL. */
int sim_batch_results(sim_batch b, double* stats_out, void* subset_out);

/* Circuit i of the batch: {qubits, cut CZs c, fuse width, contraction kernel
 * (0 CTA pair, 1 single CTA), raster group} and the autotuner's time in ms of
 * the chosen sweep + contraction of that shape (0 when not tuned on this circuit). */
int sim_batch_info(sim_batch b, int i, int32_t info_out[5], double* tuned_ms);

void sim_destroy_batch(sim_batch b);

void sim_destroy_circuit(sim_circuit circ);
void sim_destroy_cut(sim_cut_plan plan);
void sim_destroy_halves(sim_halves h);

/* Description of the last error on the calling thread ("" if none). */
const char* sim_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int sim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBSIM_SIM_H */
