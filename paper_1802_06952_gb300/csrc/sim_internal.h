// Internal declarations shared by the host code and the CUDA kernels of libsim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

struct sim_halves_s;

namespace sim {

// One-time set-up per device.  Function attributes (the dynamic shared-memory
// opt-in) and occupancy answers belong to a device's context, so a process that
// launches on several devices sets each one up with that device current.
// run(fn) calls fn(value) once per device ordinal under a lock and caches the int
// it writes; later calls on that device return the cached value.
constexpr int kMaxDeviceSlots = 64;
struct DeviceOnce {
  std::mutex mu;
  bool done[kMaxDeviceSlots] = {};
  int value[kMaxDeviceSlots] = {};
  template <class F>
  cudaError_t run(F&& fn, int* value_out = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDeviceSlots) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
      int v = 0;
      e = fn(v);
      if (e != cudaSuccess) return e;
      value[dev] = v;
      done[dev] = true;
    }
    if (value_out) *value_out = value[dev];
    return cudaSuccess;
  }
};

// ---------------------------------------------------------------------------
// Circuit IR (Supplementary A, Eq. 3: layers of single-qubit gates and CZ edges)
// ---------------------------------------------------------------------------
// G_CX, G_CT, G_CY2: controlled X, T and Y^1/2, q1 control, q2 target (only across
// the cut, where each becomes P_l on the control and U^l on the target:
// Supplementary A, Eq. 1 with U = X, T, Y^1/2); G_X: the X of a controlled-X slot
// (not a gate of the circuit text)
enum GateCode : int { G_H = 0, G_X2 = 1, G_Y2 = 2, G_T = 3, G_CZ = 4, G_CX = 5, G_X = 6, G_CT = 7, G_CY2 = 8 };
inline bool is_two_qubit(int code) { return code == G_CZ || code == G_CX || code == G_CT || code == G_CY2; }
inline bool is_controlled_u(int code) { return code == G_CX || code == G_CT || code == G_CY2; }

struct Gate {
  int t, code, q1, q2;
};

struct Circuit {
  int R = 0, C = 0, depth = 0, cut_row = 0;
  uint64_t seed = 0;
  int n = 0;
  std::vector<Gate> gates;  // ordered by layer, then first qubit
};

// ---------------------------------------------------------------------------
// Device op records of the fused complex64 sweeps and the plain complex128 path
// ---------------------------------------------------------------------------
// OP_SWAP (register-blocked sweep only): exchange the data of warp ranks 5+m with
// register ranks 10+m (m < min(3, R-2)) so that the qubits at those warp ranks
// become register qubits; the staged sweep ignores it (its layout never moves).
enum OpType : int { OP_GATE = 0, OP_DIAG = 1, OP_SWAP = 2 };
constexpr int kMaxShift = 6;   // CZ shift classes per diagonal op
constexpr int kMaxCutSlots = 16;

// One op of a pass.  A GATE is a 2x2 complex matrix on local bit `lq` (fused
// path) or on qubit `q` (plain path).  A DIAG is the combined diagonal of one
// layer (Section 2.4, Eqs. 4 and 6) plus the copy-dependent cut slots:
//   phase(x) = w^{popc(x & tmask)} * (-1)^{sum_s popc(x & (x >> sh_d[s]) & sh_m[s])}
//   slot i with bit i of cutz clear:  * [bit cutq[i] of x == bit cutm[i] of the copy id]    (P_l)
//   slot i with bit i of cutz set:    * w^{cutw[i] * bit cutq[i] of x * bit cutm[i] of the copy id}
// with w = e^{i pi / 4}.  P_l sits on the upper end of a cut CZ and on the control
// of a cut controlled gate (in either half); the phase slots on the lower end of a
// cut CZ (cutw = 4: Z^l) and on the target of a cut controlled T (1: T^l), and
// between the copy-independent gates that write X^l (4) and (Y^1/2)^l (2).
struct OpRec {
  int32_t type;
  int32_t lq;
  int32_t q;
  int32_t nsh;
  int32_t ncut;
  uint32_t cutz;
  uint32_t tmask;
  int32_t kind;          // GATE: 0 general 2x2, 1 X^1/2, 2 Y^1/2, 3 H, 4 X (closed-form updates)
  int32_t cond;          // GATE: -1, or copy bit m: applied only where l_m = 1 (the X^l slot
                         // of the plain path; fused passes take H Z^l H instead)
  uint32_t sh_d[kMaxShift];
  uint32_t sh_m[kMaxShift];
  uint8_t cutq[kMaxCutSlots];
  uint8_t cutm[kMaxCutSlots];
  uint8_t cutw[kMaxCutSlots];  // phase slots: exponent weight of w (1..7)
  float m[8];
  double md[8];
  // DIAG in the register-blocked sweep (set per pass by the scheduler): with x the
  // thread part of the index plus the register part r(j) of element j,
  //   ereg: exponent (mod 8) of the T and CZ terms within the register qubits,
  //         4 bits per j (entry j at bits 4(j % 8) of ereg[j / 8])
  //   pq[r]: the non-register CZ partner qubit of register rank r (0xFF: none)
  uint32_t ereg[4];
  uint8_t pq[8];
  // register-blocked sweep, per op with the rank -> qubit map at that op:
  //   GATE: lq is the current rank of q, lq0 its rank in the pass's initial order
  //         (the staged sweep's layout)
  //   DIAG: rq[r] the qubit at register rank 8 + r, regmask their mask
  //   SWAP: tq[r] the qubit at thread rank r (r < 8) after the exchange
  int32_t lq0;
  uint32_t regmask;
  uint8_t rq[8];
  uint8_t tq[8];
  // DIAG: 1 when every exponent of the op is 0 or 4 (no T, no phase slot of weight
  // other than 4): the register-blocked sweep then flips signs instead of
  // multiplying by w^e
  int32_t sign_only;
};

// At most this many ops per fused pass (the register-blocked sweep copies a pass's
// ops into shared memory).
constexpr int kMaxPassOps = 64;

// One fused pass: stage 2^k amplitudes whose local bits are `local_mask`, run
// ops [op_begin, op_begin + op_count), write back.
enum PassSrc : int { SRC_SELF = 0, SRC_PARENT = 1, SRC_UNIFORM = 2, SRC_ZERO = 3 };

struct PassDesc {
  int k;
  int low;              // low bits 0..low-1 are local (coalesced global rows)
  uint32_t local_mask;
  int op_begin, op_count;
  int src;
  // qubit held by each local rank r (bit r of the staged index): ranks 0..low-1
  // are qubits 0..low-1; with k >= 8 ranks 5..7 are the warp bits and ranks
  // 8..k-1 the register bits of the register-blocked sweep, which take the qubits
  // with the most gates in the pass
  uint8_t order[16];
  int warp_gates;       // gates of the pass on warp-bit ranks (need a smem exchange)
  int general_gates;    // gates of the pass without a closed-form update (kind 0)
  // The register-blocked sweep applies X^1/2, Y^1/2 and H without their common
  // factors ((1+i)/2, (1+i)/2, 1/sqrt2): scale = 2^(-(n_xy + n_h)/2) is applied when
  // the pass stores, and the phase w^(n_xy) (w = e^{i pi/4}) is added to the exponent
  // of diagonal op phase_op of the pass (relative index; -1: applied at the store).
  float scale;
  int phase_e;
  int phase_op;
  // register-blocked sweep with k >= 8: `order` is the compute order (lane ranks
  // 0..4 may be any qubits); `sorder` is the storage order used for the global
  // loads and stores (ranks 0..4 = qubits 0..4, coalesced); `swz[r]` is the 4-bit
  // XOR mask storage rank r adds to the low bits of the shared-memory slot so
  // both orders read and write shared memory without bank conflicts
  uint8_t sorder[16];
  uint8_t swz[16];
  // register-blocked sweep with k >= 10: register ranks 8 and 9 hold qubits 0 and 1,
  // so each thread's elements come in runs of 4 consecutive amplitudes (32 bytes)
  // loaded and stored with one 256-bit access each; any qubits can then be lanes,
  // and the compute order is also the load order (no transposes)
  int vec4;
  int transpose;        // compute order differs from storage order
};

// One level of the copy tree of a half: nodes share all gates up to the branch
// layer; a level-j node id is the copy index masked to its low `bits_total` bits.
struct Level {
  int branch_layer;     // layer whose cut slots this level applies first (-1: root)
  int bits_before;      // copy bits fixed by earlier levels
  int bits_total;       // bits fixed up to and including this level
  std::vector<PassDesc> passes;
};

struct HalfSchedule {
  int n = 0;                     // qubits in the half
  std::vector<Level> levels;
  std::vector<OpRec> ops;        // all ops of all passes
  int plain_passes = 0;          // Section 2.4 pass count per copy (for reports)
};

// Per-layer description of a half for the plain complex128 path.
struct PlainLayer {
  std::vector<OpRec> gates;      // GATE ops with q set
  std::vector<OpRec> diags;      // DIAG ops (0 or more, cut slots included)
};

struct CutCZ {
  int t, h, k;  // layer, upper qubit, lower qubit (global indices)
  int kind = 0;  // 0 CZ; 1 controlled gate with the control in the upper half; 2 control in the lower half
  int code = G_CZ;  // gate code (G_CZ, G_CX, G_CT, G_CY2)
};

struct CutPlan {
  Circuit circ;
  int n_u = 0, n_l = 0, c = 0;
  std::vector<CutCZ> cuts;
  HalfSchedule sched[2];
  std::vector<PlainLayer> plain[2];
  int fuse_qubits = 0;
  int pass_order = 0;
  // output-phase cuts: (upper qubit, lower qubit) of each cut CZ applied as the sign
  // (-1)^{x_h x_k} of the final amplitudes instead of a copy bit
  bool out_phase_cuts = false;
  std::vector<std::pair<int, int>> out_cz;
  // device copies of the op tables (uploaded lazily, freed with the plan)
  OpRec* d_ops[2] = {nullptr, nullptr};
  OpRec* d_plain_ops[2] = {nullptr, nullptr};
  void* ops_stream = nullptr;  // cudaStream_t of the last evolve that used the tables
  std::vector<int> plain_op_offsets[2];  // per layer: first op index (gates then diags)
  std::vector<OpRec> plain_flat[2];       // host copy of the uploaded plain op table
  int device = -1;
};

// Multi-part cut (Section 3, Fig. 3): the grid cut into row bands; every CZ across
// a band boundary is rewritten by Eq. 1 (P_l on its upper qubit, Z^l on its lower
// one).  Part p carries the Z^l slots of boundary p (above it) and the P_l slots of
// boundary p + 1 (below it); its copy bits number its slots by (layer, upper
// qubit), so that its copy tree branches at its own slot layers.
struct MultiPlan {
  Circuit circ;
  int t = 0;                        // parts
  std::vector<int> offset, nq;      // first global qubit and qubit count per part
  std::vector<int> c;               // cut CZs per boundary j = 1 .. t-1 (c[0] = 0)
  // per part, per local copy bit: (boundary, bit within that boundary)
  std::vector<std::vector<std::pair<int, int>>> slot_bits;
  std::vector<CutPlan> part;        // part p as half 0 (sched[0], plain[0], n_u = nq[p])
};
std::string build_multi_plan(const Circuit& c, const std::vector<int>& cut_rows, int fuse_qubits, int pass_order,
                             MultiPlan& mp);

// Read-only view of an evolved-halves handle (defined in api.cpp), for entry
// points kept in other files; returns false for a NULL handle.
struct HalvesView {
  int precision;
  uint64_t K;  // copies held (leaf rows)
  int64_t nsel[2];
  const void* leafsel[2];
  const uint32_t* out_code[2];  // output-phase codes of the upper / lower selection (NULL: none)
};
bool halves_view(const sim_halves_s* h, HalvesView* v);
// Sets the thread's last-error text and returns code.
int set_error(int code, const std::string& msg);

// Accuracy rule of the split-bf16 contraction.  Each bf16 hi/lo pair keeps a
// residual of up to 2^-17 of its value, so one product U_k L_k can be off by
// 3 * 2^-16 |U_k| |L_k| (4.6e-5 relative): only a sum over many copies, whose
// rounding errors do not line up, stays within 1e-5 of max |A|.  Split-bf16 is
// therefore refused (SIM_EUNSUPPORTED, naming SIM_SPLIT_FP16, whose residual is
// 2^-22) for fewer than kBf16MinCopies copies in one contraction and for chained
// contractions (multi-part sums of three or more parts), whose roundings add up.
constexpr int64_t kBf16MinCopies = 16;
int check_split_bf16(int contraction, int64_t copies, bool chained);

// Phase profiler hooks (api.cpp): kernel launch and host<->device byte counters.
void note_launches(int phase, int count);
void note_bytes(uint64_t h2d, uint64_t d2h);

// Host logic (host.cpp)
std::string generate_circuit(int R, int C, int depth, uint64_t seed, int cut_row, Circuit& out, int t_in_pool = 0);
std::string parse_circuit(const char* text, Circuit& out);
std::string circuit_text(const Circuit& c);
// pass_order: 0 dependency-aware pass formation, 1 in order (sim_opts.pass_order);
// out_phase_cuts: cut CZs with no later non-diagonal gate on their qubits become
// output signs instead of copy bits (sim_cut_opts.output_phase_cuts)
std::string build_cut_plan(const Circuit& c, int cut_row, int fuse_qubits, CutPlan& plan, int pass_order = 0,
                           bool out_phase_cuts = false);
void select_indices(int nq, uint64_t count, uint64_t& state, std::vector<uint64_t>& out);
uint64_t splitmix64_next(uint64_t& state);

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files); all enqueue on `stream`.
// ---------------------------------------------------------------------------
struct NodeEntry {
  uint64_t node_id;     // copy bits fixed so far (selects cut-slot values)
  int64_t parent_slot;  // slot of the parent in the parent level buffer
  int64_t dst_row;      // row of the destination buffer
};

struct SweepLaunch {
  int n, k, low;
  uint32_t local_mask;
  const OpRec* ops;       // device pointer to the pass's first op
  int op_count;
  int src;                // PassSrc
  const NodeEntry* nodes; // device node table for this launch
  int64_t nslots;
  const void* src_base;   // parent level buffer (SRC_PARENT) or the own buffer
  void* dst_base;
  int threads;
  uint8_t order[16];      // qubit of each local rank (PassDesc::order)
  int warp_gates;
  int general_gates;
  float scale;
  int phase_e, phase_op;  // PassDesc::phase_e, phase_op
  uint8_t sorder[16];     // PassDesc::sorder, swz, transpose, vec4
  uint8_t swz[16];
  int transpose;
  int vec4;
};
// staged-block sweep (any k, any threads)
cudaError_t launch_sweep_c64(const SweepLaunch& L, cudaStream_t s);
// register-blocked sweep (k in 8..13, low == 5): preferred when supported
bool sweep2_supported(const SweepLaunch& L);
cudaError_t launch_sweep2_c64(const SweepLaunch& L, cudaStream_t s);

struct PlainLaunch {
  int n;
  int q;                  // target qubit of a GATE (host copy of op->q)
  const OpRec* op;        // one GATE or DIAG op (device)
  const uint64_t* copy_ids;  // device: copy index of each state in the batch
  int64_t nstates;
  void* psi;              // nstates x 2^n complex128
};
cudaError_t launch_plain_gate(const PlainLaunch& L, cudaStream_t s);
cudaError_t launch_plain_diag(const PlainLaunch& L, cudaStream_t s);
cudaError_t launch_plain_init_zero(void* psi, int n, int64_t nstates, cudaStream_t s);

// leafsel[row][i] = src[slot][sel[i]] for each slot of a node table (rows = dst_row)
cudaError_t launch_gather(const void* src, int n, const NodeEntry* nodes, int64_t nslots,
                          const uint64_t* sel, int64_t nsel, void* dst, int is_c128,
                          cudaStream_t s);

// Split-pack (complex64 leaves [K][nsel] -> K-major split operands).
//   A-operand (lower half, rows = n_sel_l):  row m: cols 2k, 2k+1 = (re, im) of L_k[m]
//   B-operand (upper half, rows = 2 n_sel_u): row 2j: (re, -im), row 2j+1: (im, re)
// hi = round(v * scale), lo = round(v * scale - hi) in bf16 or fp16; scale_dev is a
// device float (NULL: 1).
cudaError_t launch_pack_a(const void* leaves, int64_t K, int64_t nsel, int64_t kpad,
                          int fp16, const float* scale_dev, void* hi, void* lo, cudaStream_t s);
cudaError_t launch_pack_b(const void* leaves, int64_t K, int64_t nsel, int64_t kpad,
                          int fp16, const float* scale_dev, void* hi, void* lo, cudaStream_t s);
// out_dev[0] = max |re|, |im| over a complex64 array; out_dev[1] = the power-of-two
// fp16 pre-scale derived from it
cudaError_t launch_absmax_c64(const void* x, int64_t count, float* out_dev, cudaStream_t s);
// dst[i] = src[idx[i]] for n complex64 values (a flat-index gather of amplitudes)
cudaError_t launch_gather_flat_c64(const void* src, const uint64_t* idx, int64_t n, void* dst, cudaStream_t s);

// Selected entries of leaf half-states computed from their parents (the leaf level's
// ops are non-diagonal on the nq qubits qpos only): for each leaf node and selected
// index, the 2^nq parent entries that agree with it outside those qubits, the
// level's ops on them, and the entry at its own bits; replaces the leaf level's
// passes and the gather.
constexpr int kMaxSparseQ = 10;
struct SparseLeafLaunch {
  int n, nq;
  uint8_t qpos[kMaxSparseQ];
  const OpRec* ops;           // device ops of the leaf level's passes, in order
  int op_count;
  const NodeEntry* nodes;     // node_id, parent_slot, dst_row = leaf row
  int64_t nslots;
  const void* parent_base;    // complex64 parent states, slot stride 2^n
  const uint64_t* sel;        // device selection
  int64_t nsel;
  void* leafsel;              // complex64 [row][nsel]
};
cudaError_t launch_sparse_leaf(const SparseLeafLaunch& L, cudaStream_t s);

// tcgen05 contraction: C[M][2N] fp32 (= complex64 [M][N]) (+)= sum over 3 split
// segments of A_seg[M][kpad] * B_seg[2N][kpad]^T.
struct TcGemmArgs {
  const void* a_hi; const void* a_lo; const void* b_hi; const void* b_lo;
  int64_t M, N2, kpad;    // N2 = 2 * n_sel_u
  int fp16;
  const float* scale_a;   // device pre-scales of A and B (NULL: 1); output / (sa * sb)
  const float* scale_b;
  int accumulate;
  void* C;
  int group_m;
  int num_sms;
  int* d_status;          // device word, set non-zero if a wait gave up
  // optional fused statistics (both NULL: none); the caller zeroes them first
  float w_scale = 1.f;            // 2^n
  double* st_acc = nullptr;       // [sum |A|^2, sum ln 2^n|A|^2 over |A| > 0, count]
  unsigned long long* st_hist = nullptr;  // SIM_KS_BINS counts of u = 1 - exp(-2^n |A|^2)
  // 0: the CTA-pair kernel where it applies (SIM_TC_PAIR=0 in the environment
  // selects the single-CTA one); 1: single-CTA kernel; 2: CTA-pair kernel where it
  // applies (16-byte output rows), the single-CTA kernel otherwise
  int variant = 0;
  // output-phase cuts (both NULL: none): entry (r, c) of the block is multiplied by
  // (-1)^{popc(out_lcode[r] & out_ucode[c])}, c the complex column (< N2 / 2); an
  // accumulated block gets the sign on this contraction's part only
  const uint32_t* out_lcode = nullptr;
  const uint32_t* out_ucode = nullptr;
};
cudaError_t launch_tc_gemm(const TcGemmArgs& a, cudaStream_t s);
// CTA-pair variant of the same contraction (tcgen05 cta_group::2, M = 256 per pair)
bool tc_gemm_pair_enabled();
bool tc_gemm_pair_supported(const TcGemmArgs& a);
cudaError_t launch_tc_gemm_pair(const TcGemmArgs& a, cudaStream_t s);
// values written to *d_status when a bounded wait of the contraction gives up
constexpr int SIM_TIMEOUT_CODE_TMA = 0x101;
constexpr int SIM_TIMEOUT_CODE_MMA = 0x102;
constexpr int SIM_TIMEOUT_CODE_EPI = 0x103;
constexpr int SIM_TIMEOUT_CODE_SELFTEST = 0x104;
// the health check of the bounded waits (sim_selftest_wait)
cudaError_t launch_wait_selftest(int* d_status, unsigned long long limit_ns, cudaStream_t s);

// Plain FP64 contraction C[M][N] (+)= sum_k Lsel[k][m] * Usel[k][j] (complex128 out)
cudaError_t launch_fp64_gemm(const void* lsel, const void* usel, int in_c128, int64_t K,
                             int64_t M, int64_t N, int accumulate, void* C, cudaStream_t s);

// Output-phase cuts (phase.cu): out[i] = bit m set where index x = sel[i] (or i
// when sel is NULL) has bit qubits[m], m < nm <= 32; and the sign flip of an
// M x N complex64 (is_c128 = 0) or complex128 block by the parity of
// lcode[row] & ucode[column]
cudaError_t launch_out_codes(const uint64_t* sel, int64_t n, const int* qubits, int nm, uint32_t* out,
                             cudaStream_t s);
cudaError_t launch_out_sign(void* C, int is_c128, int64_t M, int64_t N, const uint32_t* lcode, const uint32_t* ucode,
                            cudaStream_t s);

// FP64 statistics over an amplitude block: acc[0] = sum p, acc[1] = sum ln w over
// p > 0, acc[2] = number of p > 0 (as double); hist[SIM_KS_BINS] counts.
cudaError_t launch_stats(const void* amps, int is_c128, uint64_t count, int nq,
                         double* acc_dev, unsigned long long* hist_dev, cudaStream_t s);

}  // namespace sim
