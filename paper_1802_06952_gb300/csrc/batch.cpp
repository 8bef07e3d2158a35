// Batches of circuits of different sizes and cuts, each evaluated in full (all
// copies, all amplitudes) into one reused output buffer.
//
// Everything a batch needs is planned and allocated when it is created: the
// circuits, their cuts and pass schedules, the copy-tree programs of both halves
// (Section 2.3.2), the level, leaf and operand buffers sized for the largest
// circuit, and the op and node tables in device memory.  A run is then a pure
// sequence of kernel launches on one stream per circuit: the sweeps of both halves,
// the split-pack, the tensor-core contraction (Supplementary A, Eq. 8) with its
// statistics (Section 3) fused into the epilogue, and a gather of the caller's
// amplitude subset.  With use_graph the first run is captured into a CUDA graph
// and later runs replay it.
//
// The autotuner times, on the first circuit of each shape (rows, cols, cut row,
// number of cut CZs), the fused-pass width k of the sweeps and three contraction
// variants, and keeps the fastest of each for every circuit of that shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sim.h"
#include "runtime.h"
#include "sim_internal.h"

using namespace sim;

namespace {

constexpr int kMaxLevels = 16;

// contraction variants the autotuner chooses from: {TcGemmArgs::variant, raster group}
constexpr int kGemmVariants[3][2] = {{2, 32}, {2, 8}, {1, 16}};
constexpr int kFixedFuse = 13;
constexpr int kFixedGemm = 0;

struct Item {
  Circuit circ;
  CutPlan plan;
  int cut_row = 0;
  int n = 0;
  int64_t M = 0, N = 0, K = 0, kpad = 0;
  int fuse = kFixedFuse;
  int gemm = kFixedGemm;
  double tuned_ms = 0;
  TreeProgram prog[2];
  int64_t table_off[2] = {0, 0};
};

#define BCK(x)                                                                                  \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) {                                                                    \
      cudaGetLastError();                                                                       \
      return set_error(e_ == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,                \
                       std::string(#x) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                           \
  } while (0)

#define BRC(x)             \
  do {                     \
    const int r_ = (x);    \
    if (r_) return r_;     \
  } while (0)

}  // namespace

struct sim_batch_s {
  std::vector<Item> items;
  int contraction = SIM_SPLIT_BF16;
  bool use_graph = false;
  uint64_t subset_n = 0;
  int device = 0;
  int* d_status = nullptr;
  int num_sms = 0;
  // device buffers (pool blocks owned by the batch until it is destroyed)
  std::vector<void*> owned;
  void* lvl[kMaxLevels] = {};
  size_t lvl_bytes[kMaxLevels] = {};
  void* leaf[2] = {nullptr, nullptr};
  size_t leaf_bytes[2] = {0, 0};
  void *ahi = nullptr, *alo = nullptr, *bhi = nullptr, *blo = nullptr, *scales = nullptr;
  size_t a_bytes = 0, b_bytes = 0;
  void* out = nullptr;
  size_t out_bytes = 0;
  double* acc = nullptr;                // 4 per circuit (3 used)
  unsigned long long* hist = nullptr;   // SIM_KS_BINS per circuit
  uint64_t* subset_idx = nullptr;       // subset_n per circuit
  void* subset = nullptr;               // complex64, subset_n per circuit
  NodeEntry* table = nullptr;
  bool warmed = false;
  uint64_t launches_per_run[SIM_NUM_PHASES] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;  // the capture runs here; the graph launches on the caller's stream

  cudaStream_t create_stream = nullptr;  // the stream sim_batch_create works on
  cudaError_t alloc(void** p, size_t bytes) {
    cudaError_t e = rt_alloc(p, bytes > 0 ? bytes : 256, create_stream);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
  }
  ~sim_batch_s() {
    // runs may still be in flight on the caller's streams: the blocks go back to the
    // pool once the device is idle
    cudaDeviceSynchronize();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* p : owned) rt_free(p, nullptr);
    for (Item& it : items) rt_free_plan(it.plan);
  }
};

namespace {

// Tree programs and node-table layout of every circuit with its current fuse width.
int plan_items(sim_batch_s& B, size_t level_budget, std::vector<NodeEntry>& table) {
  table.clear();
  for (Item& it : B.items) {
    CopySet cs;
    cs.kb = 0;
    cs.ke = 1ull << it.plan.c;
    for (int h = 0; h < 2; ++h) {
      it.prog[h] = rt_plan_tree(it.plan.sched[h], cs, true, level_budget);
      it.table_off[h] = (int64_t)table.size();
      table.insert(table.end(), it.prog[h].table.begin(), it.prog[h].table.end());
      if ((int)it.plan.sched[h].levels.size() > kMaxLevels)
        return set_error(SIM_EUNSUPPORTED, "too many copy-tree levels for a batch");
    }
  }
  return SIM_OK;
}

int set_fuse(Item& it, int fuse, cudaStream_t st) {
  if (it.plan.fuse_qubits == fuse && it.plan.d_ops[0]) return SIM_OK;
  CutPlan np;
  const std::string err = build_cut_plan(it.circ, it.cut_row, fuse, np);
  if (!err.empty()) return set_error(SIM_EINVAL, err);
  rt_free_plan(it.plan);
  it.plan = np;
  return rt_upload_plan(it.plan, st);
}

// the sweeps of both halves of one circuit (all copies; leaves into their rows)
int enqueue_sweeps(sim_batch_s& B, Item& it, const NodeEntry* table, cudaStream_t st) {
  for (int h = 0; h < 2; ++h)
    BRC(rt_enqueue_tree(it.plan, h, it.prog[h], B.lvl, table + it.table_off[h], nullptr, 0, B.leaf[h], st, 0, 256));
  return SIM_OK;
}

// split-pack, contraction with fused statistics into the shared output buffer,
// then the gather of the circuit's amplitude subset
int enqueue_contraction(sim_batch_s& B, Item& it, int index, int gemm, cudaStream_t st) {
  const int fp16 = B.contraction == SIM_SPLIT_FP16;
  const float* sa = nullptr;
  const float* sb = nullptr;
  if (fp16) {
    float* sc = (float*)B.scales;
    BCK(launch_absmax_c64(B.leaf[1], it.K * it.M, sc, st));
    BCK(launch_absmax_c64(B.leaf[0], it.K * it.N, sc + 2, st));
    sa = sc + 1;
    sb = sc + 3;
  }
  BCK(launch_pack_a(B.leaf[1], it.K, it.M, it.kpad, fp16, sa, B.ahi, B.alo, st));
  BCK(launch_pack_b(B.leaf[0], it.K, it.N, it.kpad, fp16, sb, B.bhi, B.blo, st));
  double* acc = B.acc + 4 * (size_t)index;
  unsigned long long* hist = B.hist + (size_t)SIM_KS_BINS * index;
  BCK(cudaMemsetAsync(acc, 0, 4 * sizeof(double), st));
  BCK(cudaMemsetAsync(hist, 0, SIM_KS_BINS * sizeof(unsigned long long), st));
  TcGemmArgs g;
  g.a_hi = B.ahi;
  g.a_lo = B.alo;
  g.b_hi = B.bhi;
  g.b_lo = B.blo;
  g.M = it.M;
  g.N2 = 2 * it.N;
  g.kpad = it.kpad;
  g.fp16 = fp16;
  g.scale_a = sa;
  g.scale_b = sb;
  g.accumulate = 0;
  g.C = B.out;
  g.group_m = kGemmVariants[gemm][1];
  g.variant = kGemmVariants[gemm][0];
  g.num_sms = B.num_sms;
  g.d_status = B.d_status;
  g.w_scale = std::ldexp(1.f, it.n);
  g.st_acc = acc;
  g.st_hist = hist;
  BCK(launch_tc_gemm(g, st));
  if (B.subset_n)
    BCK(launch_gather_flat_c64(B.out, B.subset_idx + B.subset_n * (size_t)index, (int64_t)B.subset_n,
                               (char*)B.subset + 8 * B.subset_n * (size_t)index, st));
  return SIM_OK;
}

int enqueue_all(sim_batch_s& B, cudaStream_t st) {
  for (size_t i = 0; i < B.items.size(); ++i) {
    BRC(enqueue_sweeps(B, B.items[i], B.table, st));
    BRC(enqueue_contraction(B, B.items[i], (int)i, B.items[i].gemm, st));
  }
  return SIM_OK;
}

// median of reps timings (ms) of f() enqueued on st, after one warm-up
template <class F>
int time_ms(F&& f, cudaStream_t st, int reps, double* out_ms) {
  cudaEvent_t a, b;
  BCK(cudaEventCreate(&a));
  BCK(cudaEventCreate(&b));
  std::vector<double> ts;
  int rc = f();
  for (int r = 0; r < reps && rc == SIM_OK; ++r) {
    cudaEventRecord(a, st);
    rc = f();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    ts.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  std::sort(ts.begin(), ts.end());
  *out_ms = ts[ts.size() / 2];
  return SIM_OK;
}

// Autotuner: on the first circuit of each shape, the fuse width with the fastest
// sweeps of both halves, then the fastest contraction variant on those leaves.
int autotune(sim_batch_s& B, size_t level_budget, cudaStream_t st) {
  std::map<std::tuple<int, int, int, int>, std::pair<int, int>> chosen;
  for (size_t i = 0; i < B.items.size(); ++i) {
    Item& it = B.items[i];
    const auto key = std::make_tuple(it.circ.R, it.circ.C, it.cut_row, it.plan.c);
    auto f = chosen.find(key);
    if (f != chosen.end()) {
      BRC(set_fuse(it, f->second.first, st));
      it.gemm = f->second.second;
      continue;
    }
    const int nmin = std::min(it.plan.n_u, it.plan.n_l);
    double best_sweep = 1e300, best_total = 0;
    int best_fuse = kFixedFuse;
    for (int fuse = 10; fuse <= 13; ++fuse) {
      if (fuse > nmin && fuse != 10) continue;
      BRC(set_fuse(it, fuse, st));
      CopySet cs;
      cs.kb = 0;
      cs.ke = 1ull << it.plan.c;
      std::vector<NodeEntry> tab;
      for (int h = 0; h < 2; ++h) {
        it.prog[h] = rt_plan_tree(it.plan.sched[h], cs, true, level_budget);
        it.table_off[h] = (int64_t)tab.size();
        tab.insert(tab.end(), it.prog[h].table.begin(), it.prog[h].table.end());
      }
      void* dt = nullptr;
      BCK(rt_alloc(&dt, sizeof(NodeEntry) * (tab.size() + 1), st));
      cudaError_t e = cudaMemcpyAsync(dt, tab.data(), sizeof(NodeEntry) * tab.size(), cudaMemcpyHostToDevice, st);
      double ms = 0;
      int rc = e == cudaSuccess ? time_ms([&] { return enqueue_sweeps(B, it, (const NodeEntry*)dt, st); }, st, 3, &ms)
                                : set_error(SIM_ECUDA, cudaGetErrorString(e));
      cudaStreamSynchronize(st);
      rt_free(dt, st);
      BRC(rc);
      if (ms < best_sweep) {
        best_sweep = ms;
        best_fuse = fuse;
      }
    }
    BRC(set_fuse(it, best_fuse, st));
    // leaves of the chosen width for the contraction trials
    {
      CopySet cs;
      cs.kb = 0;
      cs.ke = 1ull << it.plan.c;
      std::vector<NodeEntry> tab;
      for (int h = 0; h < 2; ++h) {
        it.prog[h] = rt_plan_tree(it.plan.sched[h], cs, true, level_budget);
        it.table_off[h] = (int64_t)tab.size();
        tab.insert(tab.end(), it.prog[h].table.begin(), it.prog[h].table.end());
      }
      void* dt = nullptr;
      BCK(rt_alloc(&dt, sizeof(NodeEntry) * (tab.size() + 1), st));
      cudaError_t e = cudaMemcpyAsync(dt, tab.data(), sizeof(NodeEntry) * tab.size(), cudaMemcpyHostToDevice, st);
      int rc = e == cudaSuccess ? enqueue_sweeps(B, it, (const NodeEntry*)dt, st) : set_error(SIM_ECUDA, "table");
      cudaStreamSynchronize(st);
      rt_free(dt, st);
      BRC(rc);
    }
    double best_gemm = 1e300;
    int best_variant = kFixedGemm;
    for (int v = 0; v < 3; ++v) {
      double ms = 0;
      BRC(time_ms([&] { return enqueue_contraction(B, it, (int)i, v, st); }, st, 3, &ms));
      if (ms < best_gemm) {
        best_gemm = ms;
        best_variant = v;
      }
    }
    it.gemm = best_variant;
    best_total = best_sweep + best_gemm;
    it.tuned_ms = best_total;
    chosen[key] = {best_fuse, best_variant};
  }
  return SIM_OK;
}

}  // namespace

int sim_batch_create(const sim_circuit_desc* descs, int n_circuits, const uint64_t* subset_idx, uint64_t subset_n,
                     const sim_batch_opts* opts, void* stream, sim_batch* out) {
  try {
    if (!descs || n_circuits <= 0 || !out) return set_error(SIM_EINVAL, "descs, n_circuits > 0 and out are required");
    if (subset_n && !subset_idx) return set_error(SIM_EINVAL, "subset_idx is required when subset_n > 0");
    *out = nullptr;
    const int contraction = (opts && opts->contraction) ? opts->contraction : SIM_SPLIT_BF16;
    if (contraction != SIM_SPLIT_BF16 && contraction != SIM_SPLIT_FP16)
      return set_error(SIM_EINVAL, "a batch contracts with SIM_SPLIT_BF16 or SIM_SPLIT_FP16");
    cudaStream_t st = (cudaStream_t)stream;
    auto B = std::unique_ptr<sim_batch_s>(new sim_batch_s());
    B->create_stream = st;
    B->contraction = contraction;
    B->use_graph = opts && opts->use_graph;
    B->subset_n = subset_n;
    // host planning of every circuit (validated before any device work)
    B->items.resize((size_t)n_circuits);
    for (int i = 0; i < n_circuits; ++i) {
      Item& it = B->items[(size_t)i];
      const sim_circuit_desc& d = descs[i];
      std::string err = d.gate_list ? parse_circuit(d.gate_list, it.circ)
                                    : generate_circuit(d.rows, d.cols, d.depth, d.seed, d.cut_row, it.circ,
                                                       d.rule_t_in_pool);
      if (!err.empty()) return set_error(SIM_EINVAL, "circuit " + std::to_string(i) + ": " + err);
      it.cut_row = d.cut_row > 0 ? d.cut_row : it.circ.R / 2;
      err = build_cut_plan(it.circ, it.cut_row, kFixedFuse, it.plan);
      if (!err.empty()) return set_error(SIM_EINVAL, "circuit " + std::to_string(i) + ": " + err);
      it.n = it.circ.n;
      it.M = (int64_t)1 << it.plan.n_l;
      it.N = (int64_t)1 << it.plan.n_u;
      it.K = (int64_t)1 << it.plan.c;
      it.kpad = ((2 * it.K + 63) / 64) * 64;
      {
        const int rc = check_split_bf16(contraction, it.K, false);
        if (rc) return set_error(rc, "circuit " + std::to_string(i) + ": " + sim_last_error());
      }
      if (it.n > 34) return set_error(SIM_EUNSUPPORTED, "a batch evaluates full vectors of at most 34 qubits");
      for (uint64_t j = 0; j < subset_n; ++j)
        if (subset_idx[(size_t)i * subset_n + j] >> it.n)
          return set_error(SIM_EINVAL, "subset index out of range for circuit " + std::to_string(i));
    }
    BCK(cudaGetDevice(&B->device));
    BRC(rt_device(&B->d_status, &B->num_sms));
    for (Item& it : B->items) BRC(rt_upload_plan(it.plan, st));
    // buffers for the largest circuit (all circuits run one after another)
    size_t fr = 0, tot = 0;
    BCK(cudaMemGetInfo(&fr, &tot));
    for (const Item& it : B->items) {
      B->out_bytes = std::max(B->out_bytes, (size_t)8 << it.n);
      B->leaf_bytes[0] = std::max(B->leaf_bytes[0], (size_t)it.K * ((size_t)8 << it.plan.n_u));
      B->leaf_bytes[1] = std::max(B->leaf_bytes[1], (size_t)it.K * ((size_t)8 << it.plan.n_l));
      B->a_bytes = std::max(B->a_bytes, (size_t)it.M * (size_t)it.kpad * 2);
      B->b_bytes = std::max(B->b_bytes, (size_t)(2 * it.N) * (size_t)it.kpad * 2);
    }
    const size_t fixed = B->out_bytes + B->leaf_bytes[0] + B->leaf_bytes[1] + 2 * B->a_bytes + 2 * B->b_bytes;
    if (fixed > fr) return set_error(SIM_ENOMEM, "the batch's output, leaf and operand buffers exceed free memory");
    const size_t level_budget = (size_t)((double)(fr - fixed) * 0.5);
    std::vector<NodeEntry> table;
    BRC(plan_items(*B, level_budget, table));
    auto level_sizes = [&]() {
      for (const Item& it : B->items)
        for (int h = 0; h < 2; ++h) {
          const HalfSchedule& S = it.plan.sched[h];
          for (size_t j = 0; j + 1 < S.levels.size(); ++j)
            B->lvl_bytes[j] = std::max(B->lvl_bytes[j], (size_t)it.prog[h].level_cap[j] * ((size_t)8 << S.n));
        }
    };
    level_sizes();
    for (int j = 0; j < kMaxLevels; ++j)
      if (B->lvl_bytes[j]) BCK(B->alloc(&B->lvl[j], B->lvl_bytes[j]));
    for (int h = 0; h < 2; ++h) BCK(B->alloc(&B->leaf[h], B->leaf_bytes[h]));
    BCK(B->alloc(&B->ahi, B->a_bytes));
    BCK(B->alloc(&B->alo, B->a_bytes));
    BCK(B->alloc(&B->bhi, B->b_bytes));
    BCK(B->alloc(&B->blo, B->b_bytes));
    BCK(B->alloc(&B->scales, 4 * sizeof(float)));
    BCK(B->alloc(&B->out, B->out_bytes));
    BCK(B->alloc((void**)&B->acc, 4 * sizeof(double) * (size_t)n_circuits));
    BCK(B->alloc((void**)&B->hist, SIM_KS_BINS * sizeof(unsigned long long) * (size_t)n_circuits));
    if (subset_n) {
      BCK(B->alloc((void**)&B->subset_idx, sizeof(uint64_t) * subset_n * (size_t)n_circuits));
      BCK(B->alloc(&B->subset, 8 * subset_n * (size_t)n_circuits));
      BCK(cudaMemcpyAsync(B->subset_idx, subset_idx, sizeof(uint64_t) * subset_n * (size_t)n_circuits,
                          cudaMemcpyHostToDevice, st));
    }
    if (opts && opts->autotune) {
      const bool prof_was = rt_profile_swap(false);
      const int rc = autotune(*B, level_budget, st);
      rt_profile_swap(prof_was);
      BRC(rc);
      // re-plan with the chosen widths; level buffers grow if a choice needs more
      BRC(plan_items(*B, level_budget, table));
      size_t old[kMaxLevels];
      memcpy(old, B->lvl_bytes, sizeof old);
      level_sizes();
      for (int j = 0; j < kMaxLevels; ++j)
        if (B->lvl_bytes[j] > old[j]) BCK(B->alloc(&B->lvl[j], B->lvl_bytes[j]));
    }
    BCK(B->alloc((void**)&B->table, sizeof(NodeEntry) * (table.size() + 1)));
    BCK(cudaMemcpyAsync(B->table, table.data(), sizeof(NodeEntry) * table.size(), cudaMemcpyHostToDevice, st));
    BCK(cudaStreamSynchronize(st));
    *out = B.release();
    return SIM_OK;
  } catch (const std::bad_alloc&) {
    return set_error(SIM_ENOMEM, "host allocation failed");
  } catch (const std::exception& ex) {
    return set_error(SIM_EINVAL, std::string("internal error: ") + ex.what());
  }
}

int sim_batch_run(sim_batch b, void* stream) {
  if (!b) return set_error(SIM_EINVAL, "batch must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  if (dev != b->device) return set_error(SIM_EINVAL, "the batch belongs to another device");
  if (!b->warmed || !b->use_graph) {
    // uncaptured run: also initialises every kernel's attributes before a capture
    uint64_t before[SIM_NUM_PHASES], after[SIM_NUM_PHASES];
    rt_launch_totals(before);
    BRC(enqueue_all(*b, st));
    rt_launch_totals(after);
    for (int i = 0; i < SIM_NUM_PHASES; ++i) b->launches_per_run[i] = after[i] - before[i];
    b->warmed = true;
    return SIM_OK;
  }
  if (!b->exec) {
    // captured on a stream of the batch's own (the caller's may be the legacy
    // default stream, which cannot be captured)
    if (!b->cap_stream) BCK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    const bool prof_was = rt_profile_swap(false);
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? enqueue_all(*b, b->cap_stream) : set_error(SIM_ECUDA, cudaGetErrorString(e));
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    rt_profile_swap(prof_was);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    BCK(e2);
    b->graph = g;
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  BCK(cudaGraphLaunch(b->exec, st));
  for (int i = 0; i < SIM_NUM_PHASES; ++i) note_launches(i, (int)b->launches_per_run[i]);
  return SIM_OK;
}

int sim_batch_results(sim_batch b, double* stats_out, void* subset_out) {
  if (!b) return set_error(SIM_EINVAL, "batch must not be NULL");
  try {
    const size_t n = b->items.size();
    if (stats_out) {
      std::vector<double> acc(4 * n);
      std::vector<unsigned long long> hist((size_t)SIM_KS_BINS * n);
      BCK(cudaMemcpy(acc.data(), b->acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost));
      BCK(cudaMemcpy(hist.data(), b->hist, sizeof(unsigned long long) * hist.size(), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < n; ++i) {
        std::vector<unsigned long long> hh(hist.begin() + (ptrdiff_t)(i * SIM_KS_BINS),
                                           hist.begin() + (ptrdiff_t)((i + 1) * SIM_KS_BINS));
        rt_finish_stats(&acc[4 * i], hh, (uint64_t)1 << b->items[i].n, b->items[i].n, stats_out + 4 * i, nullptr);
      }
    }
    if (subset_out && b->subset_n)
      BCK(cudaMemcpy(subset_out, b->subset, 8 * b->subset_n * n, cudaMemcpyDeviceToHost));
    return SIM_OK;
  } catch (const std::exception& ex) {
    return set_error(SIM_EINVAL, std::string("internal error: ") + ex.what());
  }
}

int sim_batch_info(sim_batch b, int i, int32_t info_out[5], double* tuned_ms) {
  if (!b || i < 0 || i >= (int)b->items.size() || !info_out) return set_error(SIM_EINVAL, "bad arguments");
  const Item& it = b->items[(size_t)i];
  info_out[0] = it.n;
  info_out[1] = it.plan.c;
  info_out[2] = it.plan.fuse_qubits;
  info_out[3] = kGemmVariants[it.gemm][0] == 1 ? 1 : 0;
  info_out[4] = kGemmVariants[it.gemm][1];
  if (tuned_ms) *tuned_ms = it.tuned_ms;
  return SIM_OK;
}

void sim_destroy_batch(sim_batch b) { delete b; }
