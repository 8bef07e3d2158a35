// C-ABI of libsim (include/sim.h): error handling, the device memory pool, the
// copy-tree evolution engine (complex64 fused path and complex128 plain path),
// the contraction dispatch, statistics and selection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <unistd.h>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/sim.h"
#include "runtime.h"
#include "sim_internal.h"

using namespace sim;

struct sim_circuit_s {
  Circuit c;
};

struct sim_cut_s {
  CutPlan p;
};

struct sim_multi_s {
  MultiPlan mp;
};

struct sim_halves_s {
  CutPlan* plan = nullptr;
  int precision = SIM_C64;
  CopySet cs;
  int64_t nsel[2] = {0, 0};
  bool full[2] = {true, true};
  void* d_sel[2] = {nullptr, nullptr};
  void* leafsel[2] = {nullptr, nullptr};  // [K][nsel] complex64 or complex128
  uint32_t* out_code[2] = {nullptr, nullptr};  // output-phase codes per selected index (or NULL)
  cudaStream_t stream = nullptr;
  int device = 0;
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      if (e_ == cudaErrorMemoryAllocation) {                                           \
        cudaGetLastError();                                                            \
        return fail(SIM_ENOMEM, std::string(#x) + ": " + cudaGetErrorString(e_));       \
      }                                                                                \
      return fail(SIM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_));         \
    }                                                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// Device memory pool: cudaMalloc'd blocks cached by (device, rounded size).  Sizes
// are rounded up to 2 MiB above 1 MiB and to a power of two below.
// Reuse is stream-ordered.  A block freed with a stream carries an event recorded
// on that stream at the free, after all the work that used it.  A later request on
// the same stream reuses it at once (stream order already puts the new work after
// the old); a request on another stream takes a block whose event has completed,
// or else makes its stream wait for the event (cudaStreamWaitEvent, no host wait).
// So buffers can go back to the pool while kernels still use them, and callers on
// several streams never share a block across in-flight work.
// ---------------------------------------------------------------------------
struct Pool {
  struct Blk {
    void* p;
    cudaEvent_t ev;   // recorded on st at the free (null: the block was idle)
    cudaStream_t st;
  };
  std::mutex mu;
  std::map<std::pair<int, size_t>, std::vector<Blk>> free_blocks;
  std::unordered_map<void*, std::pair<int, size_t>> owner;
  std::map<int, std::vector<cudaEvent_t>> spare_ev;  // per device

  static size_t round(size_t n) {
    if (n <= 256) return 256;
    if (n <= (1u << 20)) {
      size_t r = 256;
      while (r < n) r <<= 1;
      return r;
    }
    const size_t g = (size_t)2 << 20;
    return (n + g - 1) / g * g;
  }

  // (mu held) an event of the current device
  cudaEvent_t take_event(int dev) {
    auto& v = spare_ev[dev];
    if (!v.empty()) {
      cudaEvent_t e = v.back();
      v.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }

  // n bytes for work on stream st
  cudaError_t alloc(void** p, size_t n, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t r = round(n);
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = free_blocks.find({dev, r});
      if (it != free_blocks.end() && !it->second.empty()) {
        std::vector<Blk>& v = it->second;
        // an idle block, else the latest freed on this stream, else the latest;
        // a block still in use orders st after its free (stream identity alone is
        // not trusted: a destroyed stream's handle can come back for a new one)
        int pick = -1, same = -1;
        for (int i = (int)v.size() - 1; i >= 0 && pick < 0; --i) {
          if (!v[i].ev || cudaEventQuery(v[i].ev) == cudaSuccess) pick = i;
          else if (same < 0 && v[i].st == st) same = i;
        }
        cudaGetLastError();  // a not-ready query
        cudaError_t e = cudaSuccess;
        if (pick < 0) {
          pick = same >= 0 ? same : (int)v.size() - 1;
          e = cudaStreamWaitEvent(st, v[pick].ev, 0);
        }
        if (e == cudaSuccess) {
          *p = v[pick].p;
          if (v[pick].ev) spare_ev[dev].push_back(v[pick].ev);
          v.erase(v.begin() + pick);
          owner[*p] = {dev, r};
          return cudaSuccess;
        }
        cudaGetLastError();
      }
    }
    cudaError_t e = cudaMalloc(p, r);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      release(dev);
      e = cudaMalloc(p, r);
    }
    if (e != cudaSuccess) {
      *p = nullptr;
      return e;
    }
    std::lock_guard<std::mutex> lk(mu);
    owner[*p] = {dev, r};
    return cudaSuccess;
  }

  // back to the pool after the work enqueued so far on st (ordered), or at once
  // (the caller has waited for every use of the block)
  void free(void* p, cudaStream_t st, bool ordered) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu);
    auto it = owner.find(p);
    if (it == owner.end()) return;
    Blk b{p, nullptr, st};
    if (ordered) {
      // the event belongs to the block's device, whichever device is current
      const int dev = it->second.first;
      int cur = dev;
      cudaGetDevice(&cur);
      if (cur != dev) cudaSetDevice(dev);
      b.ev = take_event(dev);
      if (!b.ev || cudaEventRecord(b.ev, st) != cudaSuccess) {
        cudaGetLastError();
        if (b.ev) spare_ev[dev].push_back(b.ev);
        b.ev = nullptr;
        cudaStreamSynchronize(st);  // no event: wait instead
        cudaGetLastError();
      }
      if (cur != dev) cudaSetDevice(cur);
    }
    free_blocks[it->second].push_back(b);
    owner.erase(it);
  }

  void release(int dev) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& kv : free_blocks) {
      if (dev >= 0 && kv.first.first != dev) continue;
      for (const Blk& b : kv.second) {
        if (b.ev) {
          cudaEventSynchronize(b.ev);
          spare_ev[kv.first.first].push_back(b.ev);
        }
        cudaFree(b.p);
      }
      kv.second.clear();
    }
  }
};

Pool& pool() {
  static Pool* p = new Pool();  // never destroyed: the CUDA context may be gone at exit
  return *p;
}

// A pool block for work on one stream, returned to the pool (stream-ordered) when
// the DevBuf goes out of scope, with its kernels possibly still running.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { pool().free(p, st, true); }
  cudaError_t alloc(size_t n, cudaStream_t s) {
    pool().free(p, st, true);
    p = nullptr;
    st = s;
    return pool().alloc(&p, n ? n : 1, s);
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

// ---------------------------------------------------------------------------
// Phase profiler: CUDA event pairs per phase instance on the launching stream,
// kernel launch and host<->device byte counters.
// ---------------------------------------------------------------------------
struct Profiler {
  std::mutex mu;
  bool on = false;
  struct Rec {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> spare;
  double ms[SIM_NUM_PHASES] = {};
  uint64_t inst[SIM_NUM_PHASES] = {};
  uint64_t launches[SIM_NUM_PHASES] = {};
  uint64_t h2d = 0, d2h = 0;
  uint64_t all_launches[SIM_NUM_PHASES] = {};  // counted whether or not the profiler is on

  cudaEvent_t get() {
    if (!spare.empty()) {
      cudaEvent_t e = spare.back();
      spare.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
};

Profiler& prof() {
  static Profiler* p = new Profiler();
  return *p;
}

// Records a begin event at construction and an end event at destruction when
// the profiler is on.
struct PhaseScope {
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  PhaseScope(int ph, cudaStream_t s) : phase(ph), st(s) {
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    if (!P.on) return;
    a = P.get();
    if (a) cudaEventRecord(a, st);
  }
  ~PhaseScope() {
    if (!a) return;
    Profiler& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    cudaEvent_t b = P.get();
    if (!b) return;
    cudaEventRecord(b, st);
    P.recs.push_back({phase, a, b});
  }
};

// per-device status word of the contraction and other per-device constants
struct DeviceInfo {
  int* d_status = nullptr;
  int num_sms = 0;
  size_t total_mem = 0;
};

std::mutex g_dev_mu;
std::map<int, DeviceInfo> g_dev;

int device_info(DeviceInfo** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo& d = g_dev[dev];
  if (!d.d_status) {
    CK(cudaMalloc(&d.d_status, sizeof(int)));
    CK(cudaMemset(d.d_status, 0, sizeof(int)));
    CK(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
    size_t fr = 0;
    CK(cudaMemGetInfo(&fr, &d.total_mem));
  }
  *out = &d;
  return SIM_OK;
}

// Op tables of a plan live in pool memory, uploaded on the caller's stream the
// first time the plan is evolved on a device.
void free_plan_ops(CutPlan& P) {
  // after the work enqueued so far on the last stream that used them
  const cudaStream_t st = (cudaStream_t)P.ops_stream;
  for (int h = 0; h < 2; ++h) {
    pool().free(P.d_ops[h], st, true);
    pool().free(P.d_plain_ops[h], st, true);
    P.d_ops[h] = P.d_plain_ops[h] = nullptr;
  }
  P.device = -1;
}

int upload_plan_ops(CutPlan& P, cudaStream_t st) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (P.device == dev && P.d_ops[0]) {
    // another stream now uses the tables: order it after their upload
    if ((cudaStream_t)P.ops_stream != st) {
      cudaEvent_t ev = nullptr;
      CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      cudaError_t e = cudaEventRecord(ev, (cudaStream_t)P.ops_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
      cudaEventDestroy(ev);
      CK(e);
      P.ops_stream = st;
    }
    return SIM_OK;
  }
  free_plan_ops(P);
  P.ops_stream = st;
  for (int h = 0; h < 2; ++h) {
    const auto& ops = P.sched[h].ops;
    void* p = nullptr;
    CK(pool().alloc(&p, sizeof(OpRec) * (ops.size() + 1), st));
    P.d_ops[h] = (OpRec*)p;
    if (!ops.empty())
      CK(cudaMemcpyAsync(P.d_ops[h], ops.data(), sizeof(OpRec) * ops.size(), cudaMemcpyHostToDevice, st));
    note_bytes(sizeof(OpRec) * ops.size(), 0);
    std::vector<OpRec>& flat = P.plain_flat[h];
    flat.clear();
    P.plain_op_offsets[h].clear();
    for (const PlainLayer& L : P.plain[h]) {
      P.plain_op_offsets[h].push_back((int)flat.size());
      flat.insert(flat.end(), L.gates.begin(), L.gates.end());
      flat.insert(flat.end(), L.diags.begin(), L.diags.end());
    }
    CK(pool().alloc(&p, sizeof(OpRec) * (flat.size() + 1), st));
    P.d_plain_ops[h] = (OpRec*)p;
    if (!flat.empty())
      CK(cudaMemcpyAsync(P.d_plain_ops[h], flat.data(), sizeof(OpRec) * flat.size(), cudaMemcpyHostToDevice, st));
    note_bytes(sizeof(OpRec) * flat.size(), 0);
  }
  P.device = dev;
  return SIM_OK;
}

// ---------------------------------------------------------------------------
// complex64 copy-tree evolution of one half
// ---------------------------------------------------------------------------
struct TreeBuilder {
  const HalfSchedule& S;
  const CopySet& cs;
  bool direct;            // leaves written straight into leafsel rows (no selection)
  int sparse_d;           // > 0: the selected leaf entries come from the level sparse_d above the leaves
  std::vector<std::vector<uint64_t>> needed;  // sorted node ids per level
  TreeProgram& prog;

  // node ids of level j on the paths to the copies: the low bits_total bits of each
  std::vector<uint64_t> needed_ids(int j) const {
    const int bits = S.levels[j].bits_total;
    std::vector<uint64_t> ids;
    const uint64_t count = bits >= 63 ? ~0ull : (1ull << bits);
    const uint64_t K = cs.size();
    if (cs.list.empty() && K >= count) {
      ids.resize(count);
      for (uint64_t i = 0; i < count; ++i) ids[i] = i;
    } else {
      ids.reserve(K);
      for (uint64_t i = 0; i < K; ++i) ids.push_back(cs.at(i) & (count - 1));
      std::sort(ids.begin(), ids.end());
      ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    }
    return ids;
  }

  void build() {
    const int J = (int)S.levels.size();
    for (int j = 0; j < J; ++j) needed.push_back(needed_ids(j));
    std::vector<uint64_t> root_ids = needed[0];
    process(0, root_ids, {});
  }

  // ids: node ids of level j to run; parent_slot: slot of each id's parent in the
  // parent level's current chunk buffer (empty at the root)
  void process(int j, const std::vector<uint64_t>& ids, const std::unordered_map<uint64_t, int64_t>& parent_slot) {
    const int J = (int)S.levels.size();
    const Level& L = S.levels[j];
    const bool leaf = (j == J - 1);
    const int64_t cap = prog.level_cap[j];
    for (size_t c0 = 0; c0 < ids.size(); c0 += (size_t)cap) {
      const size_t c1 = std::min(ids.size(), c0 + (size_t)cap);
      const int64_t off = (int64_t)prog.table.size();
      std::unordered_map<uint64_t, int64_t> my_slot;
      for (size_t i = c0; i < c1; ++i) {
        NodeEntry e;
        e.node_id = ids[i];
        e.parent_slot = 0;
        if (j > 0) {
          const uint64_t pmask = L.bits_before >= 63 ? ~0ull : ((1ull << L.bits_before) - 1);
          e.parent_slot = parent_slot.at(ids[i] & pmask);
        }
        e.dst_row = (leaf && direct) ? cs.row_of(ids[i]) : (int64_t)(i - c0);
        prog.table.push_back(e);
        my_slot[ids[i]] = (int64_t)(i - c0);
      }
      const int64_t ns = (int64_t)(c1 - c0);
      const int dst = (leaf && direct) ? -1 : j;
      for (size_t p = 0; p < L.passes.size(); ++p) {
        LaunchRec r;
        r.level = j;
        r.pass = (int)p;
        r.table_off = off;
        r.nslots = ns;
        r.src_buf = (p == 0 && j > 0) ? j - 1 : dst;
        r.dst_buf = dst;
        prog.launches.push_back(r);
      }
      if (sparse_d > 0 && j == J - 1 - sparse_d) {
        // the leaves under this chunk's nodes, read from them (one launch): ancestor
        // slot and leaf row of each leaf; the levels below are never formed
        const uint64_t amask = L.bits_total >= 63 ? ~0ull : ((1ull << L.bits_total) - 1);
        const int64_t soff = (int64_t)prog.table.size();
        for (uint64_t id : needed[J - 1]) {
          const auto it = my_slot.find(id & amask);
          if (it == my_slot.end()) continue;
          NodeEntry e;
          e.node_id = id;
          e.parent_slot = it->second;
          e.dst_row = cs.row_of(id);
          prog.table.push_back(e);
        }
        LaunchRec r;
        r.level = j;
        r.pass = -2;
        r.table_off = soff;
        r.nslots = (int64_t)prog.table.size() - soff;
        r.src_buf = j;
        r.dst_buf = -1;
        if (r.nslots > 0) prog.launches.push_back(r);
        continue;
      }
      if (leaf) {
        if (!direct) {
          // gather table: rows of leafsel
          const int64_t goff = (int64_t)prog.table.size();
          for (size_t i = c0; i < c1; ++i) {
            NodeEntry e;
            e.node_id = ids[i];
            e.parent_slot = 0;
            e.dst_row = cs.row_of(ids[i]);
            prog.table.push_back(e);
          }
          LaunchRec r;
          r.level = j;
          r.pass = -1;
          r.table_off = goff;
          r.nslots = ns;
          r.src_buf = j;
          r.dst_buf = -1;
          prog.launches.push_back(r);
        }
      } else {
        const Level& N = S.levels[j + 1];
        const int nb = N.bits_total - N.bits_before;
        std::vector<uint64_t> kids;
        const auto& nxt = needed[j + 1];
        for (size_t i = c0; i < c1; ++i)
          for (uint64_t l = 0; l < (1ull << nb); ++l) {
            const uint64_t cid = ids[i] | (l << N.bits_before);
            if (std::binary_search(nxt.begin(), nxt.end(), cid)) kids.push_back(cid);
          }
        std::sort(kids.begin(), kids.end());
        process(j + 1, kids, my_slot);
      }
    }
  }
};

TreeProgram plan_tree(const HalfSchedule& S, const CopySet& cs, bool full, size_t budget, int sparse_d = 0) {
  const size_t state_bytes = sizeof(float) * 2 * ((size_t)1 << S.n);
  const int J = (int)S.levels.size();
  TreeProgram prog;
  for (int j = 0; j < J; ++j) {
    const int64_t need_nodes = (int64_t)std::min<uint64_t>(
        cs.size(), S.levels[j].bits_total >= 63 ? ~0ull : (1ull << S.levels[j].bits_total));
    int64_t cap = (int64_t)(budget / std::max(1, J) / state_bytes);
    if (cap < 1) cap = 1;
    prog.level_cap.push_back(std::min<int64_t>(cap, std::max<int64_t>(need_nodes, 1)));
  }
  TreeBuilder tb{S, cs, full, full ? 0 : sparse_d, {}, prog};
  tb.build();
  return prog;
}

// The ops of a half's last d copy-tree levels (a contiguous run of S.ops: levels
// and their passes are laid out in order) and the qubits on which they act
// non-diagonally: the inputs of the sparse leaf evaluation.
struct LeafOps {
  uint32_t qmask = 0;
  int nq = 0, op_begin = 0, op_count = 0;
};
LeafOps leaf_ops(const HalfSchedule& S, int d) {
  LeafOps r;
  const int J = (int)S.levels.size();
  if (d < 1 || d > J || S.levels[J - d].passes.empty() || S.levels.back().passes.empty()) return r;
  r.op_begin = S.levels[J - d].passes.front().op_begin;
  r.op_count = S.levels.back().passes.back().op_begin + S.levels.back().passes.back().op_count - r.op_begin;
  for (int o = r.op_begin; o < r.op_begin + r.op_count; ++o)
    if (S.ops[o].type == OP_GATE) r.qmask |= 1u << S.ops[o].q;
  r.nq = __builtin_popcount(r.qmask);
  return r;
}

// Levels the sparse leaf evaluation covers (0: none): the most trailing levels,
// below at least the root, whose ops act non-diagonally on at most kMaxSparseQ
// qubits Q, and (mode 0) with nsel * 2^|Q| <= 2^n / 8; mode 1: the |Q| limit only;
// mode -1: none.
int sparse_depth(const HalfSchedule& S, int64_t nsel, int mode) {
  const int J = (int)S.levels.size();
  if (mode < 0 || S.n > 32) return 0;
  for (int d = J - 1; d >= 1; --d) {
    const LeafOps lo = leaf_ops(S, d);
    if (lo.nq > kMaxSparseQ) continue;
    if (mode == 1 || (((uint64_t)nsel << lo.nq) <= (((uint64_t)1 << S.n) >> 3))) return d;
  }
  return 0;
}

int enqueue_tree(const CutPlan& P, int h, const TreeProgram& prog, void* const* lvl, const NodeEntry* table,
                 const uint64_t* d_sel, int64_t nsel, void* leafsel, cudaStream_t st, int kernel_choice,
                 int threads) {
  const HalfSchedule& S = P.sched[h];
  const int n = S.n;
  for (const LaunchRec& r : prog.launches) {
    void* dstp = r.dst_buf < 0 ? leafsel : lvl[r.dst_buf];
    PhaseScope ps(r.pass < 0 ? SIM_PHASE_GATHER : SIM_PHASE_SWEEP, st);
    if (r.pass == -2) {
      const LeafOps lo = leaf_ops(S, (int)S.levels.size() - 1 - r.level);
      SparseLeafLaunch sl;
      memset(&sl, 0, sizeof sl);
      sl.n = n;
      sl.nq = lo.nq;
      int b = 0;
      for (int q = 0; q < n && b < kMaxSparseQ; ++q)
        if ((lo.qmask >> q) & 1u) sl.qpos[b++] = (uint8_t)q;
      sl.ops = P.d_ops[h] + lo.op_begin;
      sl.op_count = lo.op_count;
      sl.nodes = table + r.table_off;
      sl.nslots = r.nslots;
      sl.parent_base = lvl[r.src_buf];
      sl.sel = d_sel;
      sl.nsel = nsel;
      sl.leafsel = leafsel;
      CK(launch_sparse_leaf(sl, st));
      continue;
    }
    if (r.pass < 0) {
      CK(launch_gather(lvl[r.src_buf], n, table + r.table_off, r.nslots, d_sel, nsel, leafsel, 0, st));
      continue;
    }
    const PassDesc& pd = S.levels[r.level].passes[r.pass];
    SweepLaunch sl;
    sl.n = n;
    sl.k = pd.k;
    sl.low = pd.low;
    sl.local_mask = pd.local_mask;
    sl.ops = P.d_ops[h] + pd.op_begin;
    sl.op_count = pd.op_count;
    sl.src = pd.src;
    sl.nodes = table + r.table_off;
    sl.nslots = r.nslots;
    sl.src_base = pd.src == SRC_PARENT ? lvl[r.src_buf] : dstp;
    sl.dst_base = dstp;
    sl.threads = threads;
    memcpy(sl.order, pd.order, sizeof sl.order);
    sl.warp_gates = pd.warp_gates;
    sl.general_gates = pd.general_gates;
    sl.scale = pd.scale;
    sl.phase_e = pd.phase_e;
    sl.phase_op = pd.phase_op;
    memcpy(sl.sorder, pd.sorder, sizeof sl.sorder);
    memcpy(sl.swz, pd.swz, sizeof sl.swz);
    sl.transpose = pd.transpose;
    sl.vec4 = pd.vec4;
    if (kernel_choice != 1 && sweep2_supported(sl))
      CK(launch_sweep2_c64(sl, st));
    else
      CK(launch_sweep_c64(sl, st));
  }
  return SIM_OK;
}

// Pinned host buffer that the GPU reads and writes through its unified address;
// the owner synchronizes the stream that uses it before it is released.
struct HostBuf {
  void* p = nullptr;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t alloc(size_t n) { return cudaHostAlloc(&p, n ? n : 1, cudaHostAllocMapped); }
};

int evolve_c64_half(CutPlan& P, int h, const CopySet& cs, const uint64_t* d_sel, int64_t nsel, bool full,
                    void* leafsel, cudaStream_t st, const sim_opts* opts) {
  const HalfSchedule& S = P.sched[h];
  const size_t state_bytes = sizeof(float) * 2 * ((size_t)1 << S.n);
  const int J = (int)S.levels.size();
  const bool host = opts && opts->host_levels;
  // chunk capacity per level from the free device memory, or (host levels) a
  // quarter of the available host memory
  size_t budget = 0;
  if (host) {
    const long pages = sysconf(_SC_AVPHYS_PAGES), psz = sysconf(_SC_PAGESIZE);
    if (pages <= 0 || psz <= 0) return fail(SIM_ECUDA, "cannot read the available host memory");
    budget = (size_t)pages * (size_t)psz / 4;
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    budget = (size_t)(fr * 0.6);
  }
  // Selected leaf entries straight from the parents (no leaf states) where the
  // selection is sparse: 2^nq parent reads per entry against a pass over the whole
  // leaf (sim_opts.sparse_leaves: 1 wherever it applies, -1 never)
  const int sparse_d = (full || (uint64_t)nsel >= ((uint64_t)1 << S.n))
                           ? 0
                           : sparse_depth(S, nsel, opts ? opts->sparse_leaves : 0);
  const TreeProgram prog = plan_tree(S, cs, full, budget, sparse_d);
  std::vector<DevBuf> lvl(J);
  std::vector<HostBuf> hlvl(J);
  std::vector<void*> lp(J, nullptr);
  for (int j = 0; j < J; ++j) {
    const bool leaf = (j == J - 1);
    if ((leaf && full) || j > J - 1 - sparse_d) continue;
    const size_t bytes = state_bytes * (size_t)prog.level_cap[j];
    if (host) {
      if (hlvl[j].alloc(bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(SIM_ENOMEM, "cannot allocate pinned host memory for the copy-tree levels");
      }
      CK(cudaHostGetDevicePointer(&lp[j], hlvl[j].p, 0));
    } else {
      CK(lvl[j].alloc(bytes, st));
      lp[j] = lvl[j].p;
    }
  }
  DevBuf table;
  CK(table.alloc(sizeof(NodeEntry) * (prog.table.size() + 1), st));
  CK(cudaMemcpyAsync(table.p, prog.table.data(), sizeof(NodeEntry) * prog.table.size(), cudaMemcpyHostToDevice, st));
  note_bytes(sizeof(NodeEntry) * prog.table.size(), 0);
  // the device buffers go back to the pool (stream-ordered, behind these launches)
  // when this function returns; host level buffers only after the stream has
  // finished with them
  const int rc = enqueue_tree(P, h, prog, lp.data(), table.as<NodeEntry>(), d_sel, nsel, leafsel, st,
                              opts ? opts->sweep_kernel : 0,
                              (opts && opts->sweep_threads > 0) ? opts->sweep_threads : 256);
  if (host) CK(cudaStreamSynchronize(st));
  return rc;
}

// ---------------------------------------------------------------------------
// complex128 plain path of one half: every copy evolved on its own, one pass per
// non-diagonal gate and one combined diagonal pass per layer (Sections 2.3.1, 2.4)
// ---------------------------------------------------------------------------
int evolve_plain_half(CutPlan& P, int h, const CopySet& cs, const uint64_t* d_sel, int64_t nsel, bool full,
                      void* leafsel, cudaStream_t st) {
  const int n = h ? P.n_l : P.n_u;
  const size_t state_bytes = sizeof(double) * 2 * ((size_t)1 << n);
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  const uint64_t K = cs.size();
  uint64_t cap = (uint64_t)(fr * 0.5 / state_bytes);
  if (cap < 1) cap = 1;
  const uint64_t batch = std::min(K, cap);
  DevBuf work, ids, table;
  if (!full) CK(work.alloc(state_bytes * batch, st));
  CK(ids.alloc(sizeof(uint64_t) * batch, st));
  CK(table.alloc(sizeof(NodeEntry) * batch, st));
  std::vector<uint64_t> hid(batch);
  std::vector<NodeEntry> htab(batch);
  PhaseScope ps(SIM_PHASE_PLAIN, st);
  // copies in row order, `batch` at a time (row r = position in the copy set)
  for (uint64_t k0 = 0; k0 < K; k0 += batch) {
    const uint64_t nb = std::min(batch, K - k0);
    for (uint64_t i = 0; i < nb; ++i) {
      hid[i] = cs.at(k0 + i);
      htab[i].node_id = hid[i];
      htab[i].parent_slot = 0;
      htab[i].dst_row = (int64_t)(k0 + i);
    }
    CK(cudaMemcpyAsync(ids.p, hid.data(), sizeof(uint64_t) * nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(table.p, htab.data(), sizeof(NodeEntry) * nb, cudaMemcpyHostToDevice, st));
    note_bytes((sizeof(uint64_t) + sizeof(NodeEntry)) * nb, 0);
    void* psi = full ? (void*)((char*)leafsel + k0 * state_bytes) : work.p;
    CK(launch_plain_init_zero(psi, n, (int64_t)nb, st));
    for (size_t t = 0; t < P.plain[h].size(); ++t) {
      const PlainLayer& L = P.plain[h][t];
      const OpRec* base = P.d_plain_ops[h] + P.plain_op_offsets[h][t];
      for (size_t g = 0; g < L.gates.size(); ++g) {
        PlainLaunch pl{n, L.gates[g].q, base + g, ids.as<uint64_t>(), (int64_t)nb, psi};
        CK(launch_plain_gate(pl, st));
      }
      for (size_t d = 0; d < L.diags.size(); ++d) {
        PlainLaunch pl{n, -1, base + L.gates.size() + d, ids.as<uint64_t>(), (int64_t)nb, psi};
        CK(launch_plain_diag(pl, st));
      }
    }
    if (!full) CK(launch_gather(work.p, n, table.as<NodeEntry>(), (int64_t)nb, d_sel, nsel, leafsel, 1, st));
    if (k0 + batch < K) CK(cudaStreamSynchronize(st));  // host arrays are reused
  }
  CK(cudaStreamSynchronize(st));
  return SIM_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_device_status(DeviceInfo* di) {
  int v = 0;
  CK(cudaMemcpy(&v, di->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v != 0) {
    CK(cudaMemset(di->d_status, 0, sizeof(int)));
    char buf[96];
    snprintf(buf, sizeof buf, "a bounded device wait gave up (code 0x%x)", v);
    return fail(SIM_ETIMEOUT, buf);
  }
  return SIM_OK;
}

// Contraction into device memory; with st_acc / st_hist (zeroed by the caller)
// also the statistics of the written block (fused into the split contraction's
// epilogue; a separate pass after the FP64 contraction).
// The contraction out[M][N] (+)= sum_k lA[k][m] * lB[k][n] of two leaf arrays
// ([K][M] and [K][N], complex64 or complex128 by precision) into device memory;
// nq sets w = 2^nq |A|^2 of the optional statistics; lcode / ucode the optional
// output-phase codes of the rows and columns.
int contract_impl(const void* lA, const void* lB, int64_t K, int64_t M, int64_t N, int precision, int contraction,
                  int accumulate, void* out, cudaStream_t st, int nq, double* st_acc = nullptr,
                  unsigned long long* st_hist = nullptr, const uint32_t* lcode = nullptr,
                  const uint32_t* ucode = nullptr) {
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return rc;
  if (contraction == SIM_FP64_PLAIN) {
    {
      PhaseScope ps(SIM_PHASE_FP64_GEMM, st);
      // output-phase cuts: a separate sign pass (before and after on an accumulated
      // block, which signs only this contraction's part)
      const bool sign = lcode && ucode;
      if (sign && accumulate) CK(launch_out_sign(out, 1, M, N, lcode, ucode, st));
      CK(launch_fp64_gemm(lA, lB, precision == SIM_C128_PLAIN, K, M, N, accumulate, out, st));
      if (sign) CK(launch_out_sign(out, 1, M, N, lcode, ucode, st));
    }
    if (st_acc && st_hist) {
      PhaseScope ps(SIM_PHASE_STATS, st);
      CK(launch_stats(out, 1, (uint64_t)(M * N), nq, st_acc, st_hist, st));
    }
    return SIM_OK;
  }
  if (contraction != SIM_SPLIT_BF16 && contraction != SIM_SPLIT_FP16)
    return fail(SIM_EINVAL, "unknown contraction");
  if (precision != SIM_C64) return fail(SIM_EINVAL, "split contractions need complex64 halves (SIM_C64)");
  const int fp16 = contraction == SIM_SPLIT_FP16;
  const int64_t kpad = ((2 * K + 63) / 64) * 64;
  const int64_t N2 = 2 * N;
  DevBuf ahi, alo, bhi, blo, sc;
  CK(ahi.alloc((size_t)M * kpad * 2, st));
  CK(alo.alloc((size_t)M * kpad * 2, st));
  CK(bhi.alloc((size_t)N2 * kpad * 2, st));
  CK(blo.alloc((size_t)N2 * kpad * 2, st));
  const float* sa = nullptr;
  const float* sb = nullptr;
  {
  PhaseScope ps(SIM_PHASE_PACK, st);
  if (fp16) {
    CK(sc.alloc(4 * sizeof(float), st));
    CK(launch_absmax_c64(lA, K * M, sc.as<float>(), st));
    CK(launch_absmax_c64(lB, K * N, sc.as<float>() + 2, st));
    sa = sc.as<float>() + 1;
    sb = sc.as<float>() + 3;
  }
  CK(launch_pack_a(lA, K, M, kpad, fp16, sa, ahi.p, alo.p, st));
  CK(launch_pack_b(lB, K, N, kpad, fp16, sb, bhi.p, blo.p, st));
  }
  TcGemmArgs g;
  g.a_hi = ahi.p; g.a_lo = alo.p; g.b_hi = bhi.p; g.b_lo = blo.p;
  g.M = M; g.N2 = N2; g.kpad = kpad;
  g.fp16 = fp16;
  g.scale_a = sa; g.scale_b = sb;
  g.accumulate = accumulate;
  g.C = out;
  g.group_m = 0;
  g.num_sms = di->num_sms;
  g.d_status = di->d_status;
  g.w_scale = std::ldexp(1.f, nq);
  g.st_acc = st_acc;
  g.st_hist = st_hist;
  g.out_lcode = lcode;
  g.out_ucode = ucode;
  PhaseScope ps(SIM_PHASE_CONTRACT, st);
  CK(launch_tc_gemm(g, st));
  return SIM_OK;
}

// Contraction of evolved halves: rows are the lower half's selection, columns the
// upper half's (Supplementary A, Eq. 8).
int amplitudes_impl(sim_halves h, int contraction, int accumulate, void* out, cudaStream_t st,
                    double* st_acc = nullptr, unsigned long long* st_hist = nullptr) {
  const int rc = check_split_bf16(contraction, (int64_t)h->cs.size(), false);
  if (rc) return rc;
  return contract_impl(h->leafsel[1], h->leafsel[0], (int64_t)h->cs.size(), h->nsel[1], h->nsel[0], h->precision,
                       contraction, accumulate, out, st, h->plan->circ.n, st_acc, st_hist, h->out_code[1],
                       h->out_code[0]);
}

// stats_out from the FP64 sums {sum |A|^2, sum ln w, count of w > 0} and the
// histogram of u = 1 - exp(-w): KS distance to the uniform CDF at the bin edges.
void finish_stats(const double a[3], const std::vector<unsigned long long>& hh, uint64_t count, int nq,
                  double stats_out[4], uint64_t* hist_out) {
  stats_out[0] = a[0];
  stats_out[1] = count ? a[0] * std::ldexp(1.0, nq) / (double)count : 0.0;
  stats_out[2] = a[2] > 0 ? a[1] / a[2] : -INFINITY;
  double tot = 0;
  for (auto v : hh) tot += (double)v;
  double ks = 0, cum = 0;
  for (int b = 0; b < SIM_KS_BINS; ++b) {
    cum += (double)hh[b];
    const double edge = (double)(b + 1) / SIM_KS_BINS;
    if (tot > 0) ks = std::max(ks, std::fabs(cum / tot - edge));
  }
  stats_out[3] = ks;
  if (hist_out)
    for (int b = 0; b < SIM_KS_BINS; ++b) hist_out[b] = hh[b];
}

}  // namespace

namespace sim {
TreeProgram rt_plan_tree(const HalfSchedule& S, const CopySet& cs, bool full, size_t budget) {
  return plan_tree(S, cs, full, budget, 0);
}
int rt_enqueue_tree(const CutPlan& P, int half, const TreeProgram& prog, void* const* lvl, const NodeEntry* table,
                    const uint64_t* d_sel, int64_t nsel, void* leafsel, cudaStream_t st, int kernel_choice,
                    int threads) {
  return enqueue_tree(P, half, prog, lvl, table, d_sel, nsel, leafsel, st, kernel_choice, threads);
}
cudaError_t rt_alloc(void** p, size_t n, cudaStream_t st) { return pool().alloc(p, n, st); }
void rt_free(void* p, cudaStream_t st) { pool().free(p, st, true); }
int rt_device(int** d_status, int* num_sms) {
  DeviceInfo* di = nullptr;
  const int rc = device_info(&di);
  if (rc) return rc;
  if (d_status) *d_status = di->d_status;
  if (num_sms) *num_sms = di->num_sms;
  return SIM_OK;
}
int rt_upload_plan(CutPlan& P, cudaStream_t st) { return upload_plan_ops(P, st); }
void rt_free_plan(CutPlan& P) { free_plan_ops(P); }
void rt_finish_stats(const double acc[3], const std::vector<unsigned long long>& hist, uint64_t count, int n_qubits,
                     double stats_out[4], uint64_t* hist_out) {
  finish_stats(acc, hist, count, n_qubits, stats_out, hist_out);
}

bool halves_view(const sim_halves_s* h, HalvesView* v) {
  if (!h || !v) return false;
  v->precision = h->precision;
  v->K = h->cs.size();
  for (int i = 0; i < 2; ++i) {
    v->nsel[i] = h->nsel[i];
    v->leafsel[i] = h->leafsel[i];
    v->out_code[i] = h->out_code[i];
  }
  return true;
}

int set_error(int code, const std::string& msg) { return fail(code, msg); }

int check_split_bf16(int contraction, int64_t copies, bool chained) {
  if (contraction != SIM_SPLIT_BF16) return SIM_OK;
  if (chained)
    return fail(SIM_EUNSUPPORTED,
                "split-bf16 is not offered for chained contractions (three or more parts): their roundings add up "
                "past 1e-5 of max|A|; use SIM_SPLIT_FP16");
  if (copies < kBf16MinCopies)
    return fail(SIM_EUNSUPPORTED, "split-bf16 needs at least " + std::to_string(kBf16MinCopies) +
                                      " copies in one contraction to stay within 1e-5 of max|A| (this one sums " +
                                      std::to_string(copies) + "); use SIM_SPLIT_FP16");
  return SIM_OK;
}

void note_launches(int phase, int count) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  if (phase < 0 || phase >= SIM_NUM_PHASES) return;
  P.all_launches[phase] += (uint64_t)count;
  if (P.on) P.launches[phase] += (uint64_t)count;
}
bool rt_profile_swap(bool on) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  const bool old = P.on;
  P.on = on;
  return old;
}
void rt_launch_totals(uint64_t out[SIM_NUM_PHASES]) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  for (int i = 0; i < SIM_NUM_PHASES; ++i) out[i] = P.all_launches[i];
}
void note_bytes(uint64_t h2d, uint64_t d2h) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  if (P.on) {
    P.h2d += h2d;
    P.d2h += d2h;
  }
}
}  // namespace sim

// ===========================================================================
// C-ABI
// ===========================================================================
#define API_BEGIN try {
#define API_END                                                          \
  }                                                                      \
  catch (const std::bad_alloc&) {                                        \
    return fail(SIM_ENOMEM, "host allocation failed");                   \
  }                                                                      \
  catch (const std::exception& ex) {                                     \
    return fail(SIM_EINVAL, std::string("internal error: ") + ex.what()); \
  }                                                                      \
  catch (...) {                                                          \
    return fail(SIM_EINVAL, "internal error");                           \
  }

extern "C" {

const char* sim_last_error(void) { return g_err.c_str(); }

int sim_version(void) { return 100; }

int sim_build_circuit(const sim_circuit_desc* desc, sim_circuit* out) {
  API_BEGIN
  if (!desc || !out) return fail(SIM_EINVAL, "desc and out must not be NULL");
  *out = nullptr;
  auto* c = new sim_circuit_s();
  std::string err;
  if (desc->gate_list)
    err = parse_circuit(desc->gate_list, c->c);
  else
    err = generate_circuit(desc->rows, desc->cols, desc->depth, desc->seed, desc->cut_row, c->c, desc->rule_t_in_pool);
  if (!err.empty()) {
    delete c;
    return fail(SIM_EINVAL, err);
  }
  *out = c;
  return SIM_OK;
  API_END
}

int sim_circuit_info(sim_circuit circ, int* n_qubits, int* depth, int* n_gates) {
  if (!circ) return fail(SIM_EINVAL, "NULL circuit");
  if (n_qubits) *n_qubits = circ->c.n;
  if (depth) *depth = circ->c.depth;
  if (n_gates) *n_gates = (int)circ->c.gates.size();
  return SIM_OK;
}

int sim_circuit_text(sim_circuit circ, char* buf, size_t cap, size_t* len_out) {
  API_BEGIN
  if (!circ) return fail(SIM_EINVAL, "NULL circuit");
  std::string s = circuit_text(circ->c);
  if (len_out) *len_out = s.size();
  if (buf && cap) {
    size_t n = std::min(cap - 1, s.size());
    memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return SIM_OK;
  API_END
}

int sim_cut(sim_circuit circ, int cut_row, sim_cut_plan* out, int* c_out, uint64_t* copies_out, int* n_upper_out,
            int* n_lower_out) {
  return sim_cut_ex(circ, cut_row, nullptr, out, c_out, copies_out, n_upper_out, n_lower_out);
}

int sim_cut_output_phases(sim_cut_plan plan, int32_t* pairs_out, int cap, int* n_out) {
  if (!plan || !n_out) return fail(SIM_EINVAL, "plan and n_out must not be NULL");
  const CutPlan& P = plan->p;
  *n_out = (int)P.out_cz.size();
  if (pairs_out)
    for (int i = 0; i < (int)P.out_cz.size() && i < cap; ++i) {
      pairs_out[2 * i] = P.out_cz[i].first;
      pairs_out[2 * i + 1] = P.out_cz[i].second;
    }
  return SIM_OK;
}

int sim_cut_ex(sim_circuit circ, int cut_row, const sim_cut_opts* opts, sim_cut_plan* out, int* c_out,
               uint64_t* copies_out, int* n_upper_out, int* n_lower_out) {
  API_BEGIN
  if (!circ || !out) return fail(SIM_EINVAL, "circuit and out must not be NULL");
  *out = nullptr;
  if (opts && (opts->output_phase_cuts < 0 || opts->output_phase_cuts > 1))
    return fail(SIM_EINVAL, "output_phase_cuts must be 0 or 1");
  auto* p = new sim_cut_s();
  std::string err = build_cut_plan(circ->c, cut_row, 0, p->p, 0, opts && opts->output_phase_cuts);
  if (!err.empty()) {
    delete p;
    return fail(err.find("at most") != std::string::npos || err.find("more than") != std::string::npos ||
                        err.find("not supported") != std::string::npos
                    ? SIM_EUNSUPPORTED
                    : SIM_EINVAL,
                err);
  }
  if (c_out) *c_out = p->p.c;
  if (copies_out) *copies_out = 1ull << p->p.c;
  if (n_upper_out) *n_upper_out = p->p.n_u;
  if (n_lower_out) *n_lower_out = p->p.n_l;
  *out = p;
  return SIM_OK;
  API_END
}

int sim_cut_list(sim_cut_plan plan, int32_t* cuts_out, int* n_equiv_out) {
  if (!plan) return fail(SIM_EINVAL, "NULL plan");
  const CutPlan& P = plan->p;
  if (cuts_out)
    for (int m = 0; m < P.c; ++m) {
      cuts_out[3 * m] = P.cuts[m].t;
      cuts_out[3 * m + 1] = P.cuts[m].h;
      cuts_out[3 * m + 2] = P.cuts[m].k;
    }
  if (n_equiv_out) *n_equiv_out = std::max(P.n_u, P.n_l) + P.c + 1;
  return SIM_OK;
}

int sim_plan_levels(sim_cut_plan plan, int half, int32_t* out, int cap, int* n_levels) {
  if (!plan || half < 0 || half > 1 || cap < 0 || (cap > 0 && !out)) return fail(SIM_EINVAL, "bad arguments");
  const HalfSchedule& S = plan->p.sched[half];
  const int J = (int)S.levels.size();
  for (int j = 0; j < J && j < cap; ++j) {
    const Level& L = S.levels[j];
    out[4 * j + 0] = L.branch_layer;
    out[4 * j + 1] = L.bits_before;
    out[4 * j + 2] = L.bits_total;
    out[4 * j + 3] = (int32_t)L.passes.size();
  }
  if (n_levels) *n_levels = J;
  return SIM_OK;
}

int sim_plan_sparse_qubits(sim_cut_plan plan, int half, int levels, int* nq_out) {
  if (!plan || half < 0 || half > 1 || !nq_out) return fail(SIM_EINVAL, "bad arguments");
  const HalfSchedule& S = plan->p.sched[half];
  if (levels < 1 || levels >= (int)S.levels.size())
    return fail(SIM_EINVAL, "levels must be at least 1 and below the number of copy-tree levels");
  *nq_out = leaf_ops(S, levels).nq;
  return SIM_OK;
}

int sim_plan_sparse_depth(sim_cut_plan plan, int half, uint64_t n_sel, int mode, int* depth_out) {
  if (!plan || half < 0 || half > 1 || !depth_out || mode < -1 || mode > 1) return fail(SIM_EINVAL, "bad arguments");
  const HalfSchedule& S = plan->p.sched[half];
  // a selection of every index takes the full route (no gather, no sparse leaves)
  *depth_out = n_sel >= ((uint64_t)1 << S.n) ? 0 : sparse_depth(S, (int64_t)n_sel, mode);
  return SIM_OK;
}

int sim_plan_schedule(sim_cut_plan plan, int half, int* levels, int* fused_passes, int* plain_passes) {
  if (!plan || half < 0 || half > 1) return fail(SIM_EINVAL, "bad plan or half");
  const HalfSchedule& S = plan->p.sched[half];
  int np = 0;
  for (const Level& L : S.levels) np += (int)L.passes.size();
  if (levels) *levels = (int)S.levels.size();
  if (fused_passes) *fused_passes = np;
  if (plain_passes) *plain_passes = S.plain_passes;
  return SIM_OK;
}

namespace {

// sim_evolve_halves and sim_evolve_halves_list: evolve the copies of `cs` (already
// validated against 2^c) for both halves and gather their leaves.
int evolve_halves_impl(sim_cut_plan plan, int precision, CopySet&& cs, const uint64_t* sel_u, uint64_t n_u,
                       const uint64_t* sel_l, uint64_t n_l, const sim_opts* opts, void* stream, sim_halves* out) {
  CutPlan& P = plan->p;
  const int want_fuse = (opts && opts->fuse_qubits) ? opts->fuse_qubits : P.fuse_qubits;
  const int want_order = opts ? opts->pass_order : P.pass_order;
  if (want_fuse != P.fuse_qubits || want_order != P.pass_order) {
    CutPlan np;
    // the plan's own cut row (n_u = b C), whatever row the circuit was built with
    std::string err = build_cut_plan(P.circ, P.n_u / P.circ.C, want_fuse, np, want_order, P.out_phase_cuts);
    if (!err.empty()) return fail(SIM_EINVAL, err);
    free_plan_ops(P);
    P = np;
  }
  if (opts && opts->sweep_threads && (opts->sweep_threads < 64 || opts->sweep_threads > 256 || opts->sweep_threads % 32))
    return fail(SIM_EINVAL, "sweep_threads must be a multiple of 32 in 64..256");
  if (opts && (opts->sparse_leaves < -1 || opts->sparse_leaves > 1))
    return fail(SIM_EINVAL, "sparse_leaves must be -1, 0 or 1");
  // the copy tree's node table is built on the host: keep one call bounded
  if (cs.size() > (1ull << 26))
    return fail(SIM_EUNSUPPORTED, "more than 2^26 copies in one call: evolve copy ranges and accumulate");
  const uint64_t* sels[2] = {sel_u, sel_l};
  const uint64_t nreq[2] = {n_u, n_l};
  const int nq[2] = {P.n_u, P.n_l};
  for (int hh = 0; hh < 2; ++hh) {
    if (sels[hh]) {
      if (nreq[hh] == 0) return fail(SIM_EINVAL, "empty selection");
      for (uint64_t i = 0; i < nreq[hh]; ++i)
        if (sels[hh][i] >> nq[hh]) return fail(SIM_EINVAL, "selected index out of range for its half");
    }
  }
  int rc = upload_plan_ops(P, (cudaStream_t)stream);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  auto* h = new sim_halves_s();
  h->plan = &P;
  h->precision = precision;
  h->cs = std::move(cs);
  h->stream = st;
  CK(cudaGetDevice(&h->device));
  const uint64_t K = h->cs.size();
  const size_t esz = precision == SIM_C64 ? 8 : 16;
  auto cleanup = [&]() { sim_destroy_halves(h); };
  for (int hh = 0; hh < 2; ++hh) {
    h->full[hh] = sels[hh] == nullptr;
    h->nsel[hh] = h->full[hh] ? (int64_t)1 << nq[hh] : (int64_t)nreq[hh];
    const size_t bytes = esz * (size_t)K * (size_t)h->nsel[hh];
    cudaError_t e = pool().alloc(&h->leafsel[hh], bytes, st);
    if (e != cudaSuccess) {
      cleanup();
      return fail(e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,
                  "cannot allocate the leaf buffers of the evolved halves");
    }
    if (!h->full[hh]) {
      e = pool().alloc(&h->d_sel[hh], sizeof(uint64_t) * h->nsel[hh], st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_sel[hh], sels[hh], sizeof(uint64_t) * h->nsel[hh], cudaMemcpyHostToDevice, st);
      note_bytes(sizeof(uint64_t) * h->nsel[hh], 0);
      if (e != cudaSuccess) {
        cleanup();
        return fail(SIM_ECUDA, std::string("selection upload: ") + cudaGetErrorString(e));
      }
    }
  }
  // output-phase cuts: per selected index of each half, the bits of its cuts
  if (!P.out_cz.empty()) {
    for (int hh = 0; hh < 2; ++hh) {
      std::vector<int> qs;
      for (const auto& pr : P.out_cz) qs.push_back(hh == 0 ? pr.first : pr.second - P.n_u);
      cudaError_t e = pool().alloc((void**)&h->out_code[hh], sizeof(uint32_t) * h->nsel[hh], st);
      if (e == cudaSuccess)
        e = launch_out_codes((const uint64_t*)h->d_sel[hh], h->nsel[hh], qs.data(), (int)qs.size(), h->out_code[hh],
                             st);
      if (e != cudaSuccess) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,
                    std::string("output-phase codes: ") + cudaGetErrorString(e));
      }
    }
  }
  for (int hh = 0; hh < 2; ++hh) {
    int r = precision == SIM_C64
                ? evolve_c64_half(P, hh, h->cs, (const uint64_t*)h->d_sel[hh], h->nsel[hh], h->full[hh],
                                  h->leafsel[hh], st, opts)
                : evolve_plain_half(P, hh, h->cs, (const uint64_t*)h->d_sel[hh], h->nsel[hh], h->full[hh],
                                    h->leafsel[hh], st);
    if (r) {
      std::string keep = g_err;
      cleanup();
      return fail(r, keep);
    }
  }
  *out = h;
  return SIM_OK;
}

}  // namespace

int sim_evolve_halves(sim_cut_plan plan, int precision, uint64_t copy_begin, uint64_t copy_end, const uint64_t* sel_u,
                      uint64_t n_u, const uint64_t* sel_l, uint64_t n_l, const sim_opts* opts, void* stream,
                      sim_halves* out) {
  API_BEGIN
  if (!plan || !out) return fail(SIM_EINVAL, "plan and out must not be NULL");
  *out = nullptr;
  if (precision != SIM_C64 && precision != SIM_C128_PLAIN) return fail(SIM_EINVAL, "unknown precision");
  const uint64_t copies = 1ull << plan->p.c;
  if (copy_begin >= copy_end || copy_end > copies) return fail(SIM_EINVAL, "copy range must satisfy begin < end <= 2^c");
  CopySet cs;
  cs.kb = copy_begin;
  cs.ke = copy_end;
  return evolve_halves_impl(plan, precision, std::move(cs), sel_u, n_u, sel_l, n_l, opts, stream, out);
  API_END
}

int sim_evolve_halves_list(sim_cut_plan plan, int precision, const uint64_t* copies, uint64_t n_copies,
                           const uint64_t* sel_u, uint64_t n_u, const uint64_t* sel_l, uint64_t n_l,
                           const sim_opts* opts, void* stream, sim_halves* out) {
  API_BEGIN
  if (!plan || !out || !copies) return fail(SIM_EINVAL, "plan, copies and out must not be NULL");
  *out = nullptr;
  if (precision != SIM_C64 && precision != SIM_C128_PLAIN) return fail(SIM_EINVAL, "unknown precision");
  if (n_copies == 0) return fail(SIM_EINVAL, "empty copy list");
  const uint64_t total = 1ull << plan->p.c;
  CopySet cs;
  cs.list.assign(copies, copies + n_copies);
  cs.row.reserve((size_t)n_copies);
  for (uint64_t i = 0; i < n_copies; ++i) {
    if (cs.list[i] >= total) return fail(SIM_EINVAL, "copy index out of range (must be < 2^c)");
    if (!cs.row.emplace(cs.list[i], (int64_t)i).second) return fail(SIM_EINVAL, "copy indices must be distinct");
  }
  return evolve_halves_impl(plan, precision, std::move(cs), sel_u, n_u, sel_l, n_l, opts, stream, out);
  API_END
}

int sim_halves_leaf(sim_halves h, int half, uint64_t copy, void* out_dev, void* stream) {
  API_BEGIN
  if (!h || half < 0 || half > 1 || !out_dev) return fail(SIM_EINVAL, "bad arguments");
  if (!h->cs.contains(copy)) return fail(SIM_EINVAL, "copy not among the evolved copies");
  const size_t esz = h->precision == SIM_C64 ? 8 : 16;
  const size_t bytes = esz * (size_t)h->nsel[half];
  CK(cudaMemcpyAsync(out_dev, (const char*)h->leafsel[half] + (size_t)h->cs.row_of(copy) * bytes, bytes,
                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return SIM_OK;
  API_END
}

int sim_amplitudes(sim_halves h, int contraction, int accumulate, void* out, void* stream) {
  API_BEGIN
  if (!h || !out) return fail(SIM_EINVAL, "halves and out must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (is_device_ptr(out)) return amplitudes_impl(h, contraction, accumulate, out, st);
  // host output: compute into a device staging buffer, copy back, wait
  const size_t esz = contraction == SIM_FP64_PLAIN ? 16 : 8;
  const size_t bytes = esz * (size_t)h->nsel[0] * (size_t)h->nsel[1];
  DevBuf stage;
  CK(stage.alloc(bytes, st));
  if (accumulate) CK(cudaMemcpyAsync(stage.p, out, bytes, cudaMemcpyHostToDevice, st));
  note_bytes(accumulate ? bytes : 0, bytes);
  int rc = amplitudes_impl(h, contraction, accumulate, stage.p, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, stage.p, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SIM_OK;
  API_END
}

int sim_stats(const void* amps, int is_c128, uint64_t count, int n_qubits, double stats_out[4], uint64_t* hist_out,
              void* stream) {
  API_BEGIN
  if (!amps || !stats_out) return fail(SIM_EINVAL, "amps and stats_out must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf acc, hist;
  CK(acc.alloc(4 * sizeof(double), st));
  CK(hist.alloc(SIM_KS_BINS * sizeof(unsigned long long), st));
  {
    PhaseScope ps(SIM_PHASE_STATS, st);
    CK(launch_stats(amps, is_c128, count, n_qubits, acc.as<double>(), hist.as<unsigned long long>(), st));
  }
  note_bytes(0, 3 * sizeof(double) + SIM_KS_BINS * sizeof(unsigned long long));
  double a[3];
  std::vector<unsigned long long> hh(SIM_KS_BINS);
  CK(cudaMemcpyAsync(a, acc.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hh.data(), hist.p, SIM_KS_BINS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  finish_stats(a, hh, count, n_qubits, stats_out, hist_out);
  return SIM_OK;
  API_END
}

int sim_amplitudes_stats(sim_halves h, int contraction, int accumulate, void* out_dev, double stats_out[4],
                         uint64_t* hist_out, void* stream) {
  API_BEGIN
  if (!h || !out_dev || !stats_out) return fail(SIM_EINVAL, "halves, out_dev and stats_out must not be NULL");
  if (!is_device_ptr(out_dev)) return fail(SIM_EINVAL, "sim_amplitudes_stats writes device memory only");
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf acc, hist;
  CK(acc.alloc(4 * sizeof(double), st));
  CK(hist.alloc(SIM_KS_BINS * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(acc.p, 0, 3 * sizeof(double), st));
  CK(cudaMemsetAsync(hist.p, 0, SIM_KS_BINS * sizeof(unsigned long long), st));
  int rc = amplitudes_impl(h, contraction, accumulate, out_dev, st, acc.as<double>(), hist.as<unsigned long long>());
  if (rc) return rc;
  note_bytes(0, 3 * sizeof(double) + SIM_KS_BINS * sizeof(unsigned long long));
  double a[3];
  std::vector<unsigned long long> hh(SIM_KS_BINS);
  CK(cudaMemcpyAsync(a, acc.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hh.data(), hist.p, SIM_KS_BINS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  finish_stats(a, hh, (uint64_t)h->nsel[0] * (uint64_t)h->nsel[1], h->plan->circ.n, stats_out, hist_out);
  return SIM_OK;
  API_END
}

int sim_select(int nq_u, uint64_t n_u, int nq_l, uint64_t n_l, uint64_t seed, uint64_t* sel_u_out,
               uint64_t* sel_l_out) {
  API_BEGIN
  if (nq_u < 0 || nq_u > 40 || nq_l < 0 || nq_l > 40) return fail(SIM_EINVAL, "qubit counts must be in 0..40");
  if (!sel_u_out || !sel_l_out) return fail(SIM_EINVAL, "outputs must not be NULL");
  uint64_t state = seed;
  std::vector<uint64_t> a, b;
  select_indices(nq_u, n_u, state, a);
  select_indices(nq_l, n_l, state, b);
  std::copy(a.begin(), a.end(), sel_u_out);
  std::copy(b.begin(), b.end(), sel_l_out);
  return SIM_OK;
  API_END
}

int sim_sample(sim_cut_plan plan, uint64_t n_u, uint64_t n_l, uint64_t seed, uint64_t* sel_u_out, uint64_t* sel_l_out,
               void* amps_dev_out, double stats_out[4], const sim_opts* opts, void* stream) {
  API_BEGIN
  if (!plan || !sel_u_out || !sel_l_out || !amps_dev_out) return fail(SIM_EINVAL, "NULL argument");
  CutPlan& P = plan->p;
  const uint64_t uu = std::min<uint64_t>(n_u, 1ull << P.n_u), ll = std::min<uint64_t>(n_l, 1ull << P.n_l);
  int rc = sim_select(P.n_u, uu, P.n_l, ll, seed, sel_u_out, sel_l_out);
  if (rc) return rc;
  sim_halves h = nullptr;
  rc = sim_evolve_halves(plan, SIM_C64, 0, 1ull << P.c, sel_u_out, uu, sel_l_out, ll, opts, stream, &h);
  if (rc) return rc;
  if (stats_out)
    rc = sim_amplitudes_stats(h, SIM_SPLIT_FP16, 0, amps_dev_out, stats_out, nullptr, stream);
  else
    rc = sim_amplitudes(h, SIM_SPLIT_FP16, 0, amps_dev_out, stream);
  sim_destroy_halves(h);
  if (rc) return rc;
  return sim_status(stream);
  API_END
}

int sim_status(void* stream) {
  API_BEGIN
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaGetLastError());
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return rc;
  return check_device_status(di);
  API_END
}

int sim_release_cache(void) {
  pool().release(-1);
  return SIM_OK;
}

int sim_profile_enable(int on) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  P.on = on != 0;
  return SIM_OK;
}

int sim_profile_read(double* ms_out, uint64_t* instances_out, uint64_t* launches_out, uint64_t* bytes_out,
                     int reset) {
  API_BEGIN
  Profiler& P = prof();
  std::lock_guard<std::mutex> lk(P.mu);
  for (auto& r : P.recs) {
    CK(cudaEventSynchronize(r.b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    P.ms[r.phase] += ms;
    P.inst[r.phase] += 1;
    P.spare.push_back(r.a);
    P.spare.push_back(r.b);
  }
  P.recs.clear();
  for (int i = 0; i < SIM_NUM_PHASES; ++i) {
    if (ms_out) ms_out[i] = P.ms[i];
    if (instances_out) instances_out[i] = P.inst[i];
    if (launches_out) launches_out[i] = P.launches[i];
  }
  if (bytes_out) {
    bytes_out[0] = P.h2d;
    bytes_out[1] = P.d2h;
  }
  if (reset) {
    for (int i = 0; i < SIM_NUM_PHASES; ++i) {
      P.ms[i] = 0;
      P.inst[i] = 0;
      P.launches[i] = 0;
    }
    P.h2d = P.d2h = 0;
  }
  return SIM_OK;
  API_END
}

void sim_destroy_circuit(sim_circuit circ) { delete circ; }

void sim_destroy_cut(sim_cut_plan plan) {
  if (!plan) return;
  free_plan_ops(plan->p);
  delete plan;
}

int sim_selftest_wait(int limit_ms, void* stream) {
  API_BEGIN
  if (limit_ms < 1 || limit_ms > 10000) return fail(SIM_EINVAL, "limit_ms must be in 1..10000");
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  CK(launch_wait_selftest(di->d_status, (unsigned long long)limit_ms * 1000000ull, st));
  note_launches(SIM_PHASE_CONTRACT, 1);
  CK(cudaStreamSynchronize(st));
  return check_device_status(di);
  API_END
}

int sim_cut_multi(sim_circuit circ, int n_cut_rows, const int* cut_rows, sim_multi_plan* out, int* parts_out,
                  int* c_out, int* nq_out) {
  API_BEGIN
  if (!circ || !out || !cut_rows || n_cut_rows < 1) return fail(SIM_EINVAL, "circuit, cut rows and out are required");
  *out = nullptr;
  auto* m = new sim_multi_s();
  std::string err = build_multi_plan(circ->c, std::vector<int>(cut_rows, cut_rows + n_cut_rows), 0, 0, m->mp);
  if (!err.empty()) {
    delete m;
    return fail(err.find("more than") != std::string::npos || err.find("only") != std::string::npos
                    ? SIM_EUNSUPPORTED
                    : SIM_EINVAL,
                err);
  }
  if (parts_out) *parts_out = m->mp.t;
  if (c_out)
    for (int j = 1; j < m->mp.t; ++j) c_out[j - 1] = m->mp.c[j];
  if (nq_out)
    for (int p = 0; p < m->mp.t; ++p) nq_out[p] = m->mp.nq[p];
  *out = m;
  return SIM_OK;
  API_END
}

int sim_multi_amplitudes(sim_multi_plan plan, int precision, int contraction, const uint64_t* const* sels,
                         const uint64_t* nsel, void* out_dev, const sim_opts* opts, void* stream) {
  API_BEGIN
  if (!plan || !out_dev) return fail(SIM_EINVAL, "plan and out_dev must not be NULL");
  if (!is_device_ptr(out_dev)) return fail(SIM_EINVAL, "sim_multi_amplitudes writes device memory only");
  const bool split = contraction == SIM_SPLIT_BF16 || contraction == SIM_SPLIT_FP16;
  if (!((precision == SIM_C64 && split) || (precision == SIM_C128_PLAIN && contraction == SIM_FP64_PLAIN)))
    return fail(SIM_EINVAL, "multi-part cuts take SIM_C64 with a split contraction or SIM_C128_PLAIN with SIM_FP64_PLAIN");
  if (opts && opts->sweep_threads && (opts->sweep_threads < 64 || opts->sweep_threads > 256 || opts->sweep_threads % 32))
    return fail(SIM_EINVAL, "sweep_threads must be a multiple of 32 in 64..256");
  if (opts && (opts->sparse_leaves < -1 || opts->sparse_leaves > 1))
    return fail(SIM_EINVAL, "sparse_leaves must be -1, 0 or 1");
  MultiPlan& M = plan->mp;
  cudaStream_t st = (cudaStream_t)stream;
  // re-plan for another fuse width or pass order
  const int want_fuse = (opts && opts->fuse_qubits) ? opts->fuse_qubits : M.part[0].fuse_qubits;
  const int want_order = opts ? opts->pass_order : M.part[0].pass_order;
  if (want_fuse != M.part[0].fuse_qubits || want_order != M.part[0].pass_order) {
    std::vector<int> rows;
    for (int p = 1; p < M.t; ++p) rows.push_back(M.offset[p] / M.circ.C);
    MultiPlan np;
    std::string err = build_multi_plan(M.circ, rows, want_fuse, want_order, np);
    if (!err.empty()) return fail(SIM_EINVAL, err);
    for (auto& P : M.part) free_plan_ops(P);
    M = np;
  }
  const int t = M.t;
  {
    const int rc = check_split_bf16(contraction, t > 1 ? (int64_t)1 << M.c[1] : 1, t > 2);
    if (rc) return rc;
  }
  // every copy of every part is listed and evolved: keep the lists (and the host
  // memory behind them) bounded, before any work starts
  for (int p = 0; p < t; ++p)
    if ((p > 0 ? M.c[p] : 0) + (p + 1 < t ? M.c[p + 1] : 0) > 24)
      return fail(SIM_EUNSUPPORTED, "a part has more than 2^24 copies");
  const size_t esz = precision == SIM_C64 ? 8 : 16;
  std::vector<int64_t> n(t);
  std::vector<DevBuf> dsel(t), leaves(t);
  for (int p = 0; p < t; ++p) {
    const bool full = !sels || !sels[p];
    n[p] = full ? (int64_t)1 << M.nq[p] : (int64_t)nsel[p];
    if (!full) {
      if (n[p] == 0) return fail(SIM_EINVAL, "empty selection");
      for (int64_t i = 0; i < n[p]; ++i)
        if (sels[p][i] >> M.nq[p]) return fail(SIM_EINVAL, "selected index out of range for its part");
      CK(dsel[p].alloc(sizeof(uint64_t) * n[p], st));
      CK(cudaMemcpyAsync(dsel[p].p, sels[p], sizeof(uint64_t) * n[p], cudaMemcpyHostToDevice, st));
      note_bytes(sizeof(uint64_t) * n[p], 0);
    }
    // the part's copies in contraction order: the bits of the boundary above it
    // outermost, those of the boundary below it innermost
    const int ca = p > 0 ? M.c[p] : 0, cb = p + 1 < t ? M.c[p + 1] : 0;
    CopySet cs;
    cs.list.reserve((size_t)1 << (ca + cb));
    for (uint64_t la = 0; la < (1ull << ca); ++la)
      for (uint64_t lb = 0; lb < (1ull << cb); ++lb) {
        uint64_t k = 0;
        for (size_t m = 0; m < M.slot_bits[p].size(); ++m) {
          const auto& jb = M.slot_bits[p][m];
          const uint64_t v = jb.first == p ? la : lb;
          k |= ((v >> jb.second) & 1ull) << m;
        }
        cs.row[k] = (int64_t)cs.list.size();
        cs.list.push_back(k);
      }
    int rc = upload_plan_ops(M.part[p], st);
    if (rc) return rc;
    CK(leaves[p].alloc(esz * cs.size() * (size_t)n[p], st));
    rc = precision == SIM_C64
             ? evolve_c64_half(M.part[p], 0, cs, (const uint64_t*)dsel[p].p, n[p], full, leaves[p].p, st, opts)
             : evolve_plain_half(M.part[p], 0, cs, (const uint64_t*)dsel[p].p, n[p], full, leaves[p].p, st);
    if (rc) return rc;
  }
  // the multi-way sum, one boundary at a time from the top: after part p the
  // partial product is [l_{p+1}][x_p][x_{p-1} .. x_0], the next contraction's
  // right operand over the copy bits l_{p+1}
  DevBuf tb[2];
  const void* right = leaves[0].p;
  int64_t ncols = n[0];
  for (int p = 1; p < t; ++p) {
    const int64_t K = (int64_t)1 << M.c[p];
    const int64_t rows = (p + 1 < t ? ((int64_t)1 << M.c[p + 1]) : 1) * n[p];
    void* dst = out_dev;
    if (p + 1 < t) {
      CK(tb[p & 1].alloc(esz * (size_t)rows * (size_t)ncols, st));
      dst = tb[p & 1].p;
    }
    int rc = contract_impl(leaves[p].p, right, K, rows, ncols, precision, contraction, 0, dst, st, M.circ.n);
    if (rc) return rc;
    right = dst;
    ncols *= n[p];
  }
  CK(cudaStreamSynchronize(st));
  return SIM_OK;
  API_END
}

void sim_destroy_multi(sim_multi_plan plan) {
  if (!plan) return;
  for (auto& P : plan->mp.part) free_plan_ops(P);
  delete plan;
}

void sim_destroy_halves(sim_halves h) {
  if (!h) return;
  // the buffers go back to the pool after the work enqueued so far on the halves'
  // stream (stream-ordered: no host wait)
  for (int i = 0; i < 2; ++i) {
    pool().free(h->leafsel[i], h->stream, true);
    pool().free(h->d_sel[i], h->stream, true);
    pool().free(h->out_code[i], h->stream, true);
  }
  delete h;
}

}  // extern "C"
