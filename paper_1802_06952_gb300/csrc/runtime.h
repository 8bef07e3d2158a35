// Runtime pieces shared by the single-call entry points (api.cpp) and the batch
// runner (batch.cpp): copy sets, copy-tree programs, the stream-ordered device
// pool and the per-device status word.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <unordered_map>
#include <vector>

#include "sim_internal.h"

namespace sim {

// The copies of an evolved halves object, in leaf-row order: the range [kb, ke) or
// an explicit list of distinct copy indices.
struct CopySet {
  uint64_t kb = 0, ke = 0;
  std::vector<uint64_t> list;                 // empty: the range
  std::unordered_map<uint64_t, int64_t> row;  // list: copy index -> row
  uint64_t size() const { return list.empty() ? ke - kb : (uint64_t)list.size(); }
  uint64_t at(uint64_t i) const { return list.empty() ? kb + i : list[i]; }
  bool contains(uint64_t k) const { return list.empty() ? (k >= kb && k < ke) : row.count(k) > 0; }
  int64_t row_of(uint64_t k) const { return list.empty() ? (int64_t)(k - kb) : row.at(k); }
};

// One launch of a copy-tree program: a fused pass over a chunk of a level's nodes,
// or (pass < 0) the gather of a chunk of leaves into the selected rows.
struct LaunchRec {
  int level, pass;       // pass < 0: gather
  int64_t table_off, nslots;
  int src_buf, dst_buf;  // buffer ids: level index, or -1 = the leaf rows
};

// Host-built program for the copy tree of one half (Section 2.3.2): node table,
// launches in order, and the chunk capacity (nodes) of each level's buffer.
struct TreeProgram {
  std::vector<NodeEntry> table;
  std::vector<LaunchRec> launches;
  std::vector<int64_t> level_cap;
};

// Build the program for the copies of cs; level buffers are sized so that all of
// them together stay within budget bytes (at least one node per level).
// full: leaves are written straight into their rows (no selection, no gather).
TreeProgram rt_plan_tree(const HalfSchedule& S, const CopySet& cs, bool full, size_t budget);

// Enqueue a program's launches on st.  lvl[j]: level j's chunk buffer (complex64
// states); table: the device copy of prog.table; leafsel: the leaf rows.
// kernel_choice: 1 forces the staged sweep, otherwise the register-blocked sweep
// wherever a pass allows it; threads: block size of the staged sweep.
int rt_enqueue_tree(const CutPlan& P, int half, const TreeProgram& prog, void* const* lvl, const NodeEntry* table,
                    const uint64_t* d_sel, int64_t nsel, void* leafsel, cudaStream_t st, int kernel_choice,
                    int threads);

// Stream-ordered caching pool of device memory (blocks stay cached until
// sim_release_cache or an allocation failure).
// pool blocks for work on stream st; freed blocks return to the pool after the
// work enqueued so far on st (stream-ordered reuse)
cudaError_t rt_alloc(void** p, size_t n, cudaStream_t st);
void rt_free(void* p, cudaStream_t st);

// Device status word (timeouts of bounded device waits) and SM count of the
// current device.
int rt_device(int** d_status, int* num_sms);

// Op tables of a plan in device memory.
int rt_upload_plan(CutPlan& P, cudaStream_t st);
void rt_free_plan(CutPlan& P);

// Profiler switch (returns the previous state) and the launch counts per phase
// since the library was loaded (counted whether or not the profiler is on).
bool rt_profile_swap(bool on);
void rt_launch_totals(uint64_t out[SIM_NUM_PHASES]);

// stats_out from the FP64 sums {sum |A|^2, sum ln w, count of w > 0} and the
// u-histogram of count amplitudes of an n_qubits circuit.
void rt_finish_stats(const double acc[3], const std::vector<unsigned long long>& hist, uint64_t count, int n_qubits,
                     double stats_out[4], uint64_t* hist_out);

}  // namespace sim
