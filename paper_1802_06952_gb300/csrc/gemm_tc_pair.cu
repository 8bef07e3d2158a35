// Amplitude contraction (Supplementary A, Eq. 8) on CTA pairs: the same split-
// precision GEMM as gemm_tc.cu, issued as tcgen05.mma.cta_group::2 with M = 256,
// N = 256, K = 16 over a cluster of two CTAs on two SMs.
//
// Each CTA of the pair holds 128 rows of the A tile and 128 of the 256 rows of the
// B tile (one half of the output columns) in its own shared memory, and 128 rows x
// 256 columns of the fp32 accumulator in its own tensor memory.  A stage holds one
// 64-wide k-block of both split parts of both operands (A hi, A lo, B hi, B lo) and
// the MMA issuer takes the three split products hi*hi, hi*lo, lo*hi from them, so
// each operand tile crosses shared memory once per k-block: 64 KB written and 96 KB
// read per SM for three k-block products, against 96 + 96 KB when every product
// loads its own pair of tiles.  Shared-memory bandwidth, not the tensor pipe, is
// what bounds this kernel.
//
// Roles (both CTAs run the same warps):
//   warp 0     TMA loads of the CTA's own A and B halves into its own stage ring.
//              Both CTAs' copies complete on the leader's (rank 0) "full" barrier
//              (cp.async.bulk.tensor .cta_group::2), which the leader's producer
//              arms with the bytes of both halves.
//   warp 1     TMEM allocation (cta_group::2, both CTAs); in the leader, the MMA
//              issuer, which commits to the "empty" barriers and accumulator
//              barriers of both CTAs with one multicast commit
//   warps 2-9  epilogue of the CTA's 128 accumulator rows: tensor memory to
//              registers (statistics), shared-memory staging, TMA store (or TMA
//              reduce-add when accumulating) of 32 x 16-float boxes; each warp
//              releases the accumulator on the leader's barrier (a remote arrive
//              from the peer)
// Before leaving its loop each producer waits until the MMAs have released every
// stage it filled, so no copy is in flight when the pair exits.  All mbarrier waits
// are bounded as in gemm_tc.cu.  Both CTAs reach the final cluster barrier on every
// path, after which tensor memory is released.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <cstdlib>
#include <mutex>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace sim {
namespace {

constexpr int BM = 128;               // rows of A (and of the accumulator) per CTA
constexpr int BN = 256;               // output columns per pair tile
constexpr int BNH = 128;              // B rows per CTA
constexpr int BK = 64;
constexpr int UMMA_K = 16;
constexpr int A_BYTES = BM * BK * 2;   // 16 KB
constexpr int B_BYTES = BNH * BK * 2;  // 16 KB
constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);  // hi and lo tiles of both operands
constexpr int ACC_COLS = BN;
constexpr int TMEM_COLS = 2 * ACC_COLS;
constexpr int HIST_BYTES = SIM_KS_BINS * 4;
// Shared memory of one CTA: STG operand stages, NBUF output staging buffers of 32 rows
// x SW floats per epilogue warp (none for direct epilogues), barriers, histogram.
template <int STG, int SW, int NBUF, int EW, bool DIRECT = false>
struct PairSmem {
  // direct epilogues store from registers: no staging buffers
  static constexpr int EPI_BYTES = DIRECT ? 0 : EW * NBUF * 32 * SW * 4;
  static constexpr int BYTES = 1024 + STG * STAGE_BYTES + EPI_BYTES + 512 + HIST_BYTES;
  static_assert(BYTES <= 232448, "shared memory above the 227 KB per-block limit");
};
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr int kChunkCopies = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// arrive on a barrier given by its shared::cluster address (own CTA or the peer)
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > limit_ns || it > (1u << 30)) return false;
    }
  }
}

// Health check of the bounded waits: one thread waits, with the helper the
// contraction kernels use, for phase 0 of a fresh barrier that nothing arrives on.
// The wait gives up after limit_ns, the timeout is recorded in the status word and
// the kernel returns: no trap, no hang, the context stays usable.
__global__ void wait_selftest_kernel(int* d_status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0u, &abort_flag, limit_ns))
    atomicExch(d_status, SIM_TIMEOUT_CODE_SELFTEST);
}

// copy into this CTA's shared memory, completing on a barrier of either CTA of the
// pair (bar is a shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: SW128 K-major, 1024 B between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// kind::f16 instruction descriptor: D fp32, A/B bf16 or fp16, K-major, N = 256, M = 256
__host__ __device__ constexpr uint32_t instr_desc_pair(bool fp16) {
  return (1u << 4) | ((fp16 ? 0u : 1u) << 7) | ((fp16 ? 0u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(256 >> 4) << 24);
}
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// arrive once on the barrier at this shared-memory offset in both CTAs of the pair
// when all prior MMAs of this thread have completed
__device__ __forceinline__ void umma_commit_both(uint32_t bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void umma_commit_local(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// start a 32-lane x SW-column accumulator load; the registers are valid only after
// tmem_wait on the same array
template <int SW>
__device__ __forceinline__ void tmem_ld_async(uint32_t taddr, uint32_t (&r)[SW]) {
  if constexpr (SW == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    static_assert(SW == 8, "8- or 16-column steps");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  }
}
// wait for this thread's outstanding accumulator loads; the array is threaded through
// as an operand so that no use of it is scheduled before the wait
template <int SW>
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[SW]) {
  if constexpr (SW == 16) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
  } else {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
  }
}
// TMA store / reduce-add of one staged 32-row box into the output (bulk-group
// completion); x is the column (float) coordinate, y the row
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   map),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one committed group may still be reading shared memory
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed group has completed its global writes
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n\tfence.proxy.async.global;" ::: "memory");
}

struct PairTileMap {
  int64_t num_mb, num_nb;  // m in 256-row pair tiles, n in 256-column tiles
  int group;
  __device__ void tile(int64_t t, int64_t& mb, int64_t& nb) const {
    const int64_t per_group = (int64_t)group * num_nb;
    const int64_t g = t / per_group;
    const int64_t first = g * group;
    const int64_t gs = (num_mb - first) < group ? (num_mb - first) : group;
    const int64_t local = t - g * per_group;
    mb = first + local % gs;
    nb = local / gs;
  }
};

struct PairArgs {
  int64_t M, N2;
  int nkb, ckb, nchunks;
  PairTileMap tm;
  int64_t num_tiles;
  const float* scale_a;
  const float* scale_b;
  int accumulate;
  float* C;
  int* d_status;
  float w_scale;
  double* st_acc;
  unsigned long long* st_hist;
  const uint32_t* out_lcode;  // output-phase codes of the rows and complex columns (NULL: none)
  const uint32_t* out_ucode;
  // k-blocks of chunk c (each one stage: the three split products of one k-block)
  __device__ int chunk_kblocks(int c) const {
    const int b0 = c * ckb;
    const int b1 = b0 + ckb < nkb ? b0 + ckb : nkb;
    return b1 - b0;
  }
};

// STATS: fuse the FP64 statistics of the final amplitudes into the epilogue.
// STG: operand stages.  SW: accumulator columns per epilogue step (8 or 16), which
// sets the staging box (32 rows x SW floats, 32- or 64-byte TMA swizzle).
template <bool STATS, bool SIGN, int STG, int SW, int NBUF, int UNR, int EW, bool DIRECT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(32 * (2 + EW), 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA_hi, const __grid_constant__ CUtensorMap mapA_lo,
                        const __grid_constant__ CUtensorMap mapB_hi, const __grid_constant__ CUtensorMap mapB_lo,
                        const __grid_constant__ CUtensorMap mapC, PairArgs args, uint32_t idesc) {
  using L = PairSmem<STG, SW, NBUF, EW, DIRECT>;
  constexpr int THREADS = 32 * (2 + EW);
  constexpr int COLS = BN / (EW / 4);  // accumulator columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage s: A hi, A lo at sA + s * 2 A_BYTES; B hi, B lo at sB + s * 2 B_BYTES
  uint8_t* sA = smem;
  uint8_t* sB = smem + STG * 2 * A_BYTES;
  float* sEpi = (float*)(sB + STG * 2 * B_BYTES);
  uint64_t* bars = (uint64_t*)((uint8_t*)sEpi + L::EPI_BYTES);
  uint64_t* full = bars;                  // leader: both halves landed  (count 1 + tx)
  uint64_t* empty = bars + STG;           // leader's MMAs done          (count 1, multicast commit)
  uint64_t* acc_full = bars + 2 * STG;    // accumulator ready           (count 1, multicast commit)
  uint64_t* acc_empty = acc_full + 2;     // leader: both epilogues done (count 16)
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  unsigned int* s_hist = (unsigned int*)((uint8_t*)bars + 512);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const uint32_t rank = cta_rank();
  const bool leader = rank == 0;
  const int64_t pair = blockIdx.x / 2;
  const int64_t npairs = gridDim.x / 2;

  if (STATS)
    for (int i = threadIdx.x; i < SIM_KS_BINS; i += THREADS) s_hist[i] = 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STG; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&acc_full[a]), 1);
      mbar_init(smem_u32(&acc_empty[a]), 2 * EW);
    }
    mbar_init(smem_u32(mma_done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&mapA_hi);
    prefetch_map(&mapA_lo);
    prefetch_map(&mapB_hi);
    prefetch_map(&mapB_lo);
    prefetch_map(&mapC);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();  // barriers of both CTAs initialised, tensor memory allocated
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer (both CTAs, own halves) ----------------
    if (lane == 0) {
      int issued_parity[STG];
      for (int s = 0; s < STG; ++s) issued_parity[s] = -1;
      const uint32_t full0 = map_to(smem_u32(&full[0]), 0);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t t = pair; t < args.num_tiles && ok; t += npairs) {
        int64_t mb, nb;
        args.tm.tile(t, mb, nb);
        const int arow = (int)(mb * 2 * BM + rank * BM);
        const int brow = (int)(nb * BN + rank * BNH);
        for (int c = 0; c < args.nchunks && ok; ++c)
          for (int i = 0; i < args.chunk_kblocks(c); ++i) {
            if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            const int kx = (c * args.ckb + i) * BK;
            const uint32_t fb = full0 + (uint32_t)(stage * sizeof(uint64_t));
            // both CTAs' four tiles complete on the leader's barrier
            if (leader) mbar_arrive_expect_tx(smem_u32(&full[stage]), 2 * STAGE_BYTES);
            uint8_t* a_st = sA + stage * 2 * A_BYTES;
            uint8_t* b_st = sB + stage * 2 * B_BYTES;
            tma_load_2d_pair(smem_u32(a_st), &mapA_hi, fb, kx, arow);
            tma_load_2d_pair(smem_u32(a_st + A_BYTES), &mapA_lo, fb, kx, arow);
            tma_load_2d_pair(smem_u32(b_st), &mapB_hi, fb, kx, brow);
            tma_load_2d_pair(smem_u32(b_st + B_BYTES), &mapB_lo, fb, kx, brow);
            issued_parity[stage] = (int)phase;
            if (++stage == STG) {
              stage = 0;
              phase ^= 1u;
            }
          }
      }
      if (!ok) {
        if (args.d_status) atomicExch(args.d_status, SIM_TIMEOUT_CODE_TMA);
        *abort_flag = 1;
      }
      // the last fill of each stage is released by the leader's commit once the MMAs
      // that read it (and so the copy itself) are complete
      volatile int dummy = 0;
      for (int s = 0; s < STG; ++s)
        if (issued_parity[s] >= 0) mbar_wait(smem_u32(&empty[s]), (uint32_t)issued_parity[s], &dummy);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- leader: MMA issuer for the pair ----------------
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int it = 0;
      for (int64_t t = pair; t < args.num_tiles && ok; t += npairs)
        for (int c = 0; c < args.nchunks && ok; ++c, ++it) {
          const int acc = it & 1;
          const uint32_t acc_phase = (uint32_t)(it >> 1) & 1u;
          if (!mbar_wait(smem_u32(&acc_empty[acc]), acc_phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * ACC_COLS);
          const int nkbc = args.chunk_kblocks(c);
          for (int kb = 0; kb < nkbc; ++kb) {
            if (!mbar_wait(smem_u32(&full[stage]), phase, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ah = smem_u32(sA + stage * 2 * A_BYTES), al = ah + A_BYTES;
            const uint32_t bh = smem_u32(sB + stage * 2 * B_BYTES), bl = bh + B_BYTES;
            // the three split products of this k-block into the same accumulator
#pragma unroll
            for (int kk = 0; kk < BK / UMMA_K; ++kk) {
              const uint32_t o = kk * UMMA_K * 2;
              umma_pair(d_tmem, smem_desc(ah + o), smem_desc(bh + o), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
              umma_pair(d_tmem, smem_desc(ah + o), smem_desc(bl + o), idesc, 1u);
              umma_pair(d_tmem, smem_desc(al + o), smem_desc(bh + o), idesc, 1u);
            }
            umma_commit_both(smem_u32(&empty[stage]));
            if (++stage == STG) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (!ok) break;
          umma_commit_both(smem_u32(&acc_full[acc]));
        }
      if (!ok) {
        if (args.d_status) atomicExch(args.d_status, SIM_TIMEOUT_CODE_MMA);
        *abort_flag = 1;
      }
      umma_commit_local(smem_u32(mma_done));
      volatile int dummy = 0;
      mbar_wait(smem_u32(mma_done), 0, &dummy);
    }
  } else {
    // ---------------- epilogue: this CTA's 128 rows ----------------
    // Warp e reads the tensor-memory lane quarter of its warp slot (warp % 4): lane
    // i of the warp holds output row row0 + i.  It covers COLS of the 256
    // accumulator columns, SW columns per step; the load of step c+1 is in flight
    // while step c is processed.  The statistics are taken from the registers.
    // Each step is staged in shared memory in the TMA swizzle layout (16-byte chunk
    // j of row r at chunk j ^ ((r >> 1) & 3) for 64-byte rows, j ^ ((r >> 2) & 1)
    // for 32-byte rows, which also keeps the 128-bit shared stores free of bank
    // conflicts) and written by one TMA store, or TMA reduce-add where the output
    // accumulates.  With NBUF staging buffers per warp, a buffer is rewritten once
    // the store issued from it NBUF steps earlier has finished reading it.
    const int e = warp - 2;
    const int q = warp & 3;
    const int cpart = e >> 2;
    float* bufs = sEpi + e * (NBUF * 32 * SW);
    const float sa = args.scale_a ? *args.scale_a : 1.f;
    const float sb = args.scale_b ? *args.scale_b : 1.f;
    const float oscale = 1.f / (sa * sb);
    const uint32_t acc_empty_leader = map_to(smem_u32(&acc_empty[0]), 0);
    constexpr int NSTEP = COLS / SW;
    const int swz = SW == 16 ? ((lane >> 1) & 3) : ((lane >> 2) & 1);
    double st_p = 0.0, st_l = 0.0, st_n = 0.0;
    int it = 0, sbuf = 0;
    bool stop = false;
    for (int64_t t = pair; t < args.num_tiles && !stop; t += npairs)
      for (int kc = 0; kc < args.nchunks; ++kc, ++it) {
        const bool rmw = args.accumulate || kc > 0;
        const bool last = kc == args.nchunks - 1;
        // final values of a read-modify-write pass are formed in registers when they
        // feed the statistics; otherwise the TMA reduce-add accumulates them in L2
        // (direct launches never read back: one chunk, no accumulation)
        const bool rmw_regs = STATS && last && rmw;
        const int acc = it & 1;
        const uint32_t acc_phase = (uint32_t)(it >> 1) & 1u;
        if (!mbar_wait(smem_u32(&acc_full[acc]), acc_phase, abort_flag)) {
          if (args.d_status) atomicExch(args.d_status, SIM_TIMEOUT_CODE_EPI);
          *abort_flag = 1;
          stop = true;
          break;
        }
        tc_fence_after();
        // an earlier chunk of this tile was written by this warp: its writes must be
        // complete before they are added to or read back (direct stores: the same
        // thread wrote them, in program order)
        if (!DIRECT && kc > 0) {
          if (lane == 0) bulk_wait_all();
          __syncwarp();
        }
        int64_t mb, nb;
        args.tm.tile(t, mb, nb);
        const int64_t row0 = mb * 2 * BM + rank * BM + q * 32;
        const int64_t col_half0 = nb * BN + cpart * COLS;
        const int64_t grow = row0 + lane;
        const bool rowok = grow < args.M;
        const uint32_t lcode = (SIGN && rowok) ? __ldg(args.out_lcode + grow) : 0u;
        const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * ACC_COLS + cpart * COLS);
        // per-job partial statistics in fp32 (at most 64 terms per lane), folded into
        // the FP64 totals once per job
        float jp = 0.f, jl = 0.f;
        int jn = 0;
        auto step = [&](const uint32_t (&r)[SW], int c) {
          float v[SW];
#pragma unroll
          for (int j = 0; j < SW; ++j) v[j] = __uint_as_float(r[j]) * oscale;
          const int64_t gcol0 = col_half0 + c * SW;
          if (SIGN && lcode) {
            // output-phase cuts: (-1)^{popc(row code & column code)} on this part
            const uint32_t* uc = args.out_ucode + (gcol0 >> 1);
#pragma unroll
            for (int j = 0; j < SW / 2; ++j) {
              const uint32_t u = (gcol0 + 2 * j < args.N2) ? __ldg(uc + j) : 0u;
              if (__popc(lcode & u) & 1) {
                v[2 * j] = -v[2 * j];
                v[2 * j + 1] = -v[2 * j + 1];
              }
            }
          }
          if (rmw_regs && rowok) {
            const float* src = args.C + grow * args.N2 + gcol0;
#pragma unroll
            for (int j = 0; j < SW / 4; ++j)
              if (gcol0 + 4 * j + 4 <= args.N2) {
                const float4 old = __ldcg((const float4*)(src + 4 * j));
                v[4 * j] += old.x;
                v[4 * j + 1] += old.y;
                v[4 * j + 2] += old.z;
                v[4 * j + 3] += old.w;
              }
          }
          if (STATS && last) {
#pragma unroll
            for (int j = 0; j < SW / 2; ++j) {
              const float re = v[2 * j], im = v[2 * j + 1];
              const float pp = fmaf(re, re, im * im);
              const float w = pp * args.w_scale;
              const bool okv = rowok && (gcol0 + 2 * j < args.N2);
              const bool pos = okv && (w > 0.f);
              jp += okv ? pp : 0.f;
              jl += pos ? __log2f(w) : 0.f;  // log2; scaled by ln 2 once per job
              jn += pos ? 1 : 0;
              // bin of u = 1 - exp(-w): floor(B - B exp(-w)), the floor taken by a
              // round-down add against 2^23 (exact for 0 <= x < 2^23)
              const float x = fmaf(-(float)SIM_KS_BINS, __expf(-w), (float)SIM_KS_BINS);
              const int bin = __float_as_int(__fadd_rd(x, 8388608.f)) - 0x4B000000;
              if (okv) atomicAdd(&s_hist[min(max(bin, 0), SIM_KS_BINS - 1)], 1u);
            }
          }
          if constexpr (DIRECT) {
            // each lane writes its row's SW floats as SW / 8 full 32-byte sectors
            // (256-bit stores): the sectors a TMA box store writes, without the
            // shared-memory staging
            if (rowok) {
              float* dst = args.C + grow * args.N2 + gcol0;
#pragma unroll
              for (int j = 0; j < SW / 8; ++j)
                if (gcol0 + 8 * j < args.N2)
                  asm volatile("st.global.L1::no_allocate.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(
                                   dst + 8 * j),
                               "f"(v[8 * j]), "f"(v[8 * j + 1]), "f"(v[8 * j + 2]), "f"(v[8 * j + 3]), "f"(v[8 * j + 4]),
                               "f"(v[8 * j + 5]), "f"(v[8 * j + 6]), "f"(v[8 * j + 7])
                               : "memory");
            }
            return;
          }
          float* buf = bufs + sbuf * (32 * SW);
          if (lane == 0) {
            if (NBUF == 2)
              bulk_wait_read1();
            else
              bulk_wait_read0();
          }
          __syncwarp();
#pragma unroll
          for (int j = 0; j < SW / 4; ++j)
            *(float4*)(buf + lane * SW + ((j ^ swz) * 4)) = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            if (row0 < args.M && gcol0 < args.N2) {
              if (rmw && !rmw_regs)
                tma_reduce_add_2d(&mapC, smem_u32(buf), (int)gcol0, (int)row0);
              else
                tma_store_2d(&mapC, smem_u32(buf), (int)gcol0, (int)row0);
            }
            bulk_commit();
          }
          if (NBUF == 2) sbuf ^= 1;
        };
        uint32_t ra[SW], rb[SW];
        tmem_ld_async<SW>(tbase, ra);
#pragma unroll UNR
        for (int c = 0; c < NSTEP; c += 2) {
          tmem_wait<SW>(ra);
          tmem_ld_async<SW>(tbase + (uint32_t)((c + 1) * SW), rb);
          step(ra, c);
          tmem_wait<SW>(rb);
          if (c + 2 < NSTEP) {
            tmem_ld_async<SW>(tbase + (uint32_t)((c + 2) * SW), ra);
          } else {
            // every accumulator column of this job is in registers: release it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc_empty_leader + (uint32_t)(acc * sizeof(uint64_t)));
          }
          step(rb, c + 1);
        }
        if (STATS && last) {
          st_p += (double)jp;
          st_l += (double)jl * 0.69314718055994530942;
          st_n += (double)jn;
        }
      }
    // all output writes of this warp complete (and its staging buffers free) before exit
    if (!DIRECT) {
      if (lane == 0) bulk_wait_all();
      __syncwarp();
    }
    if (STATS) {
      for (int o = 16; o > 0; o >>= 1) {
        st_p += __shfl_xor_sync(0xffffffffu, st_p, o);
        st_l += __shfl_xor_sync(0xffffffffu, st_l, o);
        st_n += __shfl_xor_sync(0xffffffffu, st_n, o);
      }
      if (lane == 0) {
        atomicAdd(&args.st_acc[0], st_p);
        atomicAdd(&args.st_acc[1], st_l);
        atomicAdd(&args.st_acc[2], st_n);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (STATS)
    for (int i = threadIdx.x; i < SIM_KS_BINS; i += THREADS)
      if (s_hist[i]) atomicAdd(&args.st_hist[i], (unsigned long long)s_hist[i]);
  // the leader's MMAs read this CTA's shared memory and write its tensor memory:
  // neither CTA releases them before both are done
  cluster_sync();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn2() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// operand map: rows x kpad 16-bit values, SW128 boxes of 64 x box_rows
bool make_operand_map(CUtensorMap* map, const void* base, int64_t rows, int64_t kpad, int box_rows, bool fp16) {
  auto enc = get_encode_fn2();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(kpad * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// output map: M rows x N2 floats, boxes of 32 rows x sw floats in the 64-byte
// (sw = 16) or 32-byte (sw = 8) swizzle
bool make_output_map(CUtensorMap* map, float* C, int64_t M, int64_t N2, int sw) {
  auto enc = get_encode_fn2();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)N2, (cuuint64_t)M};
  cuuint64_t strides[1] = {(cuuint64_t)(N2 * 4)};
  cuuint32_t box[2] = {(cuuint32_t)sw, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   sw == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <bool STATS, bool SIGN, int STG, int SW, int NBUF, int UNR, int EW, bool DIRECT>
cudaError_t launch_variant(const CUtensorMap (&maps)[4], const CUtensorMap& mapC, const PairArgs& k, uint32_t idesc,
                           int num_sms, cudaStream_t s) {
  constexpr int SMEM = PairSmem<STG, SW, NBUF, EW, DIRECT>::BYTES;
  constexpr int THREADS = 32 * (2 + EW);
  static DeviceOnce setup;
  int max_pairs = 0;
  cudaError_t e = setup.run(
      [&](int& n) {
        cudaError_t r = cudaFuncSetAttribute(tc_gemm_pair_kernel<STATS, SIGN, STG, SW, NBUF, UNR, EW, DIRECT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (r != cudaSuccess) return r;
        // one resident pair per SM pair: as many clusters as can be co-scheduled at once
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (unsigned)(num_sms / 2), 1, 1);
        cfg.blockDim = dim3(THREADS, 1, 1);
        cfg.dynamicSmemBytes = SMEM;
        n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_gemm_pair_kernel<STATS, SIGN, STG, SW, NBUF, UNR, EW, DIRECT>, &cfg) !=
                cudaSuccess ||
            n < 1) {
          cudaGetLastError();
          n = num_sms / 2;
        }
        return cudaSuccess;
      },
      &max_pairs);
  if (e != cudaSuccess) return e;
  int pairs = max_pairs;
  if ((int64_t)pairs > k.num_tiles) pairs = (int)k.num_tiles;
  if (pairs < 1) pairs = 1;
  tc_gemm_pair_kernel<STATS, SIGN, STG, SW, NBUF, UNR, EW, DIRECT><<<2 * pairs, THREADS, SMEM, s>>>(maps[0], maps[1], maps[2], maps[3], mapC, k,
                                                                      idesc);
  return cudaGetLastError();
}

}  // namespace

// The CTA-pair kernel is the default; SIM_TC_PAIR=0 in the environment selects the
// single-CTA kernel of gemm_tc.cu instead (for comparisons).
bool tc_gemm_pair_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("SIM_TC_PAIR");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on == 1;
}

cudaError_t launch_wait_selftest(int* d_status, unsigned long long limit_ns, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(d_status, limit_ns);
  return cudaGetLastError();
}

bool tc_gemm_pair_supported(const TcGemmArgs& a) {
  // the output is written by TMA: 16-byte aligned base and row pitch
  return (((uintptr_t)a.C) & 15u) == 0 && (a.N2 % 4) == 0;
}

cudaError_t launch_tc_gemm_pair(const TcGemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N2 <= 0) return cudaSuccess;
  if (a.kpad <= 0 || a.kpad % BK != 0 || a.M > (1ll << 31) - 2 * BM || a.N2 > (1ll << 31) - BN)
    return cudaErrorInvalidValue;
  if (((uintptr_t)a.a_hi | (uintptr_t)a.a_lo | (uintptr_t)a.b_hi | (uintptr_t)a.b_lo) & 15u)
    return cudaErrorInvalidValue;
  if (!tc_gemm_pair_supported(a)) return cudaErrorInvalidValue;
  const int sw = 16;
  CUtensorMap maps[4], mapC;
  if (!make_operand_map(&maps[0], a.a_hi, a.M, a.kpad, BM, a.fp16) ||
      !make_operand_map(&maps[1], a.a_lo, a.M, a.kpad, BM, a.fp16) ||
      !make_operand_map(&maps[2], a.b_hi, a.N2, a.kpad, BNH, a.fp16) ||
      !make_operand_map(&maps[3], a.b_lo, a.N2, a.kpad, BNH, a.fp16) ||
      !make_output_map(&mapC, (float*)a.C, a.M, a.N2, sw))
    return cudaErrorInvalidValue;
  PairArgs k;
  k.M = a.M;
  k.N2 = a.N2;
  k.nkb = (int)(a.kpad / BK);
  k.ckb = kChunkCopies * 2 / BK;
  k.nchunks = (k.nkb + k.ckb - 1) / k.ckb;
  k.tm.num_mb = (a.M + 2 * BM - 1) / (2 * BM);
  k.tm.num_nb = (a.N2 + BN - 1) / BN;
  // 32 pair tiles (8192 rows of A, 16 MB of split operands) per raster group stay in
  // L2 while the group sweeps B, which is then read from DRAM once per group
  k.tm.group = a.group_m > 0 ? a.group_m : 32;
  k.num_tiles = k.tm.num_mb * k.tm.num_nb;
  k.scale_a = a.scale_a;
  k.scale_b = a.scale_b;
  k.accumulate = a.accumulate;
  k.C = (float*)a.C;
  k.d_status = a.d_status;
  k.w_scale = a.w_scale;
  k.st_acc = a.st_acc;
  k.st_hist = a.st_hist;
  k.out_lcode = (a.out_lcode && a.out_ucode) ? a.out_lcode : nullptr;
  k.out_ucode = k.out_lcode ? a.out_ucode : nullptr;
  const uint32_t idesc = instr_desc_pair(a.fp16 != 0);
  const int nsm = a.num_sms > 0 ? a.num_sms : 148;
  const bool stats = a.st_acc && a.st_hist;
  // 16-column epilogue steps, one staging buffer per epilogue warp, two steps per
  // loop iteration
  const bool sign = k.out_lcode != nullptr;
  // Epilogue shape by the length of a tile's main loop: with few k-blocks per tile
  // (K <= 128 copies) the epilogue is the bound and 16 epilogue warps hide its
  // latency (2 operand stages of 64 KB); longer main loops are set below.
  // Direct epilogue stores (each lane writes full 32-byte sectors of its row from
  // registers, no shared-memory staging) when the contraction writes each output
  // once: one copy chunk and no accumulation, 32-byte aligned rows.  Measured on the
  // 2^30-amplitude workload (K = 256): 3.86 ms against 4.22 ms with TMA box stores
  // from staging, whose shared-memory traffic competed with the operand stages.
  // Contractions that add chunks into the output keep the staging path, whose TMA
  // reduce-adds accumulate in L2 (the 42-qubit contraction, 64 chunks: 72 ms against
  // 115 ms when every chunk reads the block back through the SMs).
  // SIM_EPI_DIRECT=0 selects the staging path everywhere, for comparisons.
  static const bool direct_ok = [] {
    const char* e = getenv("SIM_EPI_DIRECT");
    return !(e && e[0] == '0');
  }();
  const bool direct = direct_ok && k.nchunks == 1 && !a.accumulate && ((((uintptr_t)a.C) & 31u) == 0) &&
                      (a.N2 % 8) == 0;
#define LV2(G, E, D)                                                                                     \
  (stats ? (sign ? launch_variant<true, true, G, 16, 1, 2, E, D>(maps, mapC, k, idesc, nsm, s)             \
                 : launch_variant<true, false, G, 16, 1, 2, E, D>(maps, mapC, k, idesc, nsm, s))           \
         : (sign ? launch_variant<false, true, G, 16, 1, 2, E, D>(maps, mapC, k, idesc, nsm, s)            \
                 : launch_variant<false, false, G, 16, 1, 2, E, D>(maps, mapC, k, idesc, nsm, s)))
#define LV(G, E) (direct ? LV2(G, E, true) : LV2(G, E, false))
  // Longer main loops: 3 stages; 8 epilogue warps, or 16 when the statistics are
  // fused into a direct epilogue (no staging buffers, 214,528 bytes of shared
  // memory).  2^30 amplitudes, K = 256: with statistics 3.25 ms on 16 warps against
  // 3.74 ms on 8; without them 3.02 ms on 8 against 3.26 ms on 16 (the extra warps
  // take issue slots from the producer and MMA warps).
  cudaError_t e = k.nkb <= 4             ? LV(2, 16)
                  : (direct && stats) ? LV2(3, 16, true)
                                      : LV(3, 8);
#undef LV
#undef LV2
  note_launches(SIM_PHASE_CONTRACT, 1);
  return e;
}

}  // namespace sim
