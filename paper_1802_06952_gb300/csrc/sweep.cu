// Gate-sweep kernels of the half-circuit state-vector evolution
// (Supplementary A, Eqs. 4-5 per half; diagonal gates of a layer combined into one
// per-amplitude phase and mask, Section 2.4, Eqs. 3-6).
//
//   sweep_c64_kernel   fused pass over complex64 states: each block stages 2^k
//                      amplitudes (its local qubits, always including the low five
//                      bits so global rows are coalesced) in shared memory, applies
//                      every gate and diagonal op of the pass, and writes back.  One
//                      launch covers all nodes of a copy-tree level (or a chunk).
//   plain_*            the plain complex128 path: one pass per non-diagonal gate and
//                      one combined diagonal pass per layer, every copy on its own.
//   gather_kernel      picks the selected entries of leaf states.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace sim {
namespace {

// w^e for w = e^{i pi / 4}, e = 0..7 (exact constants 0, +-1, +-1/sqrt2)
__constant__ float2 kOmegaF[8] = {
    {1.f, 0.f}, {0.70710678118654752f, 0.70710678118654752f}, {0.f, 1.f},
    {-0.70710678118654752f, 0.70710678118654752f}, {-1.f, 0.f},
    {-0.70710678118654752f, -0.70710678118654752f}, {0.f, -1.f},
    {0.70710678118654752f, -0.70710678118654752f}};
__constant__ double2 kOmegaD[8] = {
    {1.0, 0.0}, {0.70710678118654752440, 0.70710678118654752440}, {0.0, 1.0},
    {-0.70710678118654752440, 0.70710678118654752440}, {-1.0, 0.0},
    {-0.70710678118654752440, -0.70710678118654752440}, {0.0, -1.0},
    {0.70710678118654752440, -0.70710678118654752440}};

struct DiagState {
  uint32_t tmask, pmask, pval, zmask, w1mask, w2mask;
  int nsh;
  uint32_t sh_d[kMaxShift], sh_m[kMaxShift];
};

// Resolve a DIAG op for one copy-tree node: the cut slots become a projector
// (P_l slots: bits cutq must equal the copy bits cutm) and, for the phase slots
// whose copy bit is 1, masks of the qubits whose weight has bit 1, 2 or 4 set
// (Z^l: weight 4; T^l: 1; S^l: 2).
__device__ __forceinline__ void load_diag(const OpRec* op, uint64_t node_id, DiagState& d) {
  d.tmask = __ldg(&op->tmask);
  d.nsh = __ldg(&op->nsh);
  for (int s = 0; s < kMaxShift; ++s) {
    d.sh_d[s] = __ldg(&op->sh_d[s]);
    d.sh_m[s] = __ldg(&op->sh_m[s]);
  }
  const int ncut = __ldg(&op->ncut);
  const uint32_t cutz = __ldg(&op->cutz);
  d.pmask = d.pval = d.zmask = d.w1mask = d.w2mask = 0;
  for (int i = 0; i < ncut; ++i) {
    const uint32_t qb = 1u << op->cutq[i];
    const uint32_t l = (uint32_t)((node_id >> op->cutm[i]) & 1ull);
    if (!((cutz >> i) & 1u)) {
      d.pmask |= qb;
      if (l) d.pval |= qb;
    } else if (l) {
      const uint32_t w = op->cutw[i];
      if (w & 4u) d.zmask |= qb;
      if (w & 2u) d.w2mask |= qb;
      if (w & 1u) d.w1mask |= qb;
    }
  }
}

// exponent of w (mod 8) and the projector test for index x
__device__ __forceinline__ int diag_exp(const DiagState& d, uint32_t x, bool& keep) {
  int e = __popc(x & d.tmask) + __popc(x & d.w1mask) + 2 * __popc(x & d.w2mask);
  int s2 = __popc(x & d.zmask);
#pragma unroll
  for (int s = 0; s < kMaxShift; ++s)
    if (s < d.nsh) s2 += __popc(x & (x >> d.sh_d[s]) & d.sh_m[s]);
  keep = (x & d.pmask) == d.pval;
  return (e + 4 * s2) & 7;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct SweepArgs {
  int n, k, low;
  uint32_t local_mask;
  const OpRec* ops;
  int op_count;
  int src;
  const NodeEntry* nodes;
  int64_t slot_begin;
  const float2* src_base;
  float2* dst_base;
  uint8_t hi_pos[32];     // positions of local qubits above the low bits
  uint8_t nonlocal[32];   // positions of non-local qubits
  float init_val;
};

__global__ void __launch_bounds__(256) sweep_c64_kernel(SweepArgs a) {
  extern __shared__ float2 sm[];
  __shared__ uint32_t hi_off[256];
  __shared__ uint32_t hi_off2[32];
  const int n = a.n, k = a.k, low = a.low;
  const uint32_t nb_log = (uint32_t)(n - k);
  const uint64_t bid = blockIdx.x;
  const int64_t slot = a.slot_begin + (int64_t)(bid >> nb_log);
  const uint32_t g = (uint32_t)(bid & ((1ull << nb_log) - 1));
  const NodeEntry ne = a.nodes[slot];
  const uint64_t stride = 1ull << n;
  float2* dst = a.dst_base + (uint64_t)ne.dst_row * stride;
  const float2* src = a.src == SRC_PARENT ? a.src_base + (uint64_t)ne.parent_slot * stride
                                          : (const float2*)dst;
  // global index of local element i: base | (i & lowmask) | (hi_off[(i >> low) & 255] | hi_off2[i >> (low + 8)])
  uint32_t base = 0;
  for (uint32_t i = 0; i < nb_log; ++i)
    if ((g >> i) & 1u) base |= 1u << a.nonlocal[i];
  // offsets of the local ranks above the identity prefix: ranks low..low+7 by
  // hi_off, ranks low+8.. by hi_off2
  const int nhi = k - low;
  const int n1 = nhi < 8 ? nhi : 8;
  for (int t = threadIdx.x; t < (1 << n1); t += blockDim.x) {
    uint32_t off = 0;
    for (int i = 0; i < n1; ++i)
      if ((t >> i) & 1) off |= 1u << a.hi_pos[i];
    hi_off[t] = off;
  }
  for (int t = threadIdx.x; t < (1 << (nhi - n1)); t += blockDim.x) {
    uint32_t off = 0;
    for (int i = 0; i < nhi - n1; ++i)
      if ((t >> i) & 1) off |= 1u << a.hi_pos[8 + i];
    hi_off2[t] = off;
  }
  __syncthreads();
  const uint32_t lowmask = (1u << low) - 1;
  const int size = 1 << k;
  for (int i = threadIdx.x; i < size; i += blockDim.x) {
    const uint32_t x = base | (i & lowmask) | (hi_off[(i >> low) & 255] | hi_off2[i >> (low + 8)]);
    float2 v;
    if (a.src == SRC_UNIFORM)
      v = make_float2(a.init_val, 0.f);
    else if (a.src == SRC_ZERO)
      v = make_float2(x == 0 ? 1.f : 0.f, 0.f);
    else
      v = src[x];
    sm[i] = v;
  }
  __syncthreads();
  for (int o = 0; o < a.op_count; ++o) {
    const OpRec* op = a.ops + o;
    const int type = __ldg(&op->type);
    if (type == OP_SWAP) continue;  // layout exchanges of the register-blocked sweep
    if (type == OP_GATE) {
      // an X^l slot of a cut controlled X: only in the copies with l_m = 1
      const int cond = __ldg(&op->cond);
      if (cond >= 0 && !((ne.node_id >> cond) & 1ull)) continue;
      const int lq = __ldg(&op->lq0);
      const float2 m00 = make_float2(__ldg(&op->m[0]), __ldg(&op->m[1]));
      const float2 m01 = make_float2(__ldg(&op->m[2]), __ldg(&op->m[3]));
      const float2 m10 = make_float2(__ldg(&op->m[4]), __ldg(&op->m[5]));
      const float2 m11 = make_float2(__ldg(&op->m[6]), __ldg(&op->m[7]));
      const int lo_mask = (1 << lq) - 1;
      for (int p = threadIdx.x; p < (size >> 1); p += blockDim.x) {
        const int i0 = ((p & ~lo_mask) << 1) | (p & lo_mask);
        const int i1 = i0 | (1 << lq);
        const float2 a0 = sm[i0], a1 = sm[i1];
        float2 r0 = cmul(m00, a0), r1 = cmul(m10, a0);
        const float2 t0 = cmul(m01, a1), t1 = cmul(m11, a1);
        r0.x += t0.x; r0.y += t0.y;
        r1.x += t1.x; r1.y += t1.y;
        sm[i0] = r0;
        sm[i1] = r1;
      }
    } else {
      DiagState d;
      load_diag(op, ne.node_id, d);
      for (int i = threadIdx.x; i < size; i += blockDim.x) {
        const uint32_t x = base | (i & lowmask) | (hi_off[(i >> low) & 255] | hi_off2[i >> (low + 8)]);
        bool keep;
        const int e = diag_exp(d, x, keep);
        sm[i] = keep ? cmul(sm[i], kOmegaF[e]) : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < size; i += blockDim.x) {
    const uint32_t x = base | (i & lowmask) | (hi_off[(i >> low) & 255] | hi_off2[i >> (low + 8)]);
    dst[x] = sm[i];
  }
}

// ---------------------------------------------------------------------------
// Plain complex128 path (one pass per gate, Section 2.4 diagonal pass per layer)
// ---------------------------------------------------------------------------
__global__ void plain_init_zero_kernel(double2* psi, int n, uint64_t total) {
  const uint64_t mask = (1ull << n) - 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x)
    psi[i] = make_double2((i & mask) == 0 ? 1.0 : 0.0, 0.0);
}

__global__ void plain_gate_kernel(double2* psi, int n, int q, const OpRec* op, const uint64_t* copy_ids,
                                  uint64_t npairs_total) {
  const int cond = op->cond;  // X^l slot of a cut controlled X: copies with l_m = 1 only
  const double2 m00 = make_double2(op->md[0], op->md[1]);
  const double2 m01 = make_double2(op->md[2], op->md[3]);
  const double2 m10 = make_double2(op->md[4], op->md[5]);
  const double2 m11 = make_double2(op->md[6], op->md[7]);
  const uint64_t half = 1ull << (n - 1);
  const uint64_t lo_mask = (1ull << q) - 1;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < npairs_total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = t / half, p = t % half;
    if (cond >= 0 && !((copy_ids[s] >> cond) & 1ull)) continue;
    double2* v = psi + (s << n);
    const uint64_t i0 = ((p & ~lo_mask) << 1) | (p & lo_mask);
    const uint64_t i1 = i0 | (1ull << q);
    const double2 a0 = v[i0], a1 = v[i1];
    double2 r0 = cmul(m00, a0), r1 = cmul(m10, a0);
    const double2 t0 = cmul(m01, a1), t1 = cmul(m11, a1);
    r0.x += t0.x; r0.y += t0.y;
    r1.x += t1.x; r1.y += t1.y;
    v[i0] = r0;
    v[i1] = r1;
  }
}

__global__ void plain_diag_kernel(double2* psi, int n, const OpRec* op, const uint64_t* copy_ids,
                                  uint64_t total) {
  const uint64_t mask = (1ull << n) - 1;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = t >> n;
    const uint32_t x = (uint32_t)(t & mask);
    DiagState d;
    load_diag(op, copy_ids[s], d);
    bool keep;
    const int e = diag_exp(d, x, keep);
    psi[t] = keep ? cmul(psi[t], kOmegaD[e]) : make_double2(0.0, 0.0);
  }
}

template <typename T>
__global__ void gather_kernel(const T* src, int n, const NodeEntry* nodes, int64_t nslots,
                              const uint64_t* sel, int64_t nsel, T* dst) {
  const uint64_t total = (uint64_t)nslots * (uint64_t)nsel;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = t / (uint64_t)nsel, i = t % (uint64_t)nsel;
    const NodeEntry ne = nodes[s];
    dst[(uint64_t)ne.dst_row * nsel + i] = src[(s << n) + sel[i]];
  }
}

// Selected entries of leaf states computed from their parent states, without the
// leaf states (Section 2.3.1's sampling needs only the selected entries).  The
// ops of the leaf level act non-diagonally on the qubits Q alone (|Q| = nq), so
// for a selected index x, with x_o its bits outside Q,
//   leaf(x) = sum over y of <x| G |x_o + y> parent(x_o + y),  y over the 2^nq
// settings of the Q bits: one warp loads those 2^nq parent entries into a small
// vector (local bit b = qubit qpos[b]), applies the level's ops to it in order
// (full gate matrices as in sweep_c64_kernel; diagonal terms evaluated at the full
// index x_o + y), and keeps the entry at x's Q bits.
struct SparseLeafArgs {
  int n, nq;
  uint32_t qmask;
  uint8_t qpos[kMaxSparseQ];
  uint8_t qrank[32];          // local bit of each qubit of Q
  const OpRec* ops;
  int op_count;
  const NodeEntry* nodes;     // leaf nodes: node_id, parent_slot, dst_row = leaf row
  int64_t nslots;
  const float2* parent_base;  // parent level buffer (slot stride 2^n)
  const uint64_t* sel;
  int64_t nsel;
  float2* leafsel;            // [row][nsel]
};

constexpr int kSparseWarps = 8;

__global__ void __launch_bounds__(32 * kSparseWarps) sparse_leaf_kernel(SparseLeafArgs a) {
  extern __shared__ float2 sv_all[];  // kSparseWarps vectors of 2^nq, then the offsets
  const int size = 1 << a.nq;
  uint32_t* scat = (uint32_t*)(sv_all + kSparseWarps * size);  // index bits of each local y
  for (int e = threadIdx.x; e < size; e += blockDim.x) {
    uint32_t off = 0;
    for (int b = 0; b < a.nq; ++b)
      if ((e >> b) & 1) off |= 1u << a.qpos[b];
    scat[e] = off;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* v = sv_all + w * size;
  const uint64_t total = (uint64_t)a.nslots * (uint64_t)a.nsel;
  for (uint64_t item = (uint64_t)blockIdx.x * kSparseWarps + w; item < total;
       item += (uint64_t)gridDim.x * kSparseWarps) {
    const uint64_t s = item / (uint64_t)a.nsel, i = item % (uint64_t)a.nsel;
    const NodeEntry ne = a.nodes[s];
    const uint32_t x = (uint32_t)a.sel[i];
    const uint32_t xo = x & ~a.qmask;
    const float2* par = a.parent_base + ((uint64_t)ne.parent_slot << a.n);
    for (int e = lane; e < size; e += 32) v[e] = par[xo | scat[e]];
    __syncwarp();
    for (int o = 0; o < a.op_count; ++o) {
      const OpRec* op = a.ops + o;
      const int type = __ldg(&op->type);
      if (type == OP_SWAP) continue;  // layout exchanges of the register-blocked sweep
      if (type == OP_GATE) {
        const int cond = __ldg(&op->cond);
        if (cond >= 0 && !((ne.node_id >> cond) & 1ull)) continue;
        const int lq = a.qrank[__ldg(&op->q)];
        const float2 m00 = make_float2(__ldg(&op->m[0]), __ldg(&op->m[1]));
        const float2 m01 = make_float2(__ldg(&op->m[2]), __ldg(&op->m[3]));
        const float2 m10 = make_float2(__ldg(&op->m[4]), __ldg(&op->m[5]));
        const float2 m11 = make_float2(__ldg(&op->m[6]), __ldg(&op->m[7]));
        const int lo_mask = (1 << lq) - 1;
        for (int p = lane; p < (size >> 1); p += 32) {
          const int i0 = ((p & ~lo_mask) << 1) | (p & lo_mask);
          const int i1 = i0 | (1 << lq);
          const float2 a0 = v[i0], a1 = v[i1];
          float2 r0 = cmul(m00, a0), r1 = cmul(m10, a0);
          const float2 t0 = cmul(m01, a1), t1 = cmul(m11, a1);
          r0.x += t0.x; r0.y += t0.y;
          r1.x += t1.x; r1.y += t1.y;
          v[i0] = r0;
          v[i1] = r1;
        }
      } else {
        DiagState d;
        load_diag(op, ne.node_id, d);
        for (int e = lane; e < size; e += 32) {
          bool keep;
          const int ex = diag_exp(d, xo | scat[e], keep);
          v[e] = keep ? cmul(v[e], kOmegaF[ex]) : make_float2(0.f, 0.f);
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      uint32_t ex = 0;
      for (int b = 0; b < a.nq; ++b)
        if ((x >> a.qpos[b]) & 1u) ex |= 1u << b;
      a.leafsel[(uint64_t)ne.dst_row * (uint64_t)a.nsel + i] = v[ex];
    }
    __syncwarp();
  }
}

unsigned grid_for(uint64_t work, int threads) {
  uint64_t b = (work + threads - 1) / threads;
  if (b > (1u << 20)) b = 1u << 20;
  return (unsigned)(b ? b : 1);
}

}  // namespace

cudaError_t launch_sweep_c64(const SweepLaunch& L, cudaStream_t s) {
  SweepArgs a;
  memset(&a, 0, sizeof a);
  a.n = L.n;
  a.k = L.k;
  // the leading ranks that hold qubits 0, 1, ... in order index global memory
  // directly (coalesced); any rank order is accepted
  a.low = 0;
  while (a.low < 5 && a.low < L.k && L.order[a.low] == a.low) ++a.low;
  a.local_mask = L.local_mask;
  a.ops = L.ops;
  a.op_count = L.op_count;
  a.src = L.src;
  a.nodes = L.nodes;
  a.src_base = (const float2*)L.src_base;
  a.dst_base = (float2*)L.dst_base;
  int nh = 0, nn = 0;
  for (int r = 0; r < L.k; ++r) {
    const int q = L.order[r];
    if (q >= L.n || !(L.local_mask & (1u << q))) return cudaErrorInvalidValue;
    if (r >= a.low) a.hi_pos[nh++] = (uint8_t)q;
  }
  for (int q = 0; q < L.n; ++q)
    if (!(L.local_mask & (1u << q))) a.nonlocal[nn++] = (uint8_t)q;
  if (nh != L.k - a.low || nn != L.n - L.k) return cudaErrorInvalidValue;
  // 2^{-n/2}
  a.init_val = (float)ldexp(1.0, -(L.n / 2)) * ((L.n & 1) ? 0.70710678118654752f : 1.f);
  const int threads = L.threads > 0 ? L.threads : 256;
  const size_t smem = sizeof(float2) << L.k;
  static DeviceOnce attr;
  {
    cudaError_t e = attr.run([](int&) {
      return cudaFuncSetAttribute(sweep_c64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float2) << 13));
    });
    if (e != cudaSuccess) return e;
  }
  const uint64_t bps = 1ull << (L.n - L.k);
  // keep each launch below 2^30 blocks
  const int64_t max_slots = (int64_t)((1ull << 30) / bps) > 0 ? (int64_t)((1ull << 30) / bps) : 1;
  for (int64_t s0 = 0; s0 < L.nslots; s0 += max_slots) {
    const int64_t ns = (L.nslots - s0) < max_slots ? (L.nslots - s0) : max_slots;
    a.slot_begin = s0;
    sweep_c64_kernel<<<(unsigned)(ns * bps), threads, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launches(SIM_PHASE_SWEEP, 1);
  }
  return cudaSuccess;
}

cudaError_t launch_plain_init_zero(void* psi, int n, int64_t nstates, cudaStream_t s) {
  const uint64_t total = (uint64_t)nstates << n;
  plain_init_zero_kernel<<<grid_for(total, 256), 256, 0, s>>>((double2*)psi, n, total);
  note_launches(SIM_PHASE_PLAIN, 1);
  return cudaGetLastError();
}

cudaError_t launch_plain_gate(const PlainLaunch& L, cudaStream_t s) {
  const uint64_t total = (uint64_t)L.nstates << (L.n - 1);
  plain_gate_kernel<<<grid_for(total, 256), 256, 0, s>>>((double2*)L.psi, L.n, L.q, L.op, L.copy_ids, total);
  note_launches(SIM_PHASE_PLAIN, 1);
  return cudaGetLastError();
}

cudaError_t launch_plain_diag(const PlainLaunch& L, cudaStream_t s) {
  const uint64_t total = (uint64_t)L.nstates << L.n;
  plain_diag_kernel<<<grid_for(total, 256), 256, 0, s>>>((double2*)L.psi, L.n, L.op, L.copy_ids, total);
  note_launches(SIM_PHASE_PLAIN, 1);
  return cudaGetLastError();
}

cudaError_t launch_gather(const void* src, int n, const NodeEntry* nodes, int64_t nslots,
                          const uint64_t* sel, int64_t nsel, void* dst, int is_c128,
                          cudaStream_t s) {
  const uint64_t total = (uint64_t)nslots * (uint64_t)nsel;
  if (total == 0) return cudaSuccess;
  if (is_c128)
    gather_kernel<double2><<<grid_for(total, 256), 256, 0, s>>>((const double2*)src, n, nodes, nslots,
                                                                  sel, nsel, (double2*)dst);
  else
    gather_kernel<float2><<<grid_for(total, 256), 256, 0, s>>>((const float2*)src, n, nodes, nslots,
                                                                sel, nsel, (float2*)dst);
  note_launches(SIM_PHASE_GATHER, 1);
  return cudaGetLastError();
}


cudaError_t launch_sparse_leaf(const SparseLeafLaunch& L, cudaStream_t s) {
  if (L.nq < 0 || L.nq > kMaxSparseQ || L.n < 1 || L.n > 32) return cudaErrorInvalidValue;
  const uint64_t total = (uint64_t)L.nslots * (uint64_t)L.nsel;
  if (total == 0) return cudaSuccess;
  SparseLeafArgs a;
  memset(&a, 0, sizeof a);
  a.n = L.n;
  a.nq = L.nq;
  a.qmask = 0;
  for (int b = 0; b < L.nq; ++b) {
    if (L.qpos[b] >= L.n || (a.qmask >> L.qpos[b]) & 1u) return cudaErrorInvalidValue;
    a.qpos[b] = L.qpos[b];
    a.qrank[L.qpos[b]] = (uint8_t)b;
    a.qmask |= 1u << L.qpos[b];
  }
  a.ops = L.ops;
  a.op_count = L.op_count;
  a.nodes = L.nodes;
  a.nslots = L.nslots;
  a.parent_base = (const float2*)L.parent_base;
  a.sel = L.sel;
  a.nsel = L.nsel;
  a.leafsel = (float2*)L.leafsel;
  const size_t smem = ((size_t)kSparseWarps * sizeof(float2) + sizeof(uint32_t)) << L.nq;
  static DeviceOnce attr;
  cudaError_t e = attr.run([](int&) {
    return cudaFuncSetAttribute(sparse_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(((size_t)kSparseWarps * sizeof(float2) + sizeof(uint32_t)) << kMaxSparseQ));
  });
  if (e != cudaSuccess) return e;
  const uint64_t blocks = (total + kSparseWarps - 1) / kSparseWarps;
  sparse_leaf_kernel<<<(unsigned)(blocks < (1u << 20) ? blocks : (1u << 20)), 32 * kSparseWarps, smem, s>>>(a);
  note_launches(SIM_PHASE_GATHER, 1);
  return cudaGetLastError();
}

}  // namespace sim
