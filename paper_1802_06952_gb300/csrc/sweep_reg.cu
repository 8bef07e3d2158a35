// Register-blocked fused gate sweep over complex64 half-states (Supplementary A,
// Eq. 4 gate by gate; the diagonal gates of a layer combined into one phase and
// mask per amplitude, Section 2.4, Eqs. 3-6).
//
// A block of 256 threads handles the 2^k amplitudes (k = 8 + R) of one assignment
// of the pass's non-local qubits.  Two bit orders of the staged index are used:
//   storage order  ranks 0..4 = qubits 0..4 (the warp lanes), so every warp loads
//                  and stores 256 contiguous bytes of the state
//   compute order  ranks 0..4 (lanes), 8..k-1 (the R register bits of each thread)
//                  hold the pass's busiest gate qubits, ranks 5..7 (warps) the rest
// When the two differ, the block transposes once after the load and once before
// the store through shared memory, in a layout whose low 4 slot bits are XORed
// with a per-pass mask of the high bits so that both orders are bank-conflict free.
// For k >= 10 the planner instead puts qubits 0 and 1 on register bits 0 and 1
// (vec4): each thread's elements then form runs of 4 consecutive amplitudes, one
// 32-byte sector each, loaded and stored with 256-bit accesses, which keeps every
// access sector-coalesced for any choice of lane qubits; the compute order is the
// load order and no transpose is needed.
// In compute order each thread keeps its 2^R amplitudes in registers:
//   gate on a register rank  register pairs, no data exchange
//   gate on a lane rank      partner value by warp shuffle
//   gate on a warp rank      partner value through shared memory (two barriers)
//   diagonal op              per amplitude phase w^e and projector test
// X^1/2 = (1+i)/2 [[1, -i], [-i, 1]], Y^1/2 = (1+i)/2 [[1, -1], [1, 1]] and
// H = 1/sqrt2 [[1, 1], [1, -1]] are applied without their scalar factors (additions
// only); the pass multiplies by 2^(-(n_xy + n_h)/2) when it stores and adds the
// phase w^(n_xy) to one of its diagonal ops (or applies it at the store).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace sim {
namespace {

constexpr float kS2 = 0.70710678118654752f;  // 1/sqrt(2)

struct RegArgs {
  int n, k;
  const OpRec* ops;
  int op_count;
  int src;
  const NodeEntry* nodes;
  int64_t slot_begin;
  const float2* src_base;
  float2* dst_base;
  uint8_t cpos[16];      // qubit of each compute rank
  uint8_t spos[16];      // qubit of each storage rank
  uint8_t c2s[16];       // storage rank of each compute rank
  uint8_t swz[16];       // slot XOR mask of each storage rank (0 below rank 4)
  uint8_t cswz[16];      // swz of the storage rank of each compute rank
  uint8_t nonlocal[32];  // non-local qubits (block index bits)
  float init_val;
  float scale;           // 2^(-(n_xy + n_h)/2): the real part of the factors left out
  int phase_e;           // w^phase_e: their phase
  int phase_op;          // diagonal op that takes the phase (-1: the store)
  int transpose;
  int vec4;              // runs of 4 consecutive amplitudes on register bits 0, 1
  uint32_t xs_bytes;     // shared-memory slots before the copy of the ops
};

// 4 consecutive complex64 amplitudes (32 bytes, 32-byte aligned) in one access; the
// data is streamed once, so it does not allocate in L1
__device__ __forceinline__ void load_run4(const float2* p, float2& a, float2& b, float2& c, float2& d) {
  asm volatile("ld.global.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y), "=f"(c.x), "=f"(c.y), "=f"(d.x), "=f"(d.y)
               : "l"(p));
}
__device__ __forceinline__ void store_run4(float2* p, float2 a, float2 b, float2 c, float2 d) {
  asm volatile("st.global.L1::no_allocate.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x),
               "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
               : "memory");
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// (a0, a1) <- the unscaled update of the pair
//   [[1, -i], [-i, 1]] (X^1/2):  a0 - i a1, a1 - i a0
//   [[1, -1], [1, 1]]  (Y^1/2):  a0 - a1,   a0 + a1
//   [[1, 1], [1, -1]]  (H):      a0 + a1,   a0 - a1
// The last two are the same on both components (packed fp32x2 additions).
template <int KIND>
__device__ __forceinline__ void pair_update(float2& a0, float2& a1) {
  if (KIND == 1) {
    const float2 b0 = make_float2(a0.x + a1.y, a0.y - a1.x);
    a1 = make_float2(a1.x + a0.y, a1.y - a0.x);
    a0 = b0;
  } else if (KIND == 2) {
    const float2 b0 = sub2(a0, a1);
    a1 = add2(a0, a1);
    a0 = b0;
  } else {
    const float2 b0 = add2(a0, a1);
    a1 = sub2(a0, a1);
    a0 = b0;
  }
}

template <int R, int B, int KIND>
__device__ __forceinline__ void reg_pairs(float2 (&v)[1 << R]) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (!(j & (1 << B))) pair_update<KIND>(v[j], v[j | (1 << B)]);
}

template <int R, int B>
__device__ __forceinline__ void reg_gate_b(float2 (&v)[1 << R], int kind) {
  if constexpr (B < R) {
    if (kind == 1)
      reg_pairs<R, B, 1>(v);
    else if (kind == 2)
      reg_pairs<R, B, 2>(v);
    else
      reg_pairs<R, B, 3>(v);
  }
}

template <int R>
__device__ __forceinline__ void reg_gate(float2 (&v)[1 << R], int b, int kind) {
  switch (b) {
    case 0: reg_gate_b<R, 0>(v, kind); break;
    case 1: reg_gate_b<R, 1>(v, kind); break;
    case 2: reg_gate_b<R, 2>(v, kind); break;
    case 3: reg_gate_b<R, 3>(v, kind); break;
    case 4: reg_gate_b<R, 4>(v, kind); break;
    default: break;
  }
}

// One side of a pair from its own value o and the partner's value p; side 0 holds
// a0 and side 1 holds a1, sg = -1 on side 0 and +1 on side 1 (same unscaled updates
// as pair_update).
template <int KIND>
__device__ __forceinline__ float2 side_update(float2 o, float2 p, float sg) {
  if (KIND == 1) {  // o - i p on both sides
    return __ffma2_rn(make_float2(1.f, -1.f), make_float2(p.y, p.x), o);
  } else if (KIND == 2) {  // side 0: o - p, side 1: o + p
    return __ffma2_rn(make_float2(sg, sg), p, o);
  } else {  // side 0: p + o, side 1: p - o
    return __ffma2_rn(make_float2(-sg, -sg), o, p);
  }
}

template <int R, int KIND>
__device__ __forceinline__ void lane_gate_k(float2 (&v)[1 << R], int mask, float sg) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    float2 p;
    p.x = __shfl_xor_sync(0xffffffffu, v[j].x, mask);
    p.y = __shfl_xor_sync(0xffffffffu, v[j].y, mask);
    v[j] = side_update<KIND>(v[j], p, sg);
  }
}

template <int R, int KIND>
__device__ __forceinline__ void smem_gate_k(float2 (&v)[1 << R], float2* xs, int t, int pt, float sg) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) xs[j * 256 + t] = v[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) v[j] = side_update<KIND>(v[j], xs[j * 256 + pt], sg);
  __syncthreads();
}

struct Diag {
  uint32_t tmask, pmask, pval, zmask, w1mask, w2mask;
  int nsh;
  uint32_t sh_d[kMaxShift], sh_m[kMaxShift];
};

__device__ __forceinline__ void load_diag(const OpRec* op, uint64_t node_id, Diag& d) {
  d.tmask = op->tmask;
  d.nsh = op->nsh;
#pragma unroll
  for (int s = 0; s < kMaxShift; ++s) {
    d.sh_d[s] = op->sh_d[s];
    d.sh_m[s] = op->sh_m[s];
  }
  const int ncut = op->ncut;
  const uint32_t cutz = op->cutz;
  d.pmask = d.pval = d.zmask = d.w1mask = d.w2mask = 0;
  for (int i = 0; i < ncut; ++i) {
    const uint32_t qb = 1u << op->cutq[i];
    const uint32_t l = (uint32_t)((node_id >> op->cutm[i]) & 1ull);
    if (!((cutz >> i) & 1u)) {
      d.pmask |= qb;
      if (l) d.pval |= qb;
    } else if (l) {
      // phase slot w^{cutw l x}: weight bits 4 (Z^l), 2 and 1
      const uint32_t w = op->cutw[i];
      if (w & 4u) d.zmask |= qb;
      if (w & 2u) d.w2mask |= qb;
      if (w & 1u) d.w1mask |= qb;
    }
  }
}

// slot XOR mask of a storage index built from the thread bits t (ranks 0..7)
__device__ __forceinline__ uint32_t swz_thread(const RegArgs& a, uint32_t t) {
  uint32_t z = 0;
#pragma unroll
  for (int r = 4; r < 8; ++r)
    if ((t >> r) & 1u) z ^= a.swz[r];
  return z;
}

// Per block: the pass's ops (read by every thread) copied to shared memory, and
// the table of w^e.
__device__ __forceinline__ void block_setup(const RegArgs& a, OpRec* s_ops, float2* s_omega, int t) {
  static_assert(sizeof(OpRec) % 8 == 0, "ops are copied in 8-byte words");
  const int nw = a.op_count * (int)(sizeof(OpRec) / 8);
  const uint2* g = (const uint2*)a.ops;
  for (int i = t; i < nw; i += (int)blockDim.x) ((uint2*)s_ops)[i] = __ldg(g + i);
  if (t < 8) {
    // w^t: (+-1, 0), (0, +-1) for even t; (+-1/sqrt2, +-1/sqrt2) for odd t
    const int quad = t >> 1;
    float re, im;
    if (t & 1) {
      re = (quad == 0 || quad == 3) ? kS2 : -kS2;
      im = (quad <= 1) ? kS2 : -kS2;
    } else {
      re = quad == 0 ? 1.f : (quad == 2 ? -1.f : 0.f);
      im = quad == 1 ? 1.f : (quad == 3 ? -1.f : 0.f);
    }
    s_omega[t] = make_float2(re, im);
  }
}

// The pass's ops on one block of 2^k amplitudes held in compute order: thread t
// keeps elements j of v; base holds the block's non-local index bits and node_id
// the copy-tree node (its cut-slot values).
template <int R>
__device__ __forceinline__ void run_ops(const RegArgs& a, float2 (&v)[1 << R], float2* xs, const OpRec* s_ops,
                                        const float2* s_omega, int t, uint32_t base, uint64_t node_id) {
  constexpr int NE = 1 << R;
  const int lane = t & 31;
  // compute-order global index bits for the diagonal ops
  uint32_t xt = base;
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if ((t >> r) & 1) xt |= 1u << a.cpos[r];
  for (int o = 0; o < a.op_count; ++o) {
    const OpRec* op = s_ops + o;
    if (op->type == OP_SWAP) {
      // exchange warp ranks 5+m with register ranks 10+m (m < NSW): the element at
      // (t, j) afterwards is the one at t with warp bits from j's bits 2.., and j
      // with those bits from t's warp bits (reads conflict-free: for fixed j a
      // warp reads 32 consecutive slots)
      constexpr int NSW = R >= 5 ? 3 : 0;  // the planner exchanges only at k = 13
      if constexpr (NSW > 0) {
        constexpr int MS = (1 << NSW) - 1;
#pragma unroll
        for (int j = 0; j < NE; ++j) xs[j * 256 + t] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NE; ++j) {
          const int old_t = (t & ~(MS << 5)) | (((j >> 2) & MS) << 5);
          const int old_j = (j & ~(MS << 2)) | (((t >> 5) & MS) << 2);
          v[j] = xs[old_j * 256 + old_t];
        }
        __syncthreads();
        xt = base;
#pragma unroll
        for (int r = 0; r < 8; ++r)
          if ((t >> r) & 1) xt |= 1u << op->tq[r];
      }
      continue;
    }
    if (op->type == OP_GATE) {
      const int lq = op->lq;
      const int kind = op->kind;
      if (lq >= 8) {
        reg_gate<R>(v, lq - 8, kind);
      } else if (lq < 5) {
        const float sg = ((lane >> lq) & 1) ? 1.f : -1.f;
        const int mask = 1 << lq;
        if (kind == 1)
          lane_gate_k<R, 1>(v, mask, sg);
        else if (kind == 2)
          lane_gate_k<R, 2>(v, mask, sg);
        else
          lane_gate_k<R, 3>(v, mask, sg);
      } else {
        const float sg = ((t >> lq) & 1) ? 1.f : -1.f;
        const int pt = t ^ (1 << lq);
        if (kind == 1)
          smem_gate_k<R, 1>(v, xs, t, pt, sg);
        else if (kind == 2)
          smem_gate_k<R, 2>(v, xs, t, pt, sg);
        else
          smem_gate_k<R, 3>(v, xs, t, pt, sg);
      }
    } else {
      // exponent of w at x = xt | r(j): the thread part (T and CZ terms within xt)
      // once per op, the register part from the op's table, and the CZ pairs between
      // a register qubit and a thread or non-local qubit as 4 popc(j & B)
      const uint32_t tmask = op->tmask;
      const int nsh = op->nsh;
      int s2 = 0;
#pragma unroll 1
      for (int s = 0; s < nsh; ++s) s2 += __popc(xt & (xt >> op->sh_d[s]) & op->sh_m[s]);
      int et = __popc(xt & tmask) + 4 * s2 + (o == a.phase_op ? a.phase_e : 0);
      uint32_t B = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t pq = op->pq[r];
        if (pq != 0xFFu && ((xt >> pq) & 1u)) B |= 1u << r;
      }
      // cut slots of this copy-tree node: Z^l signs and P_l projectors, split the
      // same way
      bool proj = false, keep_t = true;
      uint32_t pm_r = 0, pv_r = 0;
      uint32_t wreg = 0;  // weights 1 and 2 of phase slots on register ranks, 2 bits per rank
      if (op->ncut) {
        Diag d;
        load_diag(op, node_id, d);
        et += 4 * __popc(xt & d.zmask) + __popc(xt & d.w1mask) + 2 * __popc(xt & d.w2mask);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t qb = 1u << op->rq[r];
          if (d.zmask & qb) B ^= 1u << r;
          if (d.w1mask & qb) wreg |= 1u << (2 * r);
          if (d.w2mask & qb) wreg |= 2u << (2 * r);
          if (d.pmask & qb) {
            pm_r |= 1u << r;
            if (d.pval & qb) pv_r |= 1u << r;
          }
        }
        if (d.pmask) {
          proj = true;
          keep_t = (xt & d.pmask & ~op->regmask) == (d.pval & ~op->regmask);
        }
      }
      // Exponents of 8 elements at a time, one 4-bit field per element (element
      // 8w + i in field i of word w): the register-part table plus et in every
      // field (each field stays below 15, so no carries), then the cross-CZ sign
      // 4 popc(B & j) mod 8 as an XOR of 4 into the fields with odd parity of
      // B & j.  kPar[r]: the fields i (of 0..7) whose bit r is set.
      constexpr uint32_t kPar[3] = {0x40404040u, 0x44004400u, 0x44440000u};
      uint32_t par0 = 0;
#pragma unroll
      for (int r = 0; r < 3 && r < R; ++r)
        if ((B >> r) & 1u) par0 ^= kPar[r];
      const uint32_t et8 = (uint32_t)(et & 7) * 0x11111111u;
      uint32_t ew[4];
#pragma unroll
      for (int w4 = 0; w4 < 4; ++w4) {
        if (w4 * 8 < NE) {
          const uint32_t hi = (uint32_t)__popc(B & (uint32_t)(w4 << 3)) & 1u;
          ew[w4] = (op->ereg[w4] + et8) ^ par0 ^ (hi ? 0x44444444u : 0u);
        } else {
          ew[w4] = 0u;
        }
      }
      if (wreg) {
        // weights 1..3 of phase slots on register rank r: + w_r in the fields of the
        // elements j with bit r set.  Each add follows a reduction of every field to
        // its value mod 8 (fields stay below 16, no carries between fields).
        constexpr uint32_t kAdd[3] = {0x10101010u, 0x11001100u, 0x11110000u};
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t wr = (wreg >> (2 * r)) & 3u;
          if (!wr) continue;
#pragma unroll
          for (int w4 = 0; w4 < 4; ++w4) {
            if (w4 * 8 >= NE) continue;
            const uint32_t pat = r < 3 ? kAdd[r] : (((w4 >> (r - 3)) & 1) ? 0x11111111u : 0u);
            ew[w4] = (ew[w4] & 0x77777777u) + wr * pat;
          }
        }
      }
      // projector: the elements j with (j & pm_r) == pv_r, as a bit mask over j
      uint32_t kmask = 0xFFFFFFFFu;
      if (proj) {
        constexpr uint32_t kJ[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
#pragma unroll
        for (int r = 0; r < R; ++r)
          if ((pm_r >> r) & 1u) kmask &= ((pv_r >> r) & 1u) ? kJ[r] : ~kJ[r];
        if (!keep_t) kmask = 0u;
      }
      // field i of a word, as the byte offset 8 e of w^e in s_omega
      auto omega_at = [&](int j) {
        const uint32_t w = ew[j >> 3];
        const int i = j & 7;
        const uint32_t off = (i == 0 ? (w << 3) : (w >> (4 * i - 3))) & 0x38u;
        return *(const float2*)((const char*)s_omega + off);
      };
      if (op->sign_only) {
        // every exponent is 0 or 4 mod 8: flip the sign where bit 2 of the field is
        // set (field i of a word at bits 4i .. 4i+3, so bit 2 moves up by 29 - 4i)
        auto flip = [&](int j) {
          const uint32_t sm = (ew[j >> 3] << (29 - 4 * (j & 7))) & 0x80000000u;
          v[j] = make_float2(__uint_as_float(__float_as_uint(v[j].x) ^ sm),
                             __uint_as_float(__float_as_uint(v[j].y) ^ sm));
        };
        if (proj) {
#pragma unroll
          for (int j = 0; j < NE; ++j) {
            flip(j);
            if (!((kmask >> j) & 1u)) v[j] = make_float2(0.f, 0.f);
          }
        } else {
#pragma unroll
          for (int j = 0; j < NE; ++j) flip(j);
        }
      } else if (proj) {
#pragma unroll
        for (int j = 0; j < NE; ++j) {
          v[j] = cmul(v[j], omega_at(j));
          if (!((kmask >> j) & 1u)) v[j] = make_float2(0.f, 0.f);
        }
      } else {
#pragma unroll
        for (int j = 0; j < NE; ++j) v[j] = cmul(v[j], omega_at(j));
      }
    }
  }
}

template <int R>
__global__ void __launch_bounds__(256, (R >= 5 ? 2 : 3)) sweep_reg_kernel(RegArgs a) {
  constexpr int NE = 1 << R;
  extern __shared__ float2 xs[];  // 2^k slots (transposes, warp-rank gates), then the ops
  __shared__ float2 s_omega[8];   // w^e, w = e^{i pi / 4}
  const int t = threadIdx.x;
  // the pass's ops, read by every thread: one copy in shared memory per block
  OpRec* s_ops = (OpRec*)((char*)xs + a.xs_bytes);
  block_setup(a, s_ops, s_omega, t);
  const uint32_t nb_log = (uint32_t)(a.n - a.k);
  const uint64_t bid = blockIdx.x;
  const int64_t slot = a.slot_begin + (int64_t)(bid >> nb_log);
  const uint32_t g = (uint32_t)(bid & ((1ull << nb_log) - 1));
  const NodeEntry ne = a.nodes[slot];
  const uint64_t stride = 1ull << a.n;
  float2* dst = a.dst_base + (uint64_t)ne.dst_row * stride;
  const float2* src = a.src == SRC_PARENT ? a.src_base + (uint64_t)ne.parent_slot * stride : (const float2*)dst;
  uint32_t base = 0;
  for (uint32_t i = 0; i < nb_log; ++i)
    if ((g >> i) & 1u) base |= 1u << a.nonlocal[i];
  // storage-order address of this thread's elements: st | sreg(j) (stores, and
  // loads outside vec4); vec4 loads use the pass's initial compute order: lt | lreg(j)
  uint32_t st = base, lt = base;
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if ((t >> r) & 1) {
      st |= 1u << a.spos[r];
      lt |= 1u << a.cpos[r];
    }
  auto sreg = [&](int j) {
    uint32_t o = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if ((j >> r) & 1) o |= 1u << a.spos[8 + r];
    return o;
  };
  auto lreg = [&](int j) {
    uint32_t o = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if ((j >> r) & 1) o |= 1u << a.cpos[8 + r];
    return o;
  };
  float2 v[NE];
  if (a.src == SRC_UNIFORM) {
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = make_float2(a.init_val, 0.f);
  } else if (a.src == SRC_ZERO) {
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = make_float2((st | sreg(j)) == 0 ? 1.f : 0.f, 0.f);
  } else if constexpr (R >= 2) {
#pragma unroll
    for (int j = 0; j < NE; j += 4) load_run4(src + (lt | lreg(j)), v[j], v[j + 1], v[j + 2], v[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = src[st | sreg(j)];
  }
  // Storage <-> compute order through shared memory, for passes with fewer than
  // two register bits (wider passes load and store 256-bit runs in compute order
  // and never transpose, so none of this is live across their ops): storage index
  // s = t + 256 j sits at s ^ swz(s); the compute-order element (t, j) is storage
  // index P(t) | P(j).  Byte offsets: the storage slot of (t, j) is
  // (sb_t ^ zb(j)) + 2048 j (the swizzle touches only the low 4 slot bits, below
  // the j bits), the compute slot cb_t ^ cb(j).
  auto transpose = [&](bool to_compute) {
    const uint32_t sb_t = ((uint32_t)t ^ swz_thread(a, (uint32_t)t)) << 3;
    uint32_t zb_r[R > 0 ? R : 1], cb_r[R > 0 ? R : 1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      zb_r[r] = (uint32_t)a.swz[8 + r] << 3;
      cb_r[r] = ((1u << a.c2s[8 + r]) ^ a.cswz[8 + r]) << 3;
    }
    auto sbyte = [&](int j) {
      uint32_t z = 0;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if ((j >> r) & 1) z ^= zb_r[r];
      return (sb_t ^ z) + ((uint32_t)j << 11);
    };
    uint32_t cb_t = 0, z = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if ((t >> r) & 1) {
        cb_t |= 1u << a.c2s[r];
        z ^= a.cswz[r];
      }
    cb_t = (cb_t ^ z) << 3;
    auto cbyte = [&](int j) {
      uint32_t o = cb_t;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if ((j >> r) & 1) o ^= cb_r[r];
      return o;
    };
    char* xsb = (char*)xs;
    if (to_compute) {
#pragma unroll
      for (int j = 0; j < NE; ++j) *(float2*)(xsb + sbyte(j)) = v[j];
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = *(const float2*)(xsb + cbyte(j));
      __syncthreads();
    } else {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NE; ++j) *(float2*)(xsb + cbyte(j)) = v[j];
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = *(const float2*)(xsb + sbyte(j));
    }
  };
  __syncthreads();  // s_omega, s_ops
  if constexpr (R < 2)
    if (a.transpose) transpose(true);
  run_ops<R>(a, v, xs, s_ops, s_omega, t, base, ne.node_id);
  if constexpr (R < 2)
    if (a.transpose) transpose(false);
  if (a.phase_op < 0 && a.phase_e != 0) {
    const float2 w = s_omega[a.phase_e & 7];
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = cmul(v[j], w);
  }
  const float2 sc2 = make_float2(a.scale, a.scale);
  if constexpr (R >= 2) {
#pragma unroll
    for (int j = 0; j < NE; j += 4)
      store_run4(dst + (st | sreg(j)), __fmul2_rn(v[j], sc2), __fmul2_rn(v[j + 1], sc2), __fmul2_rn(v[j + 2], sc2),
                 __fmul2_rn(v[j + 3], sc2));
  } else {
#pragma unroll
    for (int j = 0; j < NE; ++j) dst[st | sreg(j)] = __fmul2_rn(v[j], sc2);
  }
}


template <int R>
cudaError_t launch_r(const RegArgs& a, int64_t nslots, int use_smem, cudaStream_t s) {
  const uint32_t xs_bytes = use_smem ? (uint32_t)(sizeof(float2) << (8 + R)) : 0u;
  const size_t smem = xs_bytes + (size_t)a.op_count * sizeof(OpRec);
  static DeviceOnce attr;
  {
    cudaError_t e = attr.run([](int&) {
      return cudaFuncSetAttribute(sweep_reg_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((sizeof(float2) << (8 + R)) + kMaxPassOps * sizeof(OpRec)));
    });
    if (e != cudaSuccess) return e;
  }
  const uint64_t bps = 1ull << (a.n - a.k);
  const int64_t max_slots = (int64_t)((1ull << 30) / bps) > 0 ? (int64_t)((1ull << 30) / bps) : 1;
  RegArgs b = a;
  b.xs_bytes = xs_bytes;
  for (int64_t s0 = 0; s0 < nslots; s0 += max_slots) {
    const int64_t ns = (nslots - s0) < max_slots ? (nslots - s0) : max_slots;
    b.slot_begin = s0;
    sweep_reg_kernel<R><<<(unsigned)(ns * bps), 256, smem, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launches(SIM_PHASE_SWEEP, 1);
  }
  return cudaSuccess;
}

}  // namespace

bool sweep2_supported(const SweepLaunch& L) {
  return L.k >= 8 && L.k <= 13 && L.low == 5 && L.n >= L.k && !L.general_gates && L.op_count <= kMaxPassOps;
}

cudaError_t launch_sweep2_c64(const SweepLaunch& L, cudaStream_t s) {
  if (!sweep2_supported(L)) return cudaErrorInvalidValue;
  RegArgs a;
  memset(&a, 0, sizeof a);
  a.n = L.n;
  a.k = L.k;
  a.ops = L.ops;
  a.op_count = L.op_count;
  a.src = L.src;
  a.nodes = L.nodes;
  a.src_base = (const float2*)L.src_base;
  a.dst_base = (float2*)L.dst_base;
  // validate both orders: permutations of the same k local qubits, storage ranks
  // 0..4 = qubits 0..4, slot masks only on storage ranks >= 4 and below 16
  uint32_t seen_c = 0, seen_s = 0;
  int srank[32];
  for (int q = 0; q < 32; ++q) srank[q] = -1;
  // vec4: runs of 4 amplitudes on register bits 0, 1 in both the load (initial)
  // and the store (final) order
  // (k >= 10 always: those kernels are compiled for this layout only)
  if ((L.k >= 10) != (L.vec4 != 0)) return cudaErrorInvalidValue;
  if (L.vec4 && (L.transpose || L.order[8] != 0 || L.order[9] != 1 || L.sorder[8] != 0 || L.sorder[9] != 1))
    return cudaErrorInvalidValue;
  for (int r = 0; r < L.k; ++r) {
    const int qc = L.order[r], qs = L.sorder[r];
    if (qc >= L.n || qs >= L.n || (seen_c & (1u << qc)) || (seen_s & (1u << qs))) return cudaErrorInvalidValue;
    if (!L.vec4 && r < 5 && qs != r) return cudaErrorInvalidValue;
    if ((r < 4 && L.swz[r] != 0) || L.swz[r] > 15) return cudaErrorInvalidValue;
    seen_c |= 1u << qc;
    seen_s |= 1u << qs;
    srank[qs] = r;
    a.cpos[r] = (uint8_t)qc;
    a.spos[r] = (uint8_t)qs;
    a.swz[r] = L.swz[r];
  }
  if (seen_c != seen_s) return cudaErrorInvalidValue;
  if (!L.transpose && !L.vec4)
    for (int r = 0; r < L.k; ++r)
      if (L.order[r] != L.sorder[r]) return cudaErrorInvalidValue;
  for (int r = 0; r < L.k; ++r) {
    a.c2s[r] = (uint8_t)srank[L.order[r]];
    a.cswz[r] = L.swz[a.c2s[r]];
  }
  int nn = 0;
  for (int q = 0; q < L.n; ++q)
    if (!(seen_c & (1u << q))) a.nonlocal[nn++] = (uint8_t)q;
  if (nn != L.n - L.k) return cudaErrorInvalidValue;
  a.init_val = (float)ldexp(1.0, -(L.n / 2)) * ((L.n & 1) ? 0.70710678118654752f : 1.f);
  a.scale = L.scale;
  a.phase_e = L.phase_e & 7;
  a.phase_op = L.phase_op < L.op_count ? L.phase_op : -1;
  a.transpose = L.transpose;
  a.vec4 = L.vec4;
  const int use_smem = L.warp_gates > 0 || L.transpose;
  // passes that read a state (not the first pass of a root) at k = 13 run persistent
  switch (L.k - 8) {
    case 0: return launch_r<0>(a, L.nslots, use_smem, s);
    case 1: return launch_r<1>(a, L.nslots, use_smem, s);
    case 2: return launch_r<2>(a, L.nslots, use_smem, s);
    case 3: return launch_r<3>(a, L.nslots, use_smem, s);
    case 4: return launch_r<4>(a, L.nslots, use_smem, s);
    default: return launch_r<5>(a, L.nslots, use_smem, s);
  }
}

}  // namespace sim
