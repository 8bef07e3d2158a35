// Register-blocked fused gate sweep over complex64 half-states (Supplementary A,
// Eq. 4 gate by gate; the diagonal gates of a layer combined into one phase and
// mask per amplitude, Section 2.4, Eqs. 3-6).
//
// A block of 256 threads stages the 2^k amplitudes (k = 8 + R) whose local qubits
// the pass schedule chose.  Staged index i = t + 256 j: the 8 thread bits t are
// ranks 0..7 (ranks 0..4 = qubits 0..4, the warp lanes, so every warp reads and
// writes 256 contiguous bytes; ranks 5..7 = the warp index), the R register bits
// j are ranks 8..k-1.  Each thread keeps its 2^R amplitudes in registers for the
// whole pass:
//   gate on a register rank  pairs of registers, no data exchange
//   gate on a lane rank      partner value by warp shuffle
//   gate on a warp rank      partner value through shared memory (two barriers)
//   diagonal op              per amplitude phase w^e and projector test
// X^1/2, Y^1/2 and H are applied as 2 X^1/2, 2 Y^1/2 and sqrt2 H (additions only);
// the pass multiplies by the product of the omitted factors when it stores.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace sim {
namespace {

constexpr float kS2 = 0.70710678118654752f;  // 1/sqrt(2)

struct Sweep2Args {
  int n, k;
  const OpRec* ops;
  int op_count;
  int src;
  const NodeEntry* nodes;
  int64_t slot_begin;
  const float2* src_base;
  float2* dst_base;
  uint8_t pos[16];       // qubit of each local rank
  uint8_t nonlocal[32];  // non-local qubits (block index bits)
  float init_val;
  float scale;           // product of the factors the unscaled gate updates leave out
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// The gate updates below are the matrices of X^1/2 and Y^1/2 times 2 and of H
// times sqrt 2, so they need only additions; the pass multiplies its result once
// by the product of the removed factors (PassDesc::scale).
//   2 X^1/2 = [[1+i, 1-i], [1-i, 1+i]]      2 Y^1/2 = [[1+i, -1-i], [1+i, 1+i]]
//   sqrt2 H = [[1, 1], [1, -1]]
// (a0, a1) <- 2U (a0, a1), register pairs
template <int KIND>
__device__ __forceinline__ void pair_update(float2& a0, float2& a1) {
  const float2 s = cadd(a0, a1), d = csub(a0, a1);
  if (KIND == 1) {         // s + i d, s - i d
    a0 = make_float2(s.x - d.y, s.y + d.x);
    a1 = make_float2(s.x + d.y, s.y - d.x);
  } else if (KIND == 2) {  // (1+i) d, (1+i) s
    a0 = make_float2(d.x - d.y, d.x + d.y);
    a1 = make_float2(s.x - s.y, s.x + s.y);
  } else {                 // s, d
    a0 = s;
    a1 = d;
  }
}

// One side of a pair from its own value and the partner's: new = alpha own + beta p,
// with (alpha, beta) for side 0 (holding a0) and side 1 (holding a1):
//   2 X^1/2: (1+i, 1-i) on both sides
//   2 Y^1/2: side 0 (1+i, -1-i), side 1 (1+i, 1+i)
//   sqrt2 H: side 0 (1, 1), side 1 (-1, 1)
__device__ __forceinline__ void side_coeffs(int kind, int side, float2& al, float2& be) {
  if (kind == 1) {
    al = make_float2(1.f, 1.f);
    be = make_float2(1.f, -1.f);
  } else if (kind == 2) {
    al = make_float2(1.f, 1.f);
    be = side ? make_float2(1.f, 1.f) : make_float2(-1.f, -1.f);
  } else {
    al = make_float2(side ? -1.f : 1.f, 0.f);
    be = make_float2(1.f, 0.f);
  }
}

template <int R, int B>
__device__ __forceinline__ void reg_gate_b(float2 (&v)[1 << R], int kind) {
  if constexpr (B < R) {
    if (kind == 1) {
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j & (1 << B))) pair_update<1>(v[j], v[j | (1 << B)]);
    } else if (kind == 2) {
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j & (1 << B))) pair_update<2>(v[j], v[j | (1 << B)]);
    } else {
#pragma unroll
      for (int j = 0; j < (1 << R); ++j)
        if (!(j & (1 << B))) pair_update<3>(v[j], v[j | (1 << B)]);
    }
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

struct Diag {
  uint32_t tmask, pmask, pval, zmask;
  int nsh;
  uint32_t sh_d[kMaxShift], sh_m[kMaxShift];
};

__device__ __forceinline__ void load_diag2(const OpRec* op, uint64_t node_id, Diag& d) {
  d.tmask = __ldg(&op->tmask);
  d.nsh = __ldg(&op->nsh);
#pragma unroll
  for (int s = 0; s < kMaxShift; ++s) {
    d.sh_d[s] = __ldg(&op->sh_d[s]);
    d.sh_m[s] = __ldg(&op->sh_m[s]);
  }
  const int ncut = __ldg(&op->ncut);
  const int half = __ldg(&op->half);
  d.pmask = d.pval = d.zmask = 0;
  for (int i = 0; i < ncut; ++i) {
    const uint32_t qb = 1u << op->cutq[i];
    const uint32_t l = (uint32_t)((node_id >> op->cutm[i]) & 1ull);
    if (half == 0) {
      d.pmask |= qb;
      if (l) d.pval |= qb;
    } else if (l) {
      d.zmask |= qb;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(256, (R >= 5 ? 2 : 3)) sweep2_kernel(Sweep2Args a) {
  constexpr int NE = 1 << R;
  extern __shared__ float2 xs[];   // 256 * NE values, used by warp-rank gates
  __shared__ float2 s_omega[8];    // w^e, w = e^{i pi / 4}
  const int t = threadIdx.x;
  const int lane = t & 31;
  if (t < 8) {
    // w^t: magnitude 1 on the axes (t even), components +-1/sqrt2 on the diagonals
    const float ax = (t & 1) ? kS2 : 1.f;
    const int quad = t >> 1;  // 0: (+,+) 1: (-,+) 2: (-,-) 3: (+,-) for odd t
    float re, im;
    if (t & 1) {
      re = (quad == 0 || quad == 3) ? ax : -ax;
      im = (quad <= 1) ? ax : -ax;
    } else {
      re = quad == 0 ? 1.f : (quad == 2 ? -1.f : 0.f);
      im = quad == 1 ? 1.f : (quad == 3 ? -1.f : 0.f);
    }
    s_omega[t] = make_float2(re, im);
  }
  const uint32_t nb_log = (uint32_t)(a.n - a.k);
  const uint64_t bid = blockIdx.x;
  const int64_t slot = a.slot_begin + (int64_t)(bid >> nb_log);
  const uint32_t g = (uint32_t)(bid & ((1ull << nb_log) - 1));
  const NodeEntry ne = a.nodes[slot];
  const uint64_t stride = 1ull << a.n;
  float2* dst = a.dst_base + (uint64_t)ne.dst_row * stride;
  const float2* src = a.src == SRC_PARENT ? a.src_base + (uint64_t)ne.parent_slot * stride : (const float2*)dst;
  uint32_t xt = 0;
  for (uint32_t i = 0; i < nb_log; ++i)
    if ((g >> i) & 1u) xt |= 1u << a.nonlocal[i];
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if ((t >> r) & 1) xt |= 1u << a.pos[r];
  uint32_t xr[NE];
#pragma unroll
  for (int j = 0; j < NE; ++j) {
    uint32_t o = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if ((j >> r) & 1) o |= 1u << a.pos[8 + r];
    xr[j] = o;
  }
  float2 v[NE];
  if (a.src == SRC_UNIFORM) {
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = make_float2(a.init_val, 0.f);
  } else if (a.src == SRC_ZERO) {
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = make_float2((xt | xr[j]) == 0 ? 1.f : 0.f, 0.f);
  } else {
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = src[xt | xr[j]];
  }
  __syncthreads();
  for (int o = 0; o < a.op_count; ++o) {
    const OpRec* op = a.ops + o;
    if (__ldg(&op->type) == OP_GATE) {
      const int lq = __ldg(&op->lq);
      const int kind = __ldg(&op->kind);
      if (lq >= 8) {
        reg_gate<R>(v, lq - 8, kind);
      } else if (lq < 5) {
        float2 al, be;
        side_coeffs(kind, (lane >> lq) & 1, al, be);
        const int mask = 1 << lq;
#pragma unroll
        for (int j = 0; j < NE; ++j) {
          float2 p;
          p.x = __shfl_xor_sync(0xffffffffu, v[j].x, mask);
          p.y = __shfl_xor_sync(0xffffffffu, v[j].y, mask);
          v[j] = cfma(al, v[j], cmul(be, p));
        }
      } else {
        float2 al, be;
        side_coeffs(kind, (t >> lq) & 1, al, be);
        const int pt = t ^ (1 << lq);
#pragma unroll
        for (int j = 0; j < NE; ++j) xs[j * 256 + t] = v[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NE; ++j) v[j] = cfma(al, v[j], cmul(be, xs[j * 256 + pt]));
        __syncthreads();
      }
    } else {
      Diag d;
      load_diag2(op, ne.node_id, d);
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        const uint32_t x = xt | xr[j];
        int s2 = __popc(x & d.zmask);
#pragma unroll
        for (int s = 0; s < kMaxShift; ++s)
          if (s < d.nsh) s2 += __popc(x & (x >> d.sh_d[s]) & d.sh_m[s]);
        const int e = (__popc(x & d.tmask) + 4 * s2) & 7;
        const bool keep = (x & d.pmask) == d.pval;
        v[j] = keep ? cmul(v[j], s_omega[e]) : make_float2(0.f, 0.f);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NE; ++j) dst[xt | xr[j]] = make_float2(v[j].x * a.scale, v[j].y * a.scale);
}

template <int R>
cudaError_t launch_r(const Sweep2Args& a, int64_t nslots, int use_smem, cudaStream_t s) {
  const size_t smem = use_smem ? (sizeof(float2) << (8 + R)) : 0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(sweep2_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float2) << (8 + R)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const uint64_t bps = 1ull << (a.n - a.k);
  const int64_t max_slots = (int64_t)((1ull << 30) / bps) > 0 ? (int64_t)((1ull << 30) / bps) : 1;
  Sweep2Args b = a;
  for (int64_t s0 = 0; s0 < nslots; s0 += max_slots) {
    const int64_t ns = (nslots - s0) < max_slots ? (nslots - s0) : max_slots;
    b.slot_begin = s0;
    sweep2_kernel<R><<<(unsigned)(ns * bps), 256, smem, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    note_launches(SIM_PHASE_SWEEP, 1);
  }
  return cudaSuccess;
}

}  // namespace

bool sweep2_supported(const SweepLaunch& L) {
  return L.k >= 8 && L.k <= 13 && L.low == 5 && L.n >= L.k && !L.general_gates;
}

cudaError_t launch_sweep2_c64(const SweepLaunch& L, cudaStream_t s) {
  if (!sweep2_supported(L)) return cudaErrorInvalidValue;
  Sweep2Args a;
  memset(&a, 0, sizeof a);
  a.n = L.n;
  a.k = L.k;
  a.ops = L.ops;
  a.op_count = L.op_count;
  a.src = L.src;
  a.nodes = L.nodes;
  a.src_base = (const float2*)L.src_base;
  a.dst_base = (float2*)L.dst_base;
  uint32_t seen = 0;
  for (int r = 0; r < L.k; ++r) {
    const int q = L.order[r];
    if (q >= L.n || (seen & (1u << q))) return cudaErrorInvalidValue;
    if (r < 5 && q != r) return cudaErrorInvalidValue;
    seen |= 1u << q;
    a.pos[r] = (uint8_t)q;
  }
  int nn = 0;
  for (int q = 0; q < L.n; ++q)
    if (!(seen & (1u << q))) a.nonlocal[nn++] = (uint8_t)q;
  if (nn != L.n - L.k) return cudaErrorInvalidValue;
  a.init_val = (float)ldexp(1.0, -(L.n / 2)) * ((L.n & 1) ? 0.70710678118654752f : 1.f);
  a.scale = L.scale;
  const int use_smem = L.warp_gates > 0;
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
