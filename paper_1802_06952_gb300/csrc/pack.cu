// Split-pack of the leaf half-states into the operands of the tensor-core
// contraction A(x_u, x_l) = sum_k U_k[x_u] L_k[x_l] (Supplementary A, Eq. 8).
//
// The complex product is embedded in a real GEMM whose fp32 output row is the
// complex64 output row: with a = L_k[m] and b = U_k[j],
//   C[m][2j]   = sum_k  a.re * b.re + a.im * (-b.im)     (real part)
//   C[m][2j+1] = sum_k  a.re * b.im + a.im *   b.re      (imaginary part)
// so the A operand row m holds (a.re, a.im) at columns (2k, 2k+1) and the B
// operand holds row 2j = (b.re, -b.im) and row 2j+1 = (b.im, b.re) at the same
// columns.  Each value v is split as hi = round(v), lo = round(v - hi) in bf16 or
// fp16; the contraction sums hi*hi + hi*lo + lo*hi.  Columns 2K .. kpad-1 are zero.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace sim {
namespace {

constexpr int TR = 64;   // rows (selected indices) per block
constexpr int TK = 32;   // copies per block -> 64 operand columns = 128 bytes

template <bool FP16>
struct Split;
template <>
struct Split<false> {
  __device__ static void run(float v, uint16_t& hi, uint16_t& lo) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  }
};
template <>
struct Split<true> {
  __device__ static void run(float v, uint16_t& hi, uint16_t& lo) {
    __half h = __float2half_rn(v);
    __half l = __float2half_rn(v - __half2float(h));
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
  }
};

// IS_B = false: A operand (rows = nsel); IS_B = true: B operand (rows = 2 nsel).
template <bool IS_B, bool FP16>
__global__ void __launch_bounds__(256) pack_kernel(const float2* __restrict__ leaves, int64_t K,
                                                   int64_t nsel, int64_t kpad, const float* scale_dev,
                                                   float scale_host, uint16_t* __restrict__ hi,
                                                   uint16_t* __restrict__ lo) {
  __shared__ float2 tile[TK][TR + 1];
  const int64_t r0 = (int64_t)blockIdx.x * TR;
  const int64_t k0 = (int64_t)blockIdx.y * TK;
  const float scale = scale_dev ? *scale_dev : scale_host;
  // load TK copies x TR entries (coalesced along the entries)
  for (int t = threadIdx.x; t < TK * TR; t += blockDim.x) {
    const int kk = t / TR, rr = t % TR;
    const int64_t k = k0 + kk, r = r0 + rr;
    float2 v = make_float2(0.f, 0.f);
    if (k < K && r < nsel) v = leaves[k * nsel + r];
    tile[kk][rr] = make_float2(v.x * scale, v.y * scale);
  }
  __syncthreads();
  // each thread writes 16 consecutive operand columns (8 copies) of one row
  const int rows_out = IS_B ? 2 * TR : TR;
  for (int t = threadIdx.x; t < rows_out * 4; t += blockDim.x) {
    const int orow = t / 4, quarter = t % 4;
    const int rr = IS_B ? orow / 2 : orow;
    const int64_t grow = IS_B ? 2 * r0 + orow : r0 + orow;
    if (r0 + rr >= nsel) continue;
    uint16_t h[16], l[16];
    for (int c = 0; c < 8; ++c) {
      const float2 v = tile[quarter * 8 + c][rr];
      float x0, x1;
      if (!IS_B) {
        x0 = v.x; x1 = v.y;
      } else if ((orow & 1) == 0) {
        x0 = v.x; x1 = -v.y;
      } else {
        x0 = v.y; x1 = v.x;
      }
      Split<FP16>::run(x0, h[2 * c], l[2 * c]);
      Split<FP16>::run(x1, h[2 * c + 1], l[2 * c + 1]);
    }
    const int64_t col = 2 * k0 + quarter * 16;
    if (col >= kpad) continue;
    uint4* ph = reinterpret_cast<uint4*>(hi + grow * kpad + col);
    uint4* pl = reinterpret_cast<uint4*>(lo + grow * kpad + col);
    const uint32_t* h32 = reinterpret_cast<const uint32_t*>(h);
    const uint32_t* l32 = reinterpret_cast<const uint32_t*>(l);
    ph[0] = make_uint4(h32[0], h32[1], h32[2], h32[3]);
    ph[1] = make_uint4(h32[4], h32[5], h32[6], h32[7]);
    pl[0] = make_uint4(l32[0], l32[1], l32[2], l32[3]);
    pl[1] = make_uint4(l32[4], l32[5], l32[6], l32[7]);
  }
}

// block-wise max of |re|, |im|; result combined with atomicMax on the float bits
// (valid for non-negative floats)
__global__ void absmax_kernel(const float2* x, int64_t count, float* out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = x[i];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

// io[0] = max -> io[1] = power-of-two scale s with max * s in [2^13, 2^14): the
// fp16 hi parts stay below the fp16 maximum and the lo parts of typical entries
// stay above the fp16 subnormal range.
__global__ void scale_from_max_kernel(float* io) {
  const float m = io[0];
  float s = 1.f;
  if (m > 0.f && isfinite(m)) {
    int e;
    frexpf(m, &e);               // m = f * 2^e, f in [0.5, 1)
    s = ldexpf(1.f, 14 - e);     // m * s in [2^13, 2^14)
  }
  io[1] = s;
}

template <bool IS_B>
cudaError_t launch_pack(const void* leaves, int64_t K, int64_t nsel, int64_t kpad, int fp16,
                        const float* scale_dev, void* hi, void* lo, cudaStream_t s) {
  if (nsel == 0 || K == 0) return cudaSuccess;
  dim3 grid((unsigned)((nsel + TR - 1) / TR), (unsigned)((kpad / 2 + TK - 1) / TK));
  if (fp16)
    pack_kernel<IS_B, true><<<grid, 256, 0, s>>>((const float2*)leaves, K, nsel, kpad, scale_dev,
                                                  1.f, (uint16_t*)hi, (uint16_t*)lo);
  else
    pack_kernel<IS_B, false><<<grid, 256, 0, s>>>((const float2*)leaves, K, nsel, kpad, scale_dev,
                                                   1.f, (uint16_t*)hi, (uint16_t*)lo);
  note_launches(SIM_PHASE_PACK, 1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_a(const void* leaves, int64_t K, int64_t nsel, int64_t kpad, int fp16,
                          const float* scale_dev, void* hi, void* lo, cudaStream_t s) {
  return launch_pack<false>(leaves, K, nsel, kpad, fp16, scale_dev, hi, lo, s);
}

cudaError_t launch_pack_b(const void* leaves, int64_t K, int64_t nsel, int64_t kpad, int fp16,
                          const float* scale_dev, void* hi, void* lo, cudaStream_t s) {
  return launch_pack<true>(leaves, K, nsel, kpad, fp16, scale_dev, hi, lo, s);
}

cudaError_t launch_absmax_c64(const void* x, int64_t count, float* out_dev, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  absmax_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float2*)x, count, out_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scale_from_max_kernel<<<1, 1, 0, s>>>(out_dev);
  note_launches(SIM_PHASE_PACK, 2);
  return cudaGetLastError();
}

namespace {
__global__ void gather_flat_kernel(const float2* __restrict__ src, const uint64_t* __restrict__ idx, int64_t n,
                                   float2* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}
}  // namespace

cudaError_t launch_gather_flat_c64(const void* src, const uint64_t* idx, int64_t n, void* dst, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  gather_flat_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float2*)src, idx, n, (float2*)dst);
  note_launches(SIM_PHASE_GATHER, 1);
  return cudaGetLastError();
}

}  // namespace sim
