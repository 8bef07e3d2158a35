// Born-rule samples of measurement outcomes from a block of amplitudes (Section 3:
// measurement outcomes of the full vector space), by rejection sampling with a
// measured bound, and their cross-entropy statistics against Eq. 7.
//
// Proposal c draws an index i_c = r_{2c} mod count and a uniform
// u_c = (r_{2c+1} >> 11) 2^-53 from the counter-based splitmix64 stream r of the
// seed (output c: state seed + (c + 1) * 0x9E3779B97F4A7C15, then the published
// finaliser), and is accepted when u_c * p_max < p_{i_c}, with p = |A|^2 formed in
// FP64 from the complex64 amplitudes and p_max the block's maximum of p (measured
// by a reduction before sampling).  Accepted proposals keep the proposal order.
//
// Per round of kRound proposals: one kernel counts the acceptances of each group
// of 1024 proposals, one block scans the counts, and a third kernel recomputes the
// decisions and writes the accepted indices and ordinals at their scanned
// positions (warp ballots keep the order within a group).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sim.h"
#include "runtime.h"
#include "sim_internal.h"
#include "stream_c64.cuh"

using namespace sim;

namespace {

constexpr int kGroup = 1024;                 // proposals per block
constexpr int kGroupsPerRound = 1024;        // blocks per round
constexpr uint64_t kRound = (uint64_t)kGroup * kGroupsPerRound;

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double prob(const float2* a, uint64_t i) {
  const float2 v = a[i];
  return (double)v.x * (double)v.x + (double)v.y * (double)v.y;
}

__device__ __forceinline__ bool decide(const float2* amps, uint64_t count, uint64_t seed, double pmax, uint64_t c,
                                       uint64_t* idx) {
  const uint64_t ri = splitmix64_at(seed, 2ull * c);
  const uint64_t ru = splitmix64_at(seed, 2ull * c + 1ull);
  *idx = ri % count;
  const double u = (double)(ru >> 11) * 0x1.0p-53;
  return u * pmax < prob(amps, *idx);
}

// Exact FP64 maximum of |A|^2 with an FP32 screen: fmaf(re, re, im * im) is within
// 2^-23 of the FP64 value (two roundings of 2^-24), so an element whose FP32 value
// stays below (1 - 2^-20) times the largest FP32 value this thread has seen cannot
// exceed the FP64 maximum it holds.  Only the others are computed in FP64, so the
// pass runs at the speed of its loads instead of GB300's FP64 rate.
// The rare FP64 update sits in a call of its own so that it is a branch taken by
// the few candidates, not a predicated sequence on every element (GB300's FP64
// pipe is slow); its arithmetic is prob()'s, on the loaded floats.
__device__ __noinline__ double max_prob(double m, float x, float y) {
  return fmax(m, (double)x * (double)x + (double)y * (double)y);
}

// The values are streamed 32 bytes at a time (stream_c64.cuh).
__global__ void pmax_kernel(const float2* amps, uint64_t count, double* block_max) {
  double m = 0.0;
  float thr = 0.f;
  for_each_c64(amps, count, [&](float2 a) {
    const float p32 = fmaf(a.x, a.x, a.y * a.y);
    if (p32 >= thr) {
      m = max_prob(m, a.x, a.y);
      thr = fmaxf(thr, p32 * (1.f - 9.5367431640625e-07f));
    }
  });
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) block_max[blockIdx.x] = m;
  }
}

__global__ void max_final_kernel(const double* block_max, int n, double* out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, block_max[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sm[w]);
    m = fmax(m, sm[0]);
    *out = m;
  }
}

// acceptances per group of kGroup proposals (blockDim = kGroup)
__global__ void count_kernel(const float2* amps, uint64_t count, uint64_t seed, const double* pmax, uint64_t c0,
                             uint64_t c_end, uint32_t* counts) {
  const uint64_t c = c0 + blockIdx.x * (uint64_t)kGroup + threadIdx.x;
  uint64_t idx;
  const bool acc = c < c_end && decide(amps, count, seed, *pmax, c, &idx);
  const int n = __syncthreads_count(acc);
  if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)n;
}

// exclusive scan of the group counts (one block of kGroupsPerRound threads)
__global__ void scan_kernel(const uint32_t* counts, uint32_t* offsets, uint32_t* total) {
  __shared__ uint32_t s[kGroupsPerRound];
  const int t = threadIdx.x;
  s[t] = counts[t];
  __syncthreads();
  for (int d = 1; d < kGroupsPerRound; d <<= 1) {
    const uint32_t v = t >= d ? s[t - d] : 0u;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  offsets[t] = s[t] - counts[t];
  if (t == kGroupsPerRound - 1) *total = s[t];
}

// accepted (index, ordinal) at base + offset[group] + rank within the group,
// for output positions below cap
__global__ void write_kernel(const float2* amps, uint64_t count, uint64_t seed, const double* pmax, uint64_t c0,
                             uint64_t c_end, const uint32_t* offsets, uint64_t base, uint64_t cap, uint64_t* idx_out,
                             uint64_t* ord_out) {
  __shared__ uint32_t warp_cnt[kGroup / 32];
  const uint64_t c = c0 + blockIdx.x * (uint64_t)kGroup + threadIdx.x;
  uint64_t idx = 0;
  const bool acc = c < c_end && decide(amps, count, seed, *pmax, c, &idx);
  const unsigned ball = __ballot_sync(0xffffffffu, acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_cnt[warp] = (uint32_t)__popc(ball);
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += warp_cnt[w];
  before += (uint32_t)__popc(ball & ((1u << lane) - 1u));
  if (acc) {
    const uint64_t pos = base + offsets[blockIdx.x] + before;
    if (pos < cap) {
      idx_out[pos] = idx;
      ord_out[pos] = c;
    }
  }
}

// FP64 sums of w = 2^n p and ln w over the accepted samples
__global__ void xeb_kernel(const float2* amps, const uint64_t* idx, uint64_t n, double w_scale, double* acc) {
  double sw = 0.0, sl = 0.0;
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    const double w = prob(amps, idx[s]) * w_scale;
    sw += w;
    sl += log(w);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], sw);
    atomicAdd(&acc[1], sl);
  }
}

#define SCK(x)                                                                                  \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) {                                                                    \
      cudaGetLastError();                                                                       \
      for (void* p_ : bufs) rt_free(p_, st);                                                    \
      return set_error(e_ == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,                \
                       std::string(#x) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                           \
  } while (0)

}  // namespace

int sim_born_sample(const void* amps_dev, uint64_t count, int n_qubits, uint64_t seed, uint64_t n_samples,
                    uint64_t max_proposals, uint64_t* idx_out, uint64_t* ordinal_out, double xeb_out[3],
                    uint64_t* n_out, void* stream) {
  if (!amps_dev || count == 0 || n_samples == 0 || !idx_out || !n_out || n_qubits < 0 || n_qubits > 80)
    return set_error(SIM_EINVAL, "amps_dev, count > 0, n_samples > 0, idx_out and n_out are required");
  if (max_proposals > (1ull << 62)) return set_error(SIM_EINVAL, "max_proposals must be below 2^62");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void*> bufs;
  auto alloc = [&](void** p, size_t n) {
    cudaError_t e = rt_alloc(p, n, st);
    if (e == cudaSuccess) bufs.push_back(*p);
    return e;
  };
  const float2* amps = (const float2*)amps_dev;
  const int max_blocks = 4096;
  double *d_bmax = nullptr, *d_pmax = nullptr, *d_acc = nullptr;
  uint32_t *d_counts = nullptr, *d_offsets = nullptr, *d_total = nullptr;
  uint64_t *d_idx = nullptr, *d_ord = nullptr;
  SCK(alloc((void**)&d_bmax, sizeof(double) * max_blocks));
  SCK(alloc((void**)&d_pmax, sizeof(double)));
  SCK(alloc((void**)&d_acc, 2 * sizeof(double)));
  SCK(alloc((void**)&d_counts, sizeof(uint32_t) * kGroupsPerRound));
  SCK(alloc((void**)&d_offsets, sizeof(uint32_t) * kGroupsPerRound));
  SCK(alloc((void**)&d_total, sizeof(uint32_t)));
  SCK(alloc((void**)&d_idx, sizeof(uint64_t) * n_samples));
  SCK(alloc((void**)&d_ord, sizeof(uint64_t) * n_samples));
  const int nb = (int)std::min<uint64_t>((count + 255) / 256, max_blocks);
  pmax_kernel<<<nb, 256, 0, st>>>(amps, count, d_bmax);
  max_final_kernel<<<1, 1024, 0, st>>>(d_bmax, nb, d_pmax);
  note_launches(SIM_PHASE_STATS, 2);
  SCK(cudaGetLastError());
  double pmax = 0;
  SCK(cudaMemcpyAsync(&pmax, d_pmax, sizeof(double), cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  uint64_t got = 0;
  if (pmax > 0) {
    for (uint64_t c0 = 0; got < n_samples && c0 < max_proposals; c0 += kRound) {
      const uint64_t c_end = std::min<uint64_t>(max_proposals, c0 + kRound);
      const int groups = (int)((c_end - c0 + kGroup - 1) / kGroup);
      SCK(cudaMemsetAsync(d_counts, 0, sizeof(uint32_t) * kGroupsPerRound, st));
      count_kernel<<<groups, kGroup, 0, st>>>(amps, count, seed, d_pmax, c0, c_end, d_counts);
      scan_kernel<<<1, kGroupsPerRound, 0, st>>>(d_counts, d_offsets, d_total);
      write_kernel<<<groups, kGroup, 0, st>>>(amps, count, seed, d_pmax, c0, c_end, d_offsets, got, n_samples, d_idx,
                                              d_ord);
      note_launches(SIM_PHASE_STATS, 3);
      SCK(cudaGetLastError());
      uint32_t total = 0;
      SCK(cudaMemcpyAsync(&total, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      SCK(cudaStreamSynchronize(st));
      got = std::min<uint64_t>(n_samples, got + total);
    }
  }
  double acc[2] = {0, 0};
  if (got) {
    SCK(cudaMemsetAsync(d_acc, 0, 2 * sizeof(double), st));
    const int xb = (int)std::min<uint64_t>((got + 255) / 256, 1024);
    xeb_kernel<<<xb, 256, 0, st>>>(amps, d_idx, got, std::ldexp(1.0, n_qubits), d_acc);
    note_launches(SIM_PHASE_STATS, 1);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(acc, d_acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(idx_out, d_idx, sizeof(uint64_t) * got, cudaMemcpyDeviceToHost, st));
    if (ordinal_out)
      SCK(cudaMemcpyAsync(ordinal_out, d_ord, sizeof(uint64_t) * got, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
  }
  constexpr double kEulerGamma = 0.57721566490153286061;
  if (xeb_out) {
    xeb_out[0] = got ? acc[0] / (double)got - 1.0 : 0.0;
    xeb_out[1] = got ? acc[1] / (double)got + kEulerGamma : 0.0;
    xeb_out[2] = pmax * std::ldexp(1.0, n_qubits);
  }
  *n_out = got;
  for (void* p : bufs) rt_free(p, st);
  return SIM_OK;
}
