// FP64 parts of the GPU path:
//   fp64_gemm_kernel  the plain contraction A(x_u, x_l) = sum_k U_k[x_u] L_k[x_l]
//                     (Supplementary A, Eq. 8) with complex128 products and sums on
//                     CUDA cores: 64 x 64 output tiles, 256 threads, 4 x 4 outputs each
//   stats_kernel      the Section 3 statistics of an amplitude block (norm, mean of
//                     w = 2^n|A|^2, mean of ln w, histogram of u = 1 - exp(-w) for the
//                     KS distance to Eq. 7): per-element work in the input precision,
//                     running sums in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sim.h"
#include "sim_internal.h"
#include "stream_c64.cuh"

namespace sim {
namespace {

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

constexpr int GT = 64;  // output tile edge
constexpr int GK = 8;   // copies per smem stage

template <typename T>
__global__ void __launch_bounds__(256) fp64_gemm_kernel(const T* __restrict__ L, const T* __restrict__ U,
                                                        int64_t K, int64_t M, int64_t N, int accumulate,
                                                        double2* __restrict__ C) {
  __shared__ double2 Ls[GK][GT];
  __shared__ double2 Us[GK][GT];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t m0 = (int64_t)blockIdx.y * GT, j0 = (int64_t)blockIdx.x * GT;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int64_t k0 = 0; k0 < K; k0 += GK) {
    for (int t = threadIdx.x; t < GK * GT; t += blockDim.x) {
      const int kk = t / GT, c = t % GT;
      const int64_t k = k0 + kk;
      Ls[kk][c] = (k < K && m0 + c < M) ? to_d2(L[k * M + m0 + c]) : make_double2(0.0, 0.0);
      Us[kk][c] = (k < K && j0 + c < N) ? to_d2(U[k * N + j0 + c]) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ls[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Us[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t jj = j0 + tx + 16 * j;
      if (jj >= N) continue;
      double2* d = C + m * N + jj;
      if (accumulate) {
        double2 o = *d;
        o.x += acc[i][j].x;
        o.y += acc[i][j].y;
        *d = o;
      } else {
        *d = acc[i][j];
      }
    }
  }
}

// Bin of u = 1 - exp(-w) (the Eq. 7 CDF, alpha = 1, at z = ln w) on [0, 1) in
// SIM_KS_BINS equal bins; u = 1 goes to the last bin.  complex64 blocks use the
// same fp32 arithmetic as the contraction's fused statistics.
__device__ __forceinline__ int u_bin(float w) {
  int b = (int)((1.f - __expf(-w)) * (float)SIM_KS_BINS);
  return b < 0 ? 0 : (b > SIM_KS_BINS - 1 ? SIM_KS_BINS - 1 : b);
}

__device__ __forceinline__ int u_bin_d(double w) {
  const double u = -expm1(-w);
  int b = (int)(u * (double)SIM_KS_BINS);
  return b < 0 ? 0 : (b > SIM_KS_BINS - 1 ? SIM_KS_BINS - 1 : b);
}

template <bool C128>
__global__ void __launch_bounds__(256) stats_kernel(const void* amps, uint64_t count, int nq, double* acc,
                                                    unsigned long long* hist) {
  __shared__ unsigned int sh[SIM_KS_BINS];
  for (int i = threadIdx.x; i < SIM_KS_BINS; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  double sp = 0.0, sl = 0.0, nz = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if (!C128) {
    // fp32 per element, the two running sums compensated (Kahan: the rounding of
    // each add is carried in c and fed back), the count an integer; FP64 only once
    // per thread at the end (GB300's FP64 pipe retires two operations per clock
    // per SM, so no FP64 instruction may sit on the per-element path)
    const float sc = ldexpf(1.f, nq);
    float fp = 0.f, cp = 0.f, fl = 0.f, cl = 0.f;
    uint32_t cnt = 0;
    auto kahan = [](float& sum, float& c, float x) {
      const float y = x - c;
      const float t = sum + y;
      c = (t - sum) - y;
      sum = t;
    };
    for_each_c64((const float2*)amps, count, [&](float2 v) {
      const float p = fmaf(v.x, v.x, v.y * v.y);
      const float w = p * sc;
      kahan(fp, cp, p);
      const bool pos = w > 0.f;
      kahan(fl, cl, pos ? __logf(w) : 0.f);
      cnt += pos ? 1u : 0u;
      atomicAdd(&sh[u_bin(w)], 1u);
    });
    sp = (double)fp - (double)cp;
    sl = (double)fl - (double)cl;
    nz = (double)cnt;
  } else {
    const double2* a = (const double2*)amps;
    const double sc = ldexp(1.0, nq);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += stride) {
      const double2 v = a[i];
      const double p = v.x * v.x + v.y * v.y;
      const double w = p * sc;
      sp += p;
      if (w > 0.0) {
        sl += log(w);
        nz += 1.0;
      }
      atomicAdd(&sh[u_bin_d(w)], 1u);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], sp);
    atomicAdd(&acc[1], sl);
    atomicAdd(&acc[2], nz);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SIM_KS_BINS; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

}  // namespace

cudaError_t launch_fp64_gemm(const void* lsel, const void* usel, int in_c128, int64_t K, int64_t M, int64_t N,
                             int accumulate, void* C, cudaStream_t s) {
  if (M == 0 || N == 0) return cudaSuccess;
  const int64_t gx = (N + GT - 1) / GT, gy = (M + GT - 1) / GT;
  if (gy > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)gy);
  if (in_c128)
    fp64_gemm_kernel<double2><<<grid, 256, 0, s>>>((const double2*)lsel, (const double2*)usel, K, M, N, accumulate,
                                                   (double2*)C);
  else
    fp64_gemm_kernel<float2><<<grid, 256, 0, s>>>((const float2*)lsel, (const float2*)usel, K, M, N, accumulate,
                                                  (double2*)C);
  note_launches(SIM_PHASE_FP64_GEMM, 1);
  return cudaGetLastError();
}

cudaError_t launch_stats(const void* amps, int is_c128, uint64_t count, int nq, double* acc_dev,
                         unsigned long long* hist_dev, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc_dev, 0, 3 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(hist_dev, 0, SIM_KS_BINS * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaSuccess;
  // four resident blocks per SM (16 KB histogram each), as many as the block needs
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (count + 255) / 256;
  if (blocks > (uint64_t)sms * 4) blocks = (uint64_t)sms * 4;
  if (is_c128)
    stats_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(amps, count, nq, acc_dev, hist_dev);
  else
    stats_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(amps, count, nq, acc_dev, hist_dev);
  note_launches(SIM_PHASE_STATS, 1);
  return cudaGetLastError();
}

}  // namespace sim
