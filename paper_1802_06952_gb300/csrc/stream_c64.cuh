// Streaming reads of complex64 arrays for the one-pass reductions (statistics,
// the Born sampler's bound): 32-byte vector loads, two in flight per thread, so
// that a grid of a few blocks per SM keeps enough bytes in flight for HBM.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sim {

// 4 consecutive complex64 values (32 bytes, 32-byte aligned), streamed past L1
__device__ __forceinline__ void ld_run4(const float2* p, float2 (&r)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r[0].x), "=f"(r[0].y), "=f"(r[1].x), "=f"(r[1].y), "=f"(r[2].x), "=f"(r[2].y), "=f"(r[3].x),
                 "=f"(r[3].y)
               : "l"(p));
}

// Calls f(value) for every complex64 value of a[0 .. count): a head of up to 3
// values up to the first 32-byte boundary, then runs of 4 values loaded 32 bytes at
// a time with two runs in flight per thread (grid-stride), then the tail.  Every
// value is visited exactly once; the order does not matter to the callers.
template <class F>
__device__ __forceinline__ void for_each_c64(const float2* a, uint64_t count, F&& f) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  uint64_t head = (uint64_t)((32u - ((uint32_t)(uintptr_t)a & 31u)) & 31u) / sizeof(float2);
  if (head > count) head = count;
  if (tid < head) f(a[tid]);
  const float2* b = a + head;
  const uint64_t nrun = (count - head) / 4;
  uint64_t r = tid;
  for (; r + nth < nrun; r += 2 * nth) {
    float2 x[4], y[4];
    ld_run4(b + 4 * r, x);
    ld_run4(b + 4 * (r + nth), y);
#pragma unroll
    for (int i = 0; i < 4; ++i) f(x[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) f(y[i]);
  }
  if (r < nrun) {
    float2 x[4];
    ld_run4(b + 4 * r, x);
#pragma unroll
    for (int i = 0; i < 4; ++i) f(x[i]);
  }
  const uint64_t done = head + 4 * nrun;
  if (tid < count - done) f(a[done + tid]);
}

}  // namespace sim
