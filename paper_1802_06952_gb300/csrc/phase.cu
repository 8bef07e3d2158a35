// Output-phase cuts: a cut CZ (h, k) with no later non-diagonal gate on either qubit
// is applied to the final amplitudes as the sign (-1)^{x_h x_k} instead of as a copy
// bit of Supplementary A, Eq. 1.  Every output row (lower index x_l) and column
// (upper index x_u) gets a code with bit m set where its index has the bit of cut m;
// the sign of an entry is the parity of (row code & column code).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace sim {
namespace {

struct CodeQubits {
  int nm;
  int q[32];  // half-local qubit of cut m
};

__global__ void out_codes_kernel(const uint64_t* sel, int64_t n, CodeQubits cq, uint32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t x = sel ? sel[i] : (uint64_t)i;
    uint32_t c = 0;
    for (int m = 0; m < cq.nm; ++m) c |= (uint32_t)((x >> cq.q[m]) & 1ull) << m;
    out[i] = c;
  }
}

// one thread per (row, pair of columns); complex64 entries are float2, complex128
// entries double2
template <typename T>
__global__ void out_sign_kernel(T* C, int64_t M, int64_t N, const uint32_t* lcode, const uint32_t* ucode) {
  const int64_t total = M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / N, c = i - r * N;
    if (__popc(lcode[r] & ucode[c]) & 1) {
      T v = C[i];
      v.x = -v.x;
      v.y = -v.y;
      C[i] = v;
    }
  }
}

unsigned grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_out_codes(const uint64_t* sel, int64_t n, const int* qubits, int nm, uint32_t* out,
                             cudaStream_t s) {
  if (nm < 0 || nm > 32 || n <= 0) return n == 0 ? cudaSuccess : cudaErrorInvalidValue;
  CodeQubits cq;
  cq.nm = nm;
  for (int m = 0; m < 32; ++m) cq.q[m] = m < nm ? qubits[m] : 0;
  for (int m = 0; m < nm; ++m)
    if (cq.q[m] < 0 || cq.q[m] > 63) return cudaErrorInvalidValue;
  out_codes_kernel<<<grid_of(n), 256, 0, s>>>(sel, n, cq, out);
  note_launches(SIM_PHASE_CONTRACT, 1);
  return cudaGetLastError();
}

cudaError_t launch_out_sign(void* C, int is_c128, int64_t M, int64_t N, const uint32_t* lcode, const uint32_t* ucode,
                            cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (is_c128)
    out_sign_kernel<double2><<<grid_of(M * N), 256, 0, s>>>((double2*)C, M, N, lcode, ucode);
  else
    out_sign_kernel<float2><<<grid_of(M * N), 256, 0, s>>>((float2*)C, M, N, lcode, ucode);
  note_launches(SIM_PHASE_CONTRACT, 1);
  return cudaGetLastError();
}

}  // namespace sim
