// sim_amplitudes_noalloc: the split-precision tensor-core contraction of
// sim_amplitudes, for callers that must not have the library allocate device
// memory while they run.
//
// Who needs it: an application that has already handed the device memory to its
// own allocator (a cudaMalloc from this library would then fail, or carve into
// memory that application has promised elsewhere), and a latency-bound loop that
// cannot afford cudaMalloc / cudaFree, which can block the host and implicitly
// synchronise the device.  sim_amplitudes takes its operand scratch from the
// library's pool, which calls cudaMalloc whenever a size is first seen; this
// entry point never does.
//
// Its scratch (the split operands, the fp16 scales and a status word) lives in
// the file-scope device array below, SIM_NOALLOC_SCRATCH_BYTES in size.  Every
// GPU on which this entry point is used holds that array until the process
// exits.  The host reaches the array only through the device address that
// cudaGetSymbolAddress returns; the array's name in host code is a host-side
// stand-in, and handing it to a kernel would fault or touch the wrong memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/sim.h"
#include "sim_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SIM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Once per device, with that device current: look up the array's device address.
int scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sim::set_error(SIM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sim::set_error(SIM_EUNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return sim::set_error(SIM_ECUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch: ") +
                                           cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return SIM_OK;
}

inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" int sim_amplitudes_noalloc(sim_halves h, int contraction, int accumulate, void* out_dev,
                                      void* stream) {
  using namespace sim;
  HalvesView v;
  if (!halves_view(h, &v) || !out_dev) return set_error(SIM_EINVAL, "halves and out_dev must not be NULL");
  if (contraction != SIM_SPLIT_BF16 && contraction != SIM_SPLIT_FP16)
    return set_error(SIM_EINVAL, "sim_amplitudes_noalloc supports SIM_SPLIT_BF16 and SIM_SPLIT_FP16 only");
  if (v.precision != SIM_C64) return set_error(SIM_EINVAL, "split contractions need complex64 halves (SIM_C64)");
  {
    const int rc = check_split_bf16(contraction, (int64_t)v.K, false);
    if (rc) return rc;
  }
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, out_dev) != cudaSuccess ||
      (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return set_error(SIM_EINVAL, "sim_amplitudes_noalloc writes device memory only (out_dev is not device memory)");
  }
  if (pa.type == cudaMemoryTypeDevice) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return set_error(SIM_ECUDA, "sim_amplitudes_noalloc: cudaGetDevice failed");
    }
    if (pa.device != cur)
      return set_error(SIM_EINVAL, "sim_amplitudes_noalloc: out_dev is memory of device " + std::to_string(pa.device) +
                                       ", not of the current device " + std::to_string(cur));
  }
  const int64_t M = v.nsel[1], N = v.nsel[0];
  const int64_t K = (int64_t)v.K;
  const int64_t kpad = ((2 * K + 63) / 64) * 64;
  const int64_t N2 = 2 * N;
  // scratch layout: [status int][4 fp16 scale floats][A hi][A lo][B hi][B lo]
  const uint64_t a_bytes = align_up((uint64_t)M * kpad * 2, 1024);
  const uint64_t b_bytes = align_up((uint64_t)N2 * kpad * 2, 1024);
  const uint64_t head = 1024;
  const uint64_t need = head + 2 * a_bytes + 2 * b_bytes;
  if (need > (uint64_t)SIM_NOALLOC_SCRATCH_BYTES)
    return set_error(SIM_EINVAL, "sim_amplitudes_noalloc needs " + std::to_string(need) +
                                     " bytes of scratch for this contraction; its fixed scratch holds " +
                                     std::to_string((uint64_t)SIM_NOALLOC_SCRATCH_BYTES) +
                                     " (use sim_amplitudes for larger blocks)");
  void* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  unsigned char* s = (unsigned char*)base;
  int* d_status = (int*)s;
  float* scales = (float*)(s + 256);
  void* ahi = s + head;
  void* alo = s + head + a_bytes;
  void* bhi = s + head + 2 * a_bytes;
  void* blo = s + head + 2 * a_bytes + b_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: the status word must start at 0
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), st);
  const int fp16 = contraction == SIM_SPLIT_FP16;
  const float* sa = nullptr;
  const float* sb = nullptr;
  if (e == cudaSuccess && fp16) {
    e = launch_absmax_c64(v.leafsel[1], K * M, scales, st);
    if (e == cudaSuccess) e = launch_absmax_c64(v.leafsel[0], K * N, scales + 2, st);
    sa = scales + 1;
    sb = scales + 3;
  }
  if (e == cudaSuccess) e = launch_pack_a(v.leafsel[1], K, M, kpad, fp16, sa, ahi, alo, st);
  if (e == cudaSuccess) e = launch_pack_b(v.leafsel[0], K, N, kpad, fp16, sb, bhi, blo, st);
  int num_sms = 0;
  if (e == cudaSuccess) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (e == cudaSuccess) {
    TcGemmArgs g;
    g.a_hi = ahi; g.a_lo = alo; g.b_hi = bhi; g.b_lo = blo;
    g.M = M; g.N2 = N2; g.kpad = kpad;
    g.fp16 = fp16;
    g.scale_a = sa; g.scale_b = sb;
    g.accumulate = accumulate;
    g.C = out_dev;
    g.group_m = 0;
    g.num_sms = num_sms;
    g.d_status = d_status;
    g.out_lcode = v.out_code[1];
    g.out_ucode = v.out_code[0];
    e = launch_tc_gemm(g, st);
  }
  // wait, then report a bounded device wait that gave up
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(SIM_ECUDA, std::string("sim_amplitudes_noalloc: ") + cudaGetErrorString(e));
  if (status != 0) return set_error(SIM_ETIMEOUT, "sim_amplitudes_noalloc: a bounded device wait gave up");
  return SIM_OK;
}
