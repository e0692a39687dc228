// dcp_probe_fp64: measures the FP64 arithmetic rate of the current device.
//
// On GB300 every binary64 program of the library (stencil time-stepping, the
// f64 map chain, the reverse passes) is bound by the FP64 pipes, not by
// device memory, and the device's FP64 rate is not one of the published or
// otherwise measured peaks.  This probe gives the roofline denominator for
// those kernels: every SM runs warps whose threads advance independent
// chains of one FP64 operation (fused multiply-add, add or multiply), so the
// pipe, not a dependency chain, limits the issue rate; 4, 8 and 16 chains
// per thread are timed (CUDA events on the caller's stream) and the best
// rate is reported.
#include <cuda_runtime.h>

#include "dcp_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

// Results of the chains land here only when they equal a value the host
// passes (never in practice), which keeps the arithmetic live without
// writing device memory the caller would have to provide.
static __device__ double dcp_probe_sink[kChains];
// 1.0 in device memory, one per chain: values the compiler cannot see, so
// each chain's multiplier is a register of its own (op 4)
static __device__ double dcp_probe_ones[16] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};

template <int OP, int CHAINS>
__global__ void __launch_bounds__(kThreads) fp64_probe_kernel(long long iters, double b, double c,
                                                              double sentinel) {
  // every chain has its own multiplier and addend registers: operands shared
  // by all chains (one b, one c) measured about 16 % below the rate that
  // fused kernels reach on the same pipe
  double a[CHAINS], bb[CHAINS], cc[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) {
    a[k] = (double)(threadIdx.x + k) * 1e-3;
    bb[k] = OP == 4 ? dcp_probe_ones[k] : b - k * 1e-9;
    cc[k] = c + k * 1e-9;
  }
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) {
      if (OP == 0) a[k] = __fma_rn(a[k], bb[k], cc[k]);
      else if (OP == 1) a[k] = __dadd_rn(a[k], cc[k]);
      else if (OP == 2) a[k] = __dmul_rn(a[k], bb[k]);
      else if (OP == 3) a[k] = __fma_rn(a[k], b, cc[k]);  // an add as a fused multiply-add by b = 1
      else a[k] = __fma_rn(a[k], bb[k], cc[k]);  // the same, each chain with its own 1.0
    }
  }
#pragma unroll
  for (int k = 0; k < CHAINS; ++k)
    if (a[k] == sentinel) dcp_probe_sink[k % kChains] = a[k];
}

// Times one launch of the probe; returns milliseconds, and in *lane_ops the
// binary64 operations it performed.
template <int OP, int CHAINS>
float launch_and_time(long long iters, cudaStream_t s, double* lane_ops) {
  // b slightly below 1 (exactly 1 for the add issued as a fused
  // multiply-add, a value the compiler cannot see) and c small keep every
  // chain finite and normal
  const double b = OP == 3 ? 1.0 : 0.9999999, c = 1e-7, sentinel = -12345.678;
  int dev = 0, sms = 0, per_sm = 0;
  dcp::check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  dcp::check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                  "cudaDeviceGetAttribute");
  dcp::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &per_sm, fp64_probe_kernel<OP, CHAINS>, kThreads, 0), "occupancy");
  const int grid = sms * per_sm;
  cudaEvent_t e0, e1;
  dcp::check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  dcp::check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  fp64_probe_kernel<OP, CHAINS><<<grid, kThreads, 0, s>>>(iters / 8 + 1, b, c, sentinel);
  dcp::check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
  fp64_probe_kernel<OP, CHAINS><<<grid, kThreads, 0, s>>>(iters, b, c, sentinel);
  dcp::check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
  dcp::check_cuda(cudaGetLastError(), "launch of the FP64 probe");
  dcp::check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
  float ms = 0.f;
  dcp::check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *lane_ops = (double)grid * kThreads * CHAINS * (double)iters;
  return ms;
}

// Best rate over chain counts 4, 8 and 16 (10^9 lane operations per second).
template <int OP>
double best_rate(long long iters, cudaStream_t s, float* ms_out) {
  double best = 0.0, ops = 0.0;
  const float t4 = launch_and_time<OP, 4>(iters * 2, s, &ops);
  if (t4 > 0.f && ops / (t4 * 1e-3) / 1e9 > best) best = ops / (t4 * 1e-3) / 1e9, *ms_out = t4;
  const float t8 = launch_and_time<OP, 8>(iters, s, &ops);
  if (t8 > 0.f && ops / (t8 * 1e-3) / 1e9 > best) best = ops / (t8 * 1e-3) / 1e9, *ms_out = t8;
  const float t16 = launch_and_time<OP, 16>(iters / 2 + 1, s, &ops);
  if (t16 > 0.f && ops / (t16 * 1e-3) / 1e9 > best) best = ops / (t16 * 1e-3) / 1e9, *ms_out = t16;
  return best;
}

}  // namespace

extern "C" dcp_status dcp_probe_fp64(int32_t op, int64_t iters, double* gops, double* ms,
                                     void* cuda_stream) {
  try {
    if (!gops) dcp::fail(DCP_E_INVALID_ARG, "gops is NULL");
    if (op < 0 || op > 4)
      dcp::fail(DCP_E_INVALID_ARG,
                "op must be 0 (fma), 1 (add), 2 (mul), 3 or 4 (add as fma by 1, shared or per chain)");
    if (iters < 1 || iters > (1ll << 24)) dcp::fail(DCP_E_INVALID_ARG, "iters must be in [1, 2^24]");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    float t = 0.f;
    double g = op == 0   ? best_rate<0>(iters, s, &t)
               : op == 1 ? best_rate<1>(iters, s, &t)
               : op == 2 ? best_rate<2>(iters, s, &t)
               : op == 3 ? best_rate<3>(iters, s, &t)
                         : best_rate<4>(iters, s, &t);
    if (!(g > 0.0)) dcp::fail(DCP_E_CUDA, "FP64 probe timed at zero");
    *gops = g;
    if (ms) *ms = t;
    return DCP_OK;
  } catch (const dcp::Error& e) {
    dcp::set_last_error(e.msg);
    return e.code;
  } catch (...) {
    dcp::set_last_error("internal error in dcp_probe_fp64");
    return DCP_E_INVALID_ARG;
  }
}
