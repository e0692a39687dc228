// dcp_probe_fp64: measures the FP64 arithmetic rate of the current device.
//
// On GB300 every binary64 program of the library (stencil time-stepping, the
// f64 map chain, the reverse passes) is bound by the FP64 pipes, not by
// device memory, and the device's FP64 rate is not one of the published or
// otherwise measured peaks.  This probe gives the roofline denominator for
// those kernels: every SM runs warps whose threads advance eight independent
// chains of one FP64 operation (fused multiply-add, add or multiply), so the
// pipe, not a dependency chain, limits the issue rate.  The kernel is timed
// with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "dcp_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

// Results of the chains land here only when they equal a value the host
// passes (never in practice), which keeps the arithmetic live without
// writing device memory the caller would have to provide.
static __device__ double dcp_probe_sink[kChains];

template <int OP>
__global__ void __launch_bounds__(kThreads) fp64_probe_kernel(long long iters, double b, double c,
                                                              double sentinel) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) a[k] = __fma_rn(a[k], b, c);
      else if (OP == 1) a[k] = __dadd_rn(a[k], c);
      else a[k] = __dmul_rn(a[k], b);
    }
  }
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    if (a[k] == sentinel) dcp_probe_sink[k] = a[k];
}

template <int OP>
float launch_and_time(long long iters, int grid, cudaStream_t s) {
  // b slightly below 1 and c small keep every chain finite and normal
  const double b = 0.9999999, c = 1e-7, sentinel = -12345.678;
  cudaEvent_t e0, e1;
  dcp::check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
  dcp::check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
  fp64_probe_kernel<OP><<<grid, kThreads, 0, s>>>(iters / 8 + 1, b, c, sentinel);  // warm-up
  dcp::check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
  fp64_probe_kernel<OP><<<grid, kThreads, 0, s>>>(iters, b, c, sentinel);
  dcp::check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
  dcp::check_cuda(cudaGetLastError(), "launch of the FP64 probe");
  dcp::check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
  float ms = 0.f;
  dcp::check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace

extern "C" dcp_status dcp_probe_fp64(int32_t op, int64_t iters, double* gops, double* ms,
                                     void* cuda_stream) {
  try {
    if (!gops) dcp::fail(DCP_E_INVALID_ARG, "gops is NULL");
    if (op < 0 || op > 2) dcp::fail(DCP_E_INVALID_ARG, "op must be 0 (fma), 1 (add) or 2 (mul)");
    if (iters < 1 || iters > (1ll << 24)) dcp::fail(DCP_E_INVALID_ARG, "iters must be in [1, 2^24]");
    int dev = 0, sms = 0, per_sm = 0;
    dcp::check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    dcp::check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                    "cudaDeviceGetAttribute");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    float t = 0.f;
    if (op == 0) {
      dcp::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_probe_kernel<0>,
                                                                    kThreads, 0), "occupancy");
      t = launch_and_time<0>(iters, sms * per_sm, s);
    } else if (op == 1) {
      dcp::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_probe_kernel<1>,
                                                                    kThreads, 0), "occupancy");
      t = launch_and_time<1>(iters, sms * per_sm, s);
    } else {
      dcp::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_probe_kernel<2>,
                                                                    kThreads, 0), "occupancy");
      t = launch_and_time<2>(iters, sms * per_sm, s);
    }
    if (t <= 0.f) dcp::fail(DCP_E_CUDA, "FP64 probe timed at zero");
    const double lane_ops = (double)sms * per_sm * kThreads * kChains * (double)iters;
    *gops = lane_ops / (t * 1e-3) / 1e9;
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
