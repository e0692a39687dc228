// dcp_reduce_noalloc: the library's whole-array reduction for callers that
// must not allocate device memory.
//
// Who needs it: a caller whose device memory is entirely owned by its own
// pool allocator (a framework's caching allocator that has reserved the
// GPU), a caller on an out-of-memory recovery path where any new allocation
// may fail, or a caller that has promised its host application a fixed
// memory footprint.  The graph path allocates its reduction scratch with
// cudaMalloc on first run; this entry point instead uses a fixed scratch
// array compiled into the library, so a call needs no allocation at all.
//
// The reduction is the same one the fused kernels use: per-thread
// accumulators, a warp-shuffle / shared-memory tree per CTA, one partial per
// CTA, and a single deterministic cross-CTA pass done by whichever CTA takes
// the last ticket.  Here each CTA owns a fixed chunk of kChunk elements, so
// the scratch bounds the input length: n <= kChunk * kMaxCtas.
#include <cuda_runtime.h>

#include <mutex>

#include "dcp_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 32768;  // elements reduced by one CTA
constexpr int kMaxCtas = 65536;      // partial slots in the scratch
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: kMaxCtas 8-byte partials, then
// the ticket counter.  512 KiB + 256 B per device, held until the process
// exits.  Host code must not use this name as an address; it obtains the
// device address with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned long long dcp_noalloc_scratch[kMaxCtas + 32];

template <typename T> struct Fin { typedef double type; };
template <> struct Fin<int> { typedef long long type; };
template <> struct Fin<long long> { typedef long long type; };

template <typename T> __device__ __forceinline__ T nan_max(T a, T b) { return (b > a || b != b) ? b : a; }
template <typename T> __device__ __forceinline__ T nan_min(T a, T b) { return (b < a || b != b) ? b : a; }

template <typename T> __device__ __forceinline__ T absval(T a) { return a < (T)0 ? (T)(-a) : a; }
__device__ __forceinline__ int absval(int a) { return a < 0 ? (int)(0u - (unsigned)a) : a; }
__device__ __forceinline__ long long absval(long long a) {
  return a < 0 ? (long long)(0ull - (unsigned long long)a) : a;
}

template <typename A> __device__ __forceinline__ A add_wrap(A a, A b) { return a + b; }
__device__ __forceinline__ int add_wrap(int a, int b) { return (int)((unsigned)a + (unsigned)b); }
__device__ __forceinline__ long long add_wrap(long long a, long long b) {
  return (long long)((unsigned long long)a + (unsigned long long)b);
}

template <typename A> __device__ __forceinline__ A combine(int red, A a, A b) {
  if (red == DCP_SUM) return add_wrap(a, b);
  if (red == DCP_MIN_R) return nan_min(a, b);
  return nan_max(a, b);
}

template <typename T> __device__ __forceinline__ T identity(int red);
template <> __device__ __forceinline__ float identity<float>(int red) {
  return red == DCP_SUM || red == DCP_MAXABS ? 0.0f
                                             : (red == DCP_MAX_R ? -__int_as_float(0x7f800000)
                                                                 : __int_as_float(0x7f800000));
}
template <> __device__ __forceinline__ double identity<double>(int red) {
  return red == DCP_SUM || red == DCP_MAXABS
             ? 0.0
             : (red == DCP_MAX_R ? -__longlong_as_double(0x7ff0000000000000ll)
                                 : __longlong_as_double(0x7ff0000000000000ll));
}
template <> __device__ __forceinline__ int identity<int>(int red) {
  return red == DCP_SUM ? 0 : (red == DCP_MIN_R ? 0x7fffffff : (int)0x80000000);
}
template <> __device__ __forceinline__ long long identity<long long>(int red) {
  return red == DCP_SUM ? 0ll
                        : (red == DCP_MIN_R ? 0x7fffffffffffffffll : (long long)0x8000000000000000ull);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    reduce_noalloc_kernel(const T* __restrict__ in, long long n, int red, T* out,
                          typename Fin<T>::type* partials, unsigned int* ticket) {
  typedef typename Fin<T>::type F;
  __shared__ T s_w[kThreads / 32];
  __shared__ F s_f[kThreads / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long begin = (long long)blockIdx.x * kChunk;
  const long long end = begin + kChunk < n ? begin + kChunk : n;
  T acc = identity<T>(red);
  for (long long i = begin + threadIdx.x; i < end; i += kThreads) {
    T v = in[i];
    if (red == DCP_MAXABS) v = absval(v);
    acc = combine(red, acc, v);
  }
  for (int m = 16; m >= 1; m >>= 1) acc = combine(red, acc, __shfl_xor_sync(0xffffffffu, acc, m));
  if (lane == 0) s_w[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    T v = s_w[0];
    for (int w = 1; w < kThreads / 32; ++w) v = combine(red, v, s_w[w]);
    partials[blockIdx.x] = (F)v;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  F f = (F)identity<T>(red);
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += kThreads) f = combine(red, f, __ldcg(partials + b));
  for (int m = 16; m >= 1; m >>= 1) f = combine(red, f, __shfl_xor_sync(0xffffffffu, f, m));
  if (lane == 0) s_f[warp] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    F v = s_f[0];
    for (int w = 1; w < kThreads / 32; ++w) v = combine(red, v, s_f[w]);
    *out = (T)v;
    *ticket = 0u;
  }
}

std::mutex g_setup_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up once per device).
void* scratch_on_current_device() {
  int dev = -1;
  dcp::check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) dcp::fail(DCP_E_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    dcp::check_cuda(cudaGetSymbolAddress(&p, dcp_noalloc_scratch),
                    "cudaGetSymbolAddress(no-allocation scratch)");
    g_scratch[dev] = p;
  }
  return g_scratch[dev];
}

template <typename T>
void launch(const void* in, long long n, int red, void* out, cudaStream_t s, void* scratch) {
  typedef typename Fin<T>::type F;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(
      static_cast<unsigned long long*>(scratch) + kMaxCtas);
  // the ticket must start at zero; a completed call leaves it at zero, this
  // clears what an interrupted call may have left
  dcp::check_cuda(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s), "cudaMemsetAsync(ticket)");
  long long grid = (n + kChunk - 1) / kChunk;
  if (grid < 1) grid = 1;
  reduce_noalloc_kernel<T><<<(unsigned)grid, kThreads, 0, s>>>(
      static_cast<const T*>(in), n, red, static_cast<T*>(out), static_cast<F*>(scratch), ticket);
  dcp::check_cuda(cudaGetLastError(), "launch of the no-allocation reduction");
}

}  // namespace

extern "C" dcp_status dcp_reduce_noalloc(const void* in, int64_t n, int32_t dtype, int32_t red,
                                         void* out, void* cuda_stream) {
  try {
    if (!out) dcp::fail(DCP_E_INVALID_ARG, "out is NULL");
    if (n < 0) dcp::fail(DCP_E_SHAPE, "n must be >= 0");
    if (n > 0 && !in) dcp::fail(DCP_E_INVALID_ARG, "in is NULL");
    if (red < DCP_SUM || red > DCP_MAXABS) dcp::fail(DCP_E_INVALID_ARG, "unknown reduction");
    if (red != DCP_SUM && n == 0) dcp::fail(DCP_E_SHAPE, "max/min of an empty array is undefined");
    if (n > kChunk * (long long)kMaxCtas)
      dcp::fail(DCP_E_INVALID_ARG,
                "n = " + std::to_string((long long)n) +
                    " exceeds the no-allocation maximum of 2^31 elements (fixed scratch of 65536 "
                    "partials); use a graph reduction instead");
    int esz = dcp::dtype_size(dtype);
    if (!esz) dcp::fail(DCP_E_DTYPE, "unknown dtype");
    if (((uintptr_t)in % esz) || ((uintptr_t)out % esz))
      dcp::fail(DCP_E_INVALID_ARG, "buffers must be aligned to their element size");
    void* scratch = scratch_on_current_device();
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    switch (dtype) {
      case DCP_F32: launch<float>(in, n, red, out, s, scratch); break;
      case DCP_F64: launch<double>(in, n, red, out, s, scratch); break;
      case DCP_I32: launch<int>(in, n, red, out, s, scratch); break;
      case DCP_I64: launch<long long>(in, n, red, out, s, scratch); break;
    }
    return DCP_OK;
  } catch (const dcp::Error& e) {
    dcp::set_last_error(e.msg);
    return e.code;
  } catch (...) {
    dcp::set_last_error("internal error in dcp_reduce_noalloc");
    return DCP_E_INVALID_ARG;
  }
}
