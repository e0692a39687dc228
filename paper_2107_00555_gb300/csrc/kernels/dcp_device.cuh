// dcp_device.cuh -- device helpers shared by every generated dcp kernel
// (compiled at run time by NVRTC for sm_103a).  Generated sources define,
// before including this header,
//   DCP_T                     element type (float, double, int, long long)
//   constexpr dcp_red_op(r)   reduction op code of reduction slot r.
#pragma once

#define DCP_MAXIO 16

typedef unsigned int dcp_u32;
typedef unsigned long long dcp_u64;

// Final-pass (cross-block) accumulator type: binary64 for floating groups
// (an fp32 partial widens exactly), 64-bit integers for integer groups.
// Aligned pair of elements (paired-cell stencil loads).
template <typename T> struct DcpVec2;
template <> struct DcpVec2<float> { typedef float2 type; };
template <> struct DcpVec2<double> { typedef double2 type; };

template <typename T> struct DcpFin { typedef double type; };
template <> struct DcpFin<int> { typedef long long type; };
template <> struct DcpFin<long long> { typedef long long type; };

// ---------------------------------------------------------------------------
// Elementwise operations.  Floating MAX/MIN propagate NaN (np.maximum):
// a when a > b or a is NaN, else b (b NaN gives b).  Integer arithmetic
// wraps modulo 2^bits through unsigned arithmetic, like NumPy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dcp_max(float a, float b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ float dcp_min(float a, float b) { return (a < b || a != a) ? a : b; }
__device__ __forceinline__ double dcp_max(double a, double b) { return (a > b || a != a) ? a : b; }
__device__ __forceinline__ double dcp_min(double a, double b) { return (a < b || a != a) ? a : b; }
__device__ __forceinline__ int dcp_max(int a, int b) { return a > b ? a : b; }
__device__ __forceinline__ int dcp_min(int a, int b) { return a < b ? a : b; }
__device__ __forceinline__ long long dcp_max(long long a, long long b) { return a > b ? a : b; }
__device__ __forceinline__ long long dcp_min(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ float dcp_neg(float a) { return -a; }
__device__ __forceinline__ double dcp_neg(double a) { return -a; }
__device__ __forceinline__ int dcp_neg(int a) { return (int)(0u - (dcp_u32)a); }
__device__ __forceinline__ long long dcp_neg(long long a) { return (long long)(0ull - (dcp_u64)a); }

__device__ __forceinline__ float dcp_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double dcp_abs(double a) { return fabs(a); }
__device__ __forceinline__ int dcp_abs(int a) { return a < 0 ? dcp_neg(a) : a; }
__device__ __forceinline__ long long dcp_abs(long long a) { return a < 0 ? dcp_neg(a) : a; }

__device__ __forceinline__ float dcp_add(float a, float b) { return a + b; }
__device__ __forceinline__ double dcp_add(double a, double b) { return a + b; }
__device__ __forceinline__ int dcp_add(int a, int b) { return (int)((dcp_u32)a + (dcp_u32)b); }
__device__ __forceinline__ long long dcp_add(long long a, long long b) {
  return (long long)((dcp_u64)a + (dcp_u64)b);
}
__device__ __forceinline__ float dcp_sub(float a, float b) { return a - b; }
__device__ __forceinline__ double dcp_sub(double a, double b) { return a - b; }
__device__ __forceinline__ int dcp_sub(int a, int b) { return (int)((dcp_u32)a - (dcp_u32)b); }
__device__ __forceinline__ long long dcp_sub(long long a, long long b) {
  return (long long)((dcp_u64)a - (dcp_u64)b);
}
__device__ __forceinline__ float dcp_mul(float a, float b) { return a * b; }
__device__ __forceinline__ double dcp_mul(double a, double b) { return a * b; }
__device__ __forceinline__ int dcp_mul(int a, int b) { return (int)((dcp_u32)a * (dcp_u32)b); }
__device__ __forceinline__ long long dcp_mul(long long a, long long b) {
  return (long long)((dcp_u64)a * (dcp_u64)b);
}
__device__ __forceinline__ float dcp_div(float a, float b) { return a / b; }
__device__ __forceinline__ double dcp_div(double a, double b) { return a / b; }

template <typename T> __device__ __forceinline__ T dcp_square(T a) { return dcp_mul(a, a); }

// Stencil weighted sums use explicit rounding intrinsics so that every kernel
// form (tile, stream, batched, any time-tile depth) performs bit-identical
// per-step arithmetic: acc = w0*x0, then acc = fma(wk, xk, acc) in point order.
__device__ __forceinline__ float dcp_mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double dcp_mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float dcp_fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double dcp_fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T> __device__ __forceinline__ T dcp_sign(T a) {
  return a > (T)0 ? (T)1 : (a < (T)0 ? (T)-1 : (T)0);
}
template <typename T> __device__ __forceinline__ T dcp_gt(T a, T b) { return a > b ? (T)1 : (T)0; }
template <typename T> __device__ __forceinline__ T dcp_lt(T a, T b) { return a < b ? (T)1 : (T)0; }

__device__ __forceinline__ float dcp_exp(float a) { return expf(a); }
__device__ __forceinline__ double dcp_exp(double a) { return exp(a); }
__device__ __forceinline__ float dcp_sin(float a) { return sinf(a); }
__device__ __forceinline__ double dcp_sin(double a) { return sin(a); }
__device__ __forceinline__ float dcp_cos(float a) { return cosf(a); }
__device__ __forceinline__ double dcp_cos(double a) { return cos(a); }
__device__ __forceinline__ float dcp_tanh(float a) { return tanhf(a); }
__device__ __forceinline__ double dcp_tanh(double a) { return tanh(a); }
__device__ __forceinline__ float dcp_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double dcp_sqrt(double a) { return sqrt(a); }

// ---------------------------------------------------------------------------
// Reductions (write-conflict resolution).  Op codes: 0 sum, 1 max, 2 min,
// 3 maxabs.  The thread accumulator has the element type; the cross-block
// pass uses DcpFin<T>.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T dcp_red_init(int op);
template <> __device__ __forceinline__ float dcp_red_init<float>(int op) {
  return op == 0 ? 0.0f : (op == 1 ? -__int_as_float(0x7f800000) : (op == 2 ? __int_as_float(0x7f800000) : 0.0f));
}
template <> __device__ __forceinline__ double dcp_red_init<double>(int op) {
  return op == 0 ? 0.0 : (op == 1 ? -__longlong_as_double(0x7ff0000000000000ll)
                                  : (op == 2 ? __longlong_as_double(0x7ff0000000000000ll) : 0.0));
}
template <> __device__ __forceinline__ int dcp_red_init<int>(int op) {
  return op == 0 ? 0 : (op == 2 ? 0x7fffffff : (int)0x80000000);
}
template <> __device__ __forceinline__ long long dcp_red_init<long long>(int op) {
  return op == 0 ? 0ll : (op == 2 ? 0x7fffffffffffffffll : (long long)0x8000000000000000ull);
}

// Value entering the reduction (maxabs takes |y|).
template <typename T> __device__ __forceinline__ T dcp_red_lift(int op, T y) {
  return op == 3 ? dcp_abs(y) : y;
}
template <typename T> __device__ __forceinline__ T dcp_red_comb(int op, T a, T b) {
  if (op == 0) return dcp_add(a, b);
  if (op == 2) return (b < a || b != b) ? b : a;
  return (b > a || b != b) ? b : a;
}
// binary64 max|y|: both operands are magnitudes (sign bit clear), whose bit
// patterns, read as unsigned integers, order like the values, with every NaN
// above +inf, so the NaN-propagating maximum is an integer comparison and
// spends nothing on the FP64 pipe (the bound of binary64 maps on GB300).
template <> __device__ __forceinline__ double dcp_red_comb<double>(int op, double a, double b) {
  if (op == 0) return dcp_add(a, b);
  if (op == 3)
    return (dcp_u64)__double_as_longlong(b) > (dcp_u64)__double_as_longlong(a) ? b : a;
  if (op == 2) return (b < a || b != b) ? b : a;
  return (b > a || b != b) ? b : a;
}
// Cross-block combine in the final type (wraps for integer sums).
__device__ __forceinline__ double dcp_fin_comb(int op, double a, double b) {
  if (op == 0) return a + b;
  if (op == 2) return (b < a || b != b) ? b : a;
  return (b > a || b != b) ? b : a;
}
__device__ __forceinline__ long long dcp_fin_comb(int op, long long a, long long b) {
  if (op == 0) return (long long)((dcp_u64)a + (dcp_u64)b);
  if (op == 2) return b < a ? b : a;
  return b > a ? b : a;
}

template <typename T>
__device__ __forceinline__ T dcp_shfl_xor(T v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

// Deterministic block reduction of NRED accumulators followed by the
// one-launch cross-block pass: every block writes its partials, then the
// last block to take a ticket (no waiting: the ticket only tells a block it
// is last) combines all partials in block order and resets the ticket.  The
// result depends only on the grid shape, never on scheduling.
template <typename T, int NRED, int NTHREADS>
__device__ __forceinline__ void dcp_reduce_epilogue(T (&acc)[NRED > 0 ? NRED : 1],
                                                    T* const* red_out,
                                                    typename DcpFin<T>::type* partials,
                                                    unsigned int* ticket) {
  typedef typename DcpFin<T>::type F;
  constexpr int NW = NTHREADS / 32;
  // blocks are numbered over the whole (x, y) grid
  const unsigned int nblk = gridDim.x * gridDim.y;
  const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x;
  __shared__ T s_w[NRED > 0 ? NRED : 1][NW];
  __shared__ F s_f[NRED > 0 ? NRED : 1][NW];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < NRED; ++r) {
    T v = acc[r];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = dcp_red_comb(dcp_red_op(r), v, dcp_shfl_xor(v, m));
    if (lane == 0) s_w[r][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int r = 0; r < NRED; ++r) {
      T v = s_w[r][0];
      for (int w = 1; w < NW; ++w) v = dcp_red_comb(dcp_red_op(r), v, s_w[r][w]);
      partials[(size_t)r * nblk + bid] = (F)v;
    }
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == nblk - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int r = 0; r < NRED; ++r) {
    F v = (F)dcp_red_init<T>(dcp_red_op(r));
    for (unsigned int b = threadIdx.x; b < nblk; b += NTHREADS)
      v = dcp_fin_comb(dcp_red_op(r), v, __ldcg(partials + (size_t)r * nblk + b));
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = dcp_fin_comb(dcp_red_op(r), v, dcp_shfl_xor(v, m));
    if (lane == 0) s_f[r][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int r = 0; r < NRED; ++r) {
      F v = s_f[r][0];
      for (int w = 1; w < NW; ++w) v = dcp_fin_comb(dcp_red_op(r), v, s_f[r][w]);
      red_out[r][0] = (T)v;
    }
    *ticket = 0u;  // ready for the next launch
  }
}

// ---------------------------------------------------------------------------
// 16-byte global accesses with explicit cache behaviour (inline PTX):
// streaming loads that bypass L1 and ask L2 for 256-byte sectors, and
// streaming (evict-first) stores.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 dcp_ld_stream16(const void* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ void dcp_st_stream16(void* p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// Launch parameters of stencil kernels (passed by value).
template <typename T> struct DcpStParamsT {
  const T* ld[DCP_MAXIO];   // first launch: prologue loads; later launches: ld[0] = state
  const T* pld[DCP_MAXIO];  // post loads (last launch)
  T* st[DCP_MAXIO];         // last launch: stores; earlier launches: st[0] = state
  const T* sc[DCP_MAXIO];   // 0-axis operands
  T* red_out[DCP_MAXIO];
  int nz, ny, nx;
  int tiles_x, tiles_y, tiles_z;
  int seg, pad_;            // warp-stream kernels: rows per work item
  typename DcpFin<T>::type* partials;
  unsigned int* ticket;
  unsigned long long* guard;  // first launch of a deferred run: largest |input| seen
};

// The generated stencil sums take their multipliers from registers loaded
// once per thread from the kernel's table dcp_km (DCP_NK entries; values the
// compiler cannot fold into immediates, so each stays a register of its own).
template <typename T, int N>
__device__ __forceinline__ void dcp_load_multipliers(T (&km)[N], const double* tab) {
#pragma unroll
  for (int k = 0; k < N; ++k) km[k] = (T)tab[k];
}

// Bit pattern of an element type (column masks of the warp-stream kernels).
template <typename T> struct DcpBits { typedef unsigned type; };
template <> struct DcpBits<double> { typedef unsigned long long type; };
__device__ __forceinline__ float dcp_keep(float v, unsigned m) {
  return __uint_as_float(__float_as_uint(v) & m);
}
__device__ __forceinline__ double dcp_keep(double v, unsigned long long m) {
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) & m));
}

// Magnitude guard of a deferred common-weight run (DCP_GUARD kernels): the
// largest finite |value| the first launch reads, as the bit pattern with the
// sign cleared (such patterns order like the magnitudes).  Integer work only;
// non-finite inputs are skipped (they propagate the same way in either sum).
struct DcpGuard {
  unsigned long long m;
  __device__ __forceinline__ DcpGuard() : m(0ull) {}
  __device__ __forceinline__ void see(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    if (b < 0x7ff0000000000000ull && b > m) m = b;
  }
  __device__ __forceinline__ void see(float v) {
    const unsigned long long b = __float_as_uint(v) & 0x7fffffffu;
    if (b < 0x7f800000ull && b > m) m = b;
  }
  // one atomic per warp; every lane of the warp must call it
  __device__ __forceinline__ void flush(unsigned long long* dst) {
    unsigned long long v = m;
    for (int o = 16; o >= 1; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(dst, v);
  }
};

// Launch parameters of axis-reduction kernels (passed by value).  The
// iteration space is viewed as (outer, R, inner) with R the reduced axis.
template <typename T> struct DcpAxParamsT {
  const T* ld[DCP_MAXIO];   // prologue loads (full iteration space)
  const T* sc[DCP_MAXIO];   // 0-axis operands
  T* out[DCP_MAXIO];        // one output of outer * inner elements per reduction
  typename DcpFin<T>::type* partials;  // [NRED][S][outer * inner] when S > 1
  unsigned int* tickets;    // one per block tile (S > 1)
  long long outer, R, inner;
  long long rchunk;         // elements of R per split
  long long ntiles;         // tiles of TI along inner
  int TO, TI, TR, S;        // threads along outer / inner / R (powers of 2), R splits
};

template <typename T, int VEC> union DcpPack {
  uint4 u;
  T t[VEC];
};
