// k_stencil2d_stream.cuh -- register-resident, warp-streamed time tiling of
// a 1-D / 2-D iterated stencil (zero or fixed-ring boundary).
//
// A warp owns a strip of 32*C consecutive columns (C per lane) and streams
// down the rows of its strip.  The DCP_NSTEPS steps of one launch are kept as
// a pipeline of time levels in registers: when input row j arrives (level 0),
// level l computes row j - l*RY from the 2*RY+1 most recent rows of level
// l-1, so each row passes through all levels while it is in registers.
// Neighbours along x come from the adjacent lanes by warp shuffles; the strip
// loses RX columns of validity per level at each edge, so a warp writes
// W = 32*C - 2*NSTEPS*RX columns.  There is no shared memory and no barrier
// inside the stream; device memory is read once (plus the strip overlap) and
// written once per NSTEPS steps.
//
// Work items are (array, strip, row segment); a segment streams its rows plus
// NSTEPS*RY warm-up rows above it.  Warps stride through the items (items of
// the largest arrays first in batched launches).
//
// The generated prefix defines DCP_T, DCP_C, DCP_RX, DCP_RY, DCP_NSTEPS,
// DCP_BC, DCP_THREADS, DCP_KNAME, DCP_BATCH, DCP_LAST, DCP_PDM, DCP_GUARD, DCP_MINB,
// DCP_NSTORE, DCP_NRED, DCP_NSCALAR, dcp_red_op(r) and
//   T    dcp_input(const DcpStParams& p, const T* sc, long long i)   (prologue)
//   void dcp_level<L>(const T (&up)[NR][C], const T (&lf)[NR][RX], const T (&rt)[NR][RX],
//                     T (&out)[C], const T (&km)[DCP_NK])   weighted sum of step L
//                     (rows up[RY+dy]; km: its multipliers, see dcp_load_multipliers),
//   T    dcp_epi<L>(T v)                 epilogue maps fused after step L
//   bool dcp_uses_lf(int L, int d), dcp_uses_rt(int L, int d)   (constexpr)
//        whether step L reads a left / right neighbour column in row d
//   void dcp_post(const DcpStParams& p, const T* sc, long long i, T v, T* st, T* rv)
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)
#ifndef DCP_MINB
#define DCP_MINB 1   // CTAs per SM the compiler's register budget must allow
#endif

#define DCP_BC_ZERO 0
#define DCP_BC_PERIODIC 1
#define DCP_BC_FIXED_RING 2

constexpr int NR = 2 * DCP_RY + 1;                 // rows kept per level
constexpr int K = DCP_NSTEPS;
constexpr int C = DCP_C;
constexpr int SPAN = 32 * C;                       // columns held by a warp
constexpr int W = SPAN - 2 * K * DCP_RX;           // columns written by a warp
static_assert(W > 0, "strip too narrow for the number of steps");
constexpr int RXA = DCP_RX > 0 ? DCP_RX : 1;

typedef DcpStParamsT<T> DcpStParams;

__device__ __forceinline__ constexpr int dcp_mod(int a, int m) { return ((a % m) + m) % m; }

// One array (or instance) and the part of it a work item covers.
struct DcpItem {
  const T* in;   // batched: instance input; single: unused (dcp_input reads p.ld)
  T* out;        // batched: instance output
  int ny, nx;
  int x0;        // first written column
  int y0, y1;    // rows written
};

// The lane's columns in a work item: the first one, and per column a bit
// mask that keeps a value (all ones: the column lies inside the array) or
// clears it to +0 (outside), computed once per item.
struct DcpCols {
  int col0;
  typename DcpBits<T>::type keep[C];
  T km[DCP_NK];  // multipliers of the sums (see dcp_load_multipliers)
};

// CHECK: the strip reaches outside the array (per-column tests).  ROWS: every
// row touched by this iteration lies inside the array and outside a fixed
// ring (no row tests).
template <int L, int P, bool CHECK, bool ROWS>
__device__ __forceinline__ void dcp_level_step(T (&ring)[K > 1 ? K : 1][NR][C], int j,
                                               const DcpItem& it, const DcpCols& cols,
                                               T (&outv)[C],
                                               bool& out_ok) {
  // level L (1-based) computes row y = j - L*RY from level L-1
  constexpr int l = L - 1;  // source level
  const int y = j - L * DCP_RY;
  T up[NR][C];
#pragma unroll
  for (int d = 0; d < NR; ++d)
#pragma unroll
    for (int c = 0; c < C; ++c) up[d][c] = ring[l][dcp_mod(P - L * DCP_RY + d - DCP_RY, NR)][c];
  // neighbour columns from the adjacent lanes, only for the rows the step
  // reads off-centre
  T lf[NR][RXA], rt[NR][RXA];
#pragma unroll
  for (int d = 0; d < NR; ++d)
#pragma unroll
    for (int q = 0; q < RXA; ++q) lf[d][q] = rt[d][q] = (T)0;
#pragma unroll
  for (int d = 0; d < NR; ++d)
#pragma unroll
    for (int q = 0; q < DCP_RX; ++q) {
      if (dcp_uses_lf(L - 1, d))
        lf[d][DCP_RX - 1 - q] = __shfl_up_sync(0xffffffffu, up[d][C - 1 - q], 1);
      if (dcp_uses_rt(L - 1, d)) rt[d][q] = __shfl_down_sync(0xffffffffu, up[d][q], 1);
    }
  T v[C];
  dcp_level<L - 1>(up, lf, rt, v, cols.km);
  const bool row_in = ROWS || (unsigned)y < (unsigned)it.ny;
  if (!CHECK) {
    // every column of the strip lies inside the array (and outside a fixed
    // ring): only the row, uniform across the warp, needs a test
    const bool ring_row =
        !ROWS && DCP_BC == DCP_BC_FIXED_RING && (y < DCP_RY || y >= it.ny - DCP_RY);
    if (!row_in) {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = (T)0;
    } else if (ring_row) {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = dcp_epi<L - 1>(up[DCP_RY][c]);
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = dcp_epi<L - 1>(v[c]);
    }
  } else if (DCP_BC == DCP_BC_ZERO) {
    // columns outside the array read as ghost zeros at every level: the
    // item's bit masks clear them (one bitwise AND per column, and exact for
    // any value the epilogue leaves there, NaN included)
    if (!row_in) {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = (T)0;
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) v[c] = dcp_keep(dcp_epi<L - 1>(v[c]), cols.keep[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int col = cols.col0 + c;
      const bool in = row_in && (unsigned)col < (unsigned)it.nx;
      T r;
      if (!in) {
        r = (T)0;
      } else if (DCP_BC == DCP_BC_FIXED_RING &&
                 ((!ROWS && (y < DCP_RY || y >= it.ny - DCP_RY)) || col < DCP_RX ||
                  col >= it.nx - DCP_RX)) {
        r = dcp_epi<L - 1>(up[DCP_RY][c]);  // ring cell keeps its value; epilogue still applies
      } else {
        r = dcp_epi<L - 1>(v[c]);
      }
      v[c] = r;
    }
  }
  if constexpr (L < K) {
#pragma unroll
    for (int c = 0; c < C; ++c) ring[L][dcp_mod(P - L * DCP_RY, NR)][c] = v[c];
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) outv[c] = v[c];
    out_ok = row_in;
  }
}

template <int L, int P, bool CHECK, bool ROWS>
__device__ __forceinline__ void dcp_levels(T (&ring)[K > 1 ? K : 1][NR][C], int j,
                                           const DcpItem& it, const DcpCols& cols,
                                           T (&outv)[C],
                                           bool& out_ok) {
  if constexpr (L <= K) {
    dcp_level_step<L, P, CHECK, ROWS>(ring, j, it, cols, outv, out_ok);
    dcp_levels<L + 1, P, CHECK, ROWS>(ring, j, it, cols, outv, out_ok);
  }
}

// Input rows in flight.  Row j lives in queue slot j mod PD and in ring slot
// j mod NR; PD is a multiple of NR and iterations are unrolled by PD, so both
// are compile-time constants and no register holding an outstanding load is
// ever moved.  DCP_PDM row windows are requested ahead.
constexpr int PD = NR * (NR > 1 ? DCP_PDM : 2 * DCP_PDM);

template <bool CHECK, bool ROWS, class Input>
__device__ __forceinline__ void dcp_fetch_row(T (&dst)[C], int j, const DcpItem& it,
                                              const DcpCols& cols,
                                              Input& input) {
  const long long base = (long long)j * it.nx + cols.col0;
  const bool row_ok = ROWS || (unsigned)j < (unsigned)it.ny;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const bool ok = row_ok && (!CHECK || (unsigned)(cols.col0 + c) < (unsigned)it.nx);
    dst[c] = ok ? input(base + c) : (T)0;
  }
}

// One stream iteration: input row j, P = j mod PD.  Row j + PD is requested
// into the slot row j vacates before the levels are computed, so its load
// latency overlaps PD iterations of arithmetic.
template <int P, bool CHECK, bool ROWS, class Input, class Output>
__device__ __forceinline__ void dcp_iter(T (&ring)[K > 1 ? K : 1][NR][C], T (&q)[PD][C], int j,
                                         const DcpItem& it, const DcpCols& cols, Input& input,
                                         Output& output, DcpGuard& guard) {
#pragma unroll
  for (int c = 0; c < C; ++c) {
    ring[0][P % NR][c] = q[P][c];
    if (DCP_GUARD) guard.see(q[P][c]);  // arrived: requested PD iterations ago
  }
  dcp_fetch_row<CHECK, ROWS>(q[P], j + PD, it, cols, input);
  T outv[C];
  bool out_ok = false;
  dcp_levels<1, P % NR, CHECK, ROWS>(ring, j, it, cols, outv, out_ok);
  const int y = j - K * DCP_RY;
  if (ROWS || (out_ok && y >= it.y0 && y < it.y1)) output(y, outv);
}

// Iterations j .. j + (PD - P) - 1 with phases P .. PD-1.
template <int P, bool CHECK, bool ROWS, class Input, class Output>
__device__ __forceinline__ void dcp_iters(T (&ring)[K > 1 ? K : 1][NR][C], T (&q)[PD][C], int j,
                                          const DcpItem& it, const DcpCols& cols, Input& input,
                                          Output& output, DcpGuard& guard) {
  if constexpr (P < PD) {
    dcp_iter<P, CHECK, ROWS>(ring, q, j, it, cols, input, output, guard);
    dcp_iters<P + 1, CHECK, ROWS>(ring, q, j + 1, it, cols, input, output, guard);
  }
}

// A single iteration of run-time phase r (alignment and tail), rows tested.
template <int P, bool CHECK, class Input, class Output>
__device__ __forceinline__ void dcp_iter_dyn(int r, T (&ring)[K > 1 ? K : 1][NR][C],
                                             T (&q)[PD][C], int j, const DcpItem& it,
                                             const DcpCols& cols,
                                             Input& input, Output& output, DcpGuard& guard) {
  if constexpr (P < PD) {
    if (r == P) dcp_iter<P, CHECK, false>(ring, q, j, it, cols, input, output, guard);
    else dcp_iter_dyn<P + 1, CHECK>(r, ring, q, j, it, cols, input, output, guard);
  }
}

template <int P, bool CHECK, class Input>
__device__ __forceinline__ void dcp_prefill(T (&q)[PD][C], int j0, const DcpItem& it,
                                            const DcpCols& cols,
                                            Input& input) {
  if constexpr (P < PD) {
    // the row in [j0, j0 + PD) that maps to slot P
    dcp_fetch_row<CHECK, false>(q[P], j0 + dcp_mod(P - j0, PD), it, cols, input);
    dcp_prefill<P + 1, CHECK>(q, j0, it, cols, input);
  }
}

template <bool CHECK, class Input, class Output>
__device__ __forceinline__ void dcp_stream_impl(const DcpItem& it, Input& input, Output& output,
                                                DcpGuard& guard, const T (&km)[DCP_NK]) {
  const int lane = threadIdx.x & 31;
  DcpCols cols;
#pragma unroll
  for (int k = 0; k < DCP_NK; ++k) cols.km[k] = km[k];
  cols.col0 = it.x0 - K * DCP_RX + lane * C;
#pragma unroll
  for (int c = 0; c < C; ++c)
    cols.keep[c] = (unsigned)(cols.col0 + c) < (unsigned)it.nx ? ~(typename DcpBits<T>::type)0 : 0;
  T ring[K > 1 ? K : 1][NR][C];
#pragma unroll
  for (int l = 0; l < (K > 1 ? K : 1); ++l)
#pragma unroll
    for (int d = 0; d < NR; ++d)
#pragma unroll
      for (int c = 0; c < C; ++c) ring[l][d][c] = (T)0;
  // Rows before the first streamed row hold zeros: exact ghosts above the
  // array; inside the array they only feed warm-up rows that are never written.
  int j = it.y0 - K * DCP_RY;
  const int jend = it.y1 + K * DCP_RY;
  T q[PD][C];
  dcp_prefill<0, CHECK>(q, j, it, cols, input);
  // Iterations [jb0, jb1) touch only rows inside the array (and outside a
  // fixed ring): level rows j - L*RY for L = 1..K, the fetched row j + PD and
  // the written row j - K*RY in [y0, y1).  They run without row tests.
  // One loop with one call site per form keeps the unrolled code small:
  // PD-aligned groups inside [jb0, jb1) take the unchecked form, every other
  // iteration (warm-up, alignment, tail) the row-checked one.
  const int ring_w = DCP_BC == DCP_BC_FIXED_RING ? DCP_RY : 0;
  const int jb0 = K * DCP_RY + max(it.y0, ring_w);
  const int jb1 = min(min(it.y1 + K * DCP_RY, it.ny - ring_w + DCP_RY), it.ny - PD);
  while (j < jend) {
    if (j >= jb0 && j + PD <= jb1 && dcp_mod(j, PD) == 0) {
      dcp_iters<0, CHECK, true>(ring, q, j, it, cols, input, output, guard);
      j += PD;
    } else {
      dcp_iter_dyn<0, CHECK>(dcp_mod(j, PD), ring, q, j, it, cols, input, output, guard);
      ++j;
    }
  }
}

// Strips whose columns all lie inside the array (outside a fixed ring) take
// the path without per-column boundary tests.
// With DCP_GUARD every row the stream reads enters the magnitude guard.
template <class Input, class Output>
__device__ __forceinline__ void dcp_stream(const DcpItem& it, Input&& input, DcpGuard& guard,
                                           const T (&km)[DCP_NK], Output&& output) {
  const int lo = DCP_BC == DCP_BC_FIXED_RING ? DCP_RX : 0;
  const int first = it.x0 - K * DCP_RX;
  if (first >= lo && first + SPAN <= it.nx - lo)
    dcp_stream_impl<false>(it, input, output, guard, km);
  else
    dcp_stream_impl<true>(it, input, output, guard, km);
}

#if !DCP_BATCH
// Single array: items = strips x row segments of p.seg rows.
extern "C" __global__ void __launch_bounds__(DCP_THREADS, DCP_MINB) DCP_KNAME(const DcpStParams p) {
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
  T acc[DCP_ARR(DCP_NRED)];
#pragma unroll
  for (int r = 0; r < DCP_NRED; ++r) acc[r] = dcp_red_init<T>(dcp_red_op(r));
  const int ny = p.ny, nx = p.nx;
  const int strips = (nx + W - 1) / W;
  const int SEG = p.seg > 0 ? p.seg : ny;
  const int segs = (ny + SEG - 1) / SEG;
  const int items = strips * segs;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * DCP_THREADS + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * DCP_THREADS) >> 5;
  DcpGuard guard;
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
  for (int w = warp; w < items; w += nwarps) {
    const int sg = w / strips, st = w - sg * strips;
    DcpItem it{nullptr, nullptr, ny, nx, st * W, sg * SEG, min(ny, (sg + 1) * SEG)};
    const int col0 = it.x0 - K * DCP_RX + lane * C;
    dcp_stream(
        it,
        [&](long long gi) { return dcp_input(p, sc, gi); }, guard, km,
        [&](int y, const T (&v)[C]) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int col = col0 + c;
            if (col < it.x0 || col >= it.x0 + W || col >= nx) continue;
            const long long gi = (long long)y * nx + col;
#if DCP_LAST
            T stv[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
            dcp_post(p, sc, gi, v[c], stv, rv);
#pragma unroll
            for (int s = 0; s < DCP_NSTORE; ++s) p.st[s][gi] = stv[s];
#pragma unroll
            for (int r = 0; r < DCP_NRED; ++r)
              acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
#else
            p.st[0][gi] = v[c];
#endif
          }
        });
  }
#if DCP_LAST && DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
#if DCP_GUARD
  guard.flush(p.guard);
#endif
}
#else
// Batched form: items are (instance, strip, row segment); instances are
// ordered largest first by the host; the item of warp w is found by binary
// search over the instances' first item numbers.
struct DcpInst {
  const T* in;
  T* out;
  int ny, nx, tiles_x, tile0;  // tiles_x = strips of the instance, tile0 = its first item
};
struct DcpBatchParams {
  const DcpInst* inst;
  int ninst;
  int total_tiles;
  int seg;   // rows per work item
  int pad_;
  unsigned long long* guard;  // first launch of a deferred run: largest |input| seen
};

extern "C" __global__ void __launch_bounds__(DCP_THREADS, DCP_MINB) DCP_KNAME(const DcpBatchParams p) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * DCP_THREADS + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * DCP_THREADS) >> 5;
  DcpGuard guard;
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
  for (int w = warp; w < p.total_tiles; w += nwarps) {
    int lo = 0, hi = p.ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.inst[mid].tile0 <= w) lo = mid;
      else hi = mid - 1;
    }
    const DcpInst I = p.inst[lo];
    const int t = w - I.tile0;
    const int sg = t / I.tiles_x, st = t - sg * I.tiles_x;
    DcpItem it{I.in, I.out, I.ny, I.nx, st * W, sg * p.seg, min(I.ny, (sg + 1) * p.seg)};
    const T* in = I.in;
    T* out = I.out;
    const int col0 = it.x0 - K * DCP_RX + lane * C;
    dcp_stream(
        it,
        [&](long long gi) { return in[gi]; }, guard, km,
        [&](int y, const T (&v)[C]) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const int col = col0 + c;
            if (col < it.x0 || col >= it.x0 + W || col >= it.nx) continue;
            out[(long long)y * it.nx + col] = v[c];
          }
        });
  }
#if DCP_GUARD
  guard.flush(p.guard);
#endif
}
#endif
