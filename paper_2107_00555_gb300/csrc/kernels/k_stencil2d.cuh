// k_stencil2d.cuh -- skeleton of a time-tiled 1-D / 2-D iterated stencil
// (the jacobi programs of Sec. 2.2 and Sec. 4.3).  One CTA owns a
// DCP_TY x DCP_TX output tile; it stages the tile plus a halo of
// DCP_NSTEPS * radius cells in shared memory once, applies DCP_NSTEPS
// Jacobi steps there (ping-pong between two shared buffers, the valid region
// shrinking by one radius per step: overlapped time tiling), and writes the
// centre once.  Device memory is therefore read and written once per
// DCP_NSTEPS steps instead of once per step.
//
// Boundary rules (applied at every step, so out-of-array cells inside the
// halo stay exact):  ZERO -- cells outside the array are 0;  PERIODIC --
// halo cells are wrapped copies and evolve like the cells they copy;
// FIXED_RING -- ring cells keep their value.
//
// The generated prefix defines DCP_T, DCP_TX, DCP_TY, DCP_RX, DCP_RY,
// DCP_NSTEPS, DCP_BC, DCP_THREADS, DCP_KNAME, DCP_BATCH, DCP_LAST, DCP_GUARD,
// DCP_NLOAD, DCP_NPLOAD, DCP_NSTORE, DCP_NSCALAR, DCP_NRED,
// dcp_red_op(r) and the functions
//   T    dcp_input(const DcpStParams& p, const T* sc, long long i)  (prologue)
//   T    dcp_sum<S>(const T* A, int c, const T (&km)[DCP_NK])   weighted sum of step S
//        at tile cell c (km: its multipliers, see dcp_load_multipliers)
//   T    dcp_epi<S>(T v)                 epilogue maps fused after step S
//   void dcp_post(const DcpStParams& p, const T* sc, long long i, T v, T* st, T* rv)
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)

#define DCP_BC_ZERO 0
#define DCP_BC_PERIODIC 1
#define DCP_BC_FIXED_RING 2

constexpr int DCP_HX = DCP_NSTEPS * DCP_RX;
constexpr int DCP_HY = DCP_NSTEPS * DCP_RY;
constexpr int DCP_PW = DCP_TX + 2 * DCP_HX;   // shared tile pitch
constexpr int DCP_PH = DCP_TY + 2 * DCP_HY;
constexpr int DCP_TILE_ELEMS = DCP_PW * DCP_PH;

typedef DcpStParamsT<T> DcpStParams;

__device__ __forceinline__ int dcp_wrap(int q, int n) {
  if ((unsigned)q < (unsigned)n) return q;
  int r = q % n;
  return r < 0 ? r + n : r;
}

// One step over the region that is still valid after S+1 steps.  Tiles
// whose region lies where the step needs no boundary treatment (inside the
// array, outside the fixed ring; always under PERIODIC, whose halo holds
// wrapped copies) take the fast path: each work item is R consecutive rows of
// one column, all loads are issued before any store, so the R weighted sums
// share the shared-memory loads of their common neighbours.  Other tiles take
// the checked path, one cell per work item.
template <int S>
__device__ __forceinline__ void dcp_run_step(const T* __restrict__ A, T* __restrict__ B, int y0,
                                             int x0, int ny, int nx,
                                             const T (&km)[DCP_NK]) {
  constexpr int my = (S + 1) * DCP_RY, mx = (S + 1) * DCP_RX;
  constexpr int RH = DCP_PH - 2 * my, RW = DCP_PW - 2 * mx;
  constexpr int R = (RH % 4 == 0) ? 4 : ((RH % 2 == 0) ? 2 : 1);
  constexpr int NB = RH / R;
  const int ry0 = y0 + my, rx0 = x0 + mx;  // global coordinates of the region's corner
  bool fast;
  if (DCP_BC == DCP_BC_PERIODIC) {
    fast = true;
  } else {
    const int lo_y = DCP_BC == DCP_BC_FIXED_RING ? DCP_RY : 0;
    const int lo_x = DCP_BC == DCP_BC_FIXED_RING ? DCP_RX : 0;
    fast = ry0 >= lo_y && ry0 + RH <= ny - lo_y && rx0 >= lo_x && rx0 + RW <= nx - lo_x;
  }
  if (fast) {
    for (int i = threadIdx.x; i < NB * RW; i += DCP_THREADS) {
      const int rb = i / RW, lx = mx + (i - rb * RW);
      const int c0 = (my + rb * R) * DCP_PW + lx;
      T v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = dcp_sum<S>(A, c0 + r * DCP_PW, km);
#pragma unroll
      for (int r = 0; r < R; ++r) B[c0 + r * DCP_PW] = dcp_epi<S>(v[r]);
    }
    return;
  }
  for (int i = threadIdx.x; i < RH * RW; i += DCP_THREADS) {
    const int ly = my + i / RW, lx = mx + i % RW;
    const int c = ly * DCP_PW + lx;
    const int gy = y0 + ly, gx = x0 + lx;
    T v;
    const bool inside = (unsigned)gy < (unsigned)ny && (unsigned)gx < (unsigned)nx;
    if (DCP_BC != DCP_BC_PERIODIC && !inside) {
      v = (T)0;
    } else if (DCP_BC == DCP_BC_FIXED_RING &&
               (gy < DCP_RY || gy >= ny - DCP_RY || gx < DCP_RX || gx >= nx - DCP_RX)) {
      v = dcp_epi<S>(A[c]);  // ring cell keeps its value; the step's epilogue still applies
    } else {
      v = dcp_epi<S>(dcp_sum<S>(A, c, km));
    }
    B[c] = v;
  }
}

template <int S>
__device__ __forceinline__ void dcp_steps(T*& A, T*& B, int y0, int x0, int ny, int nx,
                                          const T (&km)[DCP_NK]) {
  if constexpr (S < DCP_NSTEPS) {
    dcp_run_step<S>(A, B, y0, x0, ny, nx, km);
    __syncthreads();
    T* t = A;
    A = B;
    B = t;
    dcp_steps<S + 1>(A, B, y0, x0, ny, nx, km);
  }
}

// Stage tile (tyi, txi) of an ny x nx array with its halo into A, read
// through `input(flat index)`, and run this launch's steps; on return A
// holds the tile after DCP_NSTEPS steps.
template <class Input>
__device__ __forceinline__ void dcp_tile(T*& A, T*& B, int ny, int nx, int tyi, int txi,
                                         const T (&km)[DCP_NK], Input input) {
  const int y0 = tyi * DCP_TY - DCP_HY, x0 = txi * DCP_TX - DCP_HX;
  for (int i = threadIdx.x; i < DCP_TILE_ELEMS; i += DCP_THREADS) {
    const int ly = i / DCP_PW, lx = i - ly * DCP_PW;
    int gy = y0 + ly, gx = x0 + lx;
    T v = (T)0;
    const bool inside = (unsigned)gy < (unsigned)ny && (unsigned)gx < (unsigned)nx;
    if (DCP_BC == DCP_BC_PERIODIC) {
      gy = dcp_wrap(gy, ny);
      gx = dcp_wrap(gx, nx);
      v = input((long long)gy * nx + gx);
    } else if (inside) {
      v = input((long long)gy * nx + gx);
    }
    A[i] = v;
  }
  __syncthreads();
  dcp_steps<0>(A, B, y0, x0, ny, nx, km);
}

#if !DCP_BATCH
extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpStParams p) {
  extern __shared__ __align__(16) unsigned char dcp_smem[];
  T* A = reinterpret_cast<T*>(dcp_smem);
  T* B = A + DCP_TILE_ELEMS;
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
  const int ny = p.ny, nx = p.nx;
  const int tyi = blockIdx.x / p.tiles_x, txi = blockIdx.x - tyi * p.tiles_x;
  DcpGuard guard;
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
  dcp_tile(A, B, ny, nx, tyi, txi, km, [&](long long gi) {
    const T v = dcp_input(p, sc, gi);
    if (DCP_GUARD) guard.see(v);
    return v;
  });

  // Write the tile centre (last launch: post maps, stores and reductions).
  T acc[DCP_ARR(DCP_NRED)];
#pragma unroll
  for (int r = 0; r < DCP_NRED; ++r) acc[r] = dcp_red_init<T>(dcp_red_op(r));
  for (int i = threadIdx.x; i < DCP_TX * DCP_TY; i += DCP_THREADS) {
    const int ty = i / DCP_TX, tx = i - ty * DCP_TX;
    const int gy = tyi * DCP_TY + ty, gx = txi * DCP_TX + tx;
    if (gy >= ny || gx >= nx) continue;
    const long long gi = (long long)gy * nx + gx;
    const T v = A[(ty + DCP_HY) * DCP_PW + tx + DCP_HX];
#if DCP_LAST
    T st[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
    dcp_post(p, sc, gi, v, st, rv);
#pragma unroll
    for (int s = 0; s < DCP_NSTORE; ++s) p.st[s][gi] = st[s];
#pragma unroll
    for (int r = 0; r < DCP_NRED; ++r)
      acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
#else
    p.st[0][gi] = v;
#endif
  }
#if DCP_LAST && DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
#if DCP_GUARD
  guard.flush(p.guard);
#endif
}
#else
// Batched form: many independent arrays (instances) run the same step
// program in one persistent launch.  Work items are (instance, tile) pairs
// numbered instance by instance; CTAs stride through them (instances are
// ordered largest first by the host, so the tail of the launch is made of
// small tiles).  The instance of work item w is found by binary search over
// the first-tile numbers.
struct DcpInst {
  const T* in;
  T* out;
  int ny, nx, tiles_x, tile0;
};
struct DcpBatchParams {
  const DcpInst* inst;
  int ninst;
  int total_tiles;
  int seg;   // unused by the tile form
  int pad_;
  unsigned long long* guard;  // first launch of a deferred run: largest |input| seen
};

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpBatchParams p) {
  extern __shared__ __align__(16) unsigned char dcp_smem[];
  DcpGuard guard;
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
  for (int w = blockIdx.x; w < p.total_tiles; w += gridDim.x) {
    int lo = 0, hi = p.ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.inst[mid].tile0 <= w) lo = mid;
      else hi = mid - 1;
    }
    const DcpInst I = p.inst[lo];
    const int t = w - I.tile0;
    const int tyi = t / I.tiles_x, txi = t - tyi * I.tiles_x;
    T* A = reinterpret_cast<T*>(dcp_smem);
    T* B = A + DCP_TILE_ELEMS;
    const T* in = I.in;
    dcp_tile(A, B, I.ny, I.nx, tyi, txi, km, [&](long long gi) {
      const T v = in[gi];
      if (DCP_GUARD) guard.see(v);
      return v;
    });
    for (int i = threadIdx.x; i < DCP_TX * DCP_TY; i += DCP_THREADS) {
      const int ty = i / DCP_TX, tx = i - ty * DCP_TX;
      const int gy = tyi * DCP_TY + ty, gx = txi * DCP_TX + tx;
      if (gy >= I.ny || gx >= I.nx) continue;
      I.out[(long long)gy * I.nx + gx] = A[(ty + DCP_HY) * DCP_PW + tx + DCP_HX];
    }
    __syncthreads();  // the next work item overwrites the shared tile
  }
#if DCP_GUARD
  guard.flush(p.guard);
#endif
}
#endif
