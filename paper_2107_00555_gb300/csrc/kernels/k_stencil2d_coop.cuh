// k_stencil2d_coop.cuh -- skeleton of an iterated 1-D / 2-D stencil whose
// every step runs in ONE persistent launch, for arrays small enough that one
// tile per resident CTA covers them (the 256 x 256 jacobi step: 152 tiles).
//
// Each CTA keeps its tile plus a halo of one radius in shared memory for the
// whole run.  Between steps only neighbouring tiles synchronise: after step
// s a CTA writes the cells its neighbours read (its tile's border ring, one
// radius wide) to an exchange array in device memory and publishes s + 1 in
// its flag; before the border cells of step s + 1 it waits for the flags of
// the (up to 8) tiles its halo overlaps and reads their rings.  The tile's
// interior cells of a step are computed before that wait, so the exchange
// latency overlaps arithmetic.  No halo is recomputed (unlike time tiling,
// whose halo grows by a radius per step), and no kernel boundary separates
// the steps.
//
// The launch is cooperative (every CTA resident at once, so a wait on a
// neighbour always ends); each wait is still bounded: after DCP_SPIN_LIMIT
// polls it records an error word the host reports (DCP_E_TIMEOUT) and goes
// on.  Flags carry a per-launch epoch read from a device counter that the
// last CTA of the launch to finish advances, so no flag is reset between
// launches (and a captured graph replays correctly).
//
// Per step the arithmetic is that of the tile kernel (dcp_sum<S> in point
// order, dcp_epi<S>), so every kernel form computes the same bits.
//
// The generated prefix defines DCP_T, DCP_TX, DCP_TY, DCP_RX, DCP_RY,
// DCP_NSTEPS, DCP_BC, DCP_THREADS, DCP_KNAME, DCP_GUARD, DCP_NSTORE,
// DCP_NRED, DCP_NSCALAR, dcp_red_op(r), the multiplier table and
//   T    dcp_input(const DcpStParams& p, const T* sc, long long i)  (prologue)
//   T    dcp_sum<S>(const T* A, int c, const T (&km)[DCP_NK])   (pitch DCP_PW)
//   T    dcp_epi<S>(T v)
//   void dcp_post(const DcpStParams& p, const T* sc, long long i, T v, T* st, T* rv)
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)

#define DCP_BC_ZERO 0
#define DCP_BC_PERIODIC 1
#define DCP_BC_FIXED_RING 2

constexpr int DCP_PW = DCP_TX + 2 * DCP_RX;  // shared tile pitch
constexpr int DCP_PH = DCP_TY + 2 * DCP_RY;
constexpr int DCP_TILE_ELEMS = DCP_PW * DCP_PH;
constexpr int DCP_SIDE = 2 * DCP_RX > 0 ? 2 * DCP_RX : 1;  // side cells per row (divisor)
#ifndef DCP_SPIN_LIMIT
#define DCP_SPIN_LIMIT (1 << 22)
#endif
#ifndef DCP_WAIT_SKEW
#define DCP_WAIT_SKEW 0u  // test hook: > 0 makes every wait's target unreachable
#endif

typedef DcpStParamsT<T> DcpStParams;

struct DcpCoopParams {
  DcpStParams s;
  T* xb[2];               // exchange arrays (ny x nx): border rings of step parity 0 / 1
  unsigned int* flags;    // one per tile: epoch * 64 + steps published
  unsigned int* ctr;      // [0] epoch, [1] CTAs finished in this launch
  unsigned int* err;      // set when a wait gave up
};

__device__ __forceinline__ int dcp_wrap(int q, int n) {
  if ((unsigned)q < (unsigned)n) return q;
  int r = q % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ unsigned dcp_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void dcp_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Cell (ly, lx) of the shared tile (halo included) at step S: the weighted
// sum and epilogue, or, under the fixed ring, the ring cell's own value
// (epilogue applied); cells outside the array stay 0 (zero and fixed-ring
// boundaries never write them).
template <int S>
__device__ __forceinline__ void dcp_cell(const T* __restrict__ A, T* __restrict__ B, int ly, int lx,
                                         int gy, int gx, int ny, int nx,
                                         const T (&km)[DCP_NK]) {
  const int c = ly * DCP_PW + lx;
  T v;
  if (DCP_BC == DCP_BC_FIXED_RING &&
      (gy < DCP_RY || gy >= ny - DCP_RY || gx < DCP_RX || gx >= nx - DCP_RX)) {
    v = dcp_epi<S>(A[c]);
  } else {
    v = dcp_epi<S>(dcp_sum<S>(A, c, km));
  }
  B[c] = v;
}

// Border cell i (0 <= i < h w - interior) of an h x w tile whose interior
// (cells at least a radius from every edge) is ih x iw: the top RY rows, the
// bottom RY rows, then the RX cells at each side of the rows between.
__device__ __forceinline__ void dcp_border_cell(int i, int h, int w, int ih, int iw, int& ty,
                                                int& tx) {
  const bool has_int = ih > 0 && iw > 0;
  const int top = has_int ? DCP_RY * w : h * w;
  if (i < top) {
    ty = i / w;
    tx = i - ty * w;
  } else if (has_int && i < 2 * top) {
    const int j = i - top;
    ty = h - DCP_RY + j / w;
    tx = j % w;
  } else {
    const int j = i - 2 * top, r = j / DCP_SIDE, k = j - r * DCP_SIDE;
    ty = DCP_RY + r;
    tx = k < DCP_RX ? k : w - 2 * DCP_RX + k;
  }
}

template <int S>
__device__ __forceinline__ void dcp_coop_steps(const DcpCoopParams& q, T*& A, T*& B, int tyi, int txi,
                                               int h, int w, unsigned epoch,
                                               const T (&km)[DCP_NK]) {
  if constexpr (S < DCP_NSTEPS) {
    const int ny = q.s.ny, nx = q.s.nx;
    const int y0 = tyi * DCP_TY, x0 = txi * DCP_TX;
    // interior: cells whose reads stay inside the tile
    const int ih = h - 2 * DCP_RY, iw = w - 2 * DCP_RX;
    if (ih > 0 && iw > 0)
      for (int i = threadIdx.x; i < ih * iw; i += DCP_THREADS) {
        const int ty = DCP_RY + i / iw, tx = DCP_RX + i % iw;
        dcp_cell<S>(A, B, DCP_RY + ty, DCP_RX + tx, y0 + ty, x0 + tx, ny, nx, km);
      }
    if (S > 0) {
      // wait for the neighbours' step S states, then read their border rings
      const int nb = threadIdx.x;
      if (nb < 9 && nb != 4) {
        const int dy = nb / 3 - 1, dx = nb % 3 - 1;
        int ny_t = tyi + dy, nx_t = txi + dx;
        bool exists = true;
        if (DCP_BC == DCP_BC_PERIODIC) {
          ny_t = dcp_wrap(ny_t, q.s.tiles_y);
          nx_t = dcp_wrap(nx_t, q.s.tiles_x);
        } else {
          exists = (unsigned)ny_t < (unsigned)q.s.tiles_y && (unsigned)nx_t < (unsigned)q.s.tiles_x;
        }
        if ((DCP_RY == 0 && dy != 0) || (DCP_RX == 0 && dx != 0)) exists = false;
        if (exists && !(ny_t == tyi && nx_t == txi)) {
          const unsigned* f = q.flags + (ny_t * q.s.tiles_x + nx_t);
          const unsigned target = epoch * 64u + (unsigned)S + DCP_WAIT_SKEW;
          int spins = 0;
          while ((int)(dcp_ld_acquire(f) - target) < 0) {
            if (++spins > DCP_SPIN_LIMIT) {
              atomicOr(q.err, 1u);
              break;
            }
            __nanosleep(32);
          }
        }
      }
      __syncthreads();
      const T* __restrict__ X = q.xb[S & 1];
      // halo ring of the shared tile: rows [0, RY) and [RY + h, 2 RY + h),
      // and the side columns of the rows between
      const int HW = w + 2 * DCP_RX;
      const int nring = 2 * DCP_RY * HW + 2 * DCP_RX * h;
      for (int i = threadIdx.x; i < nring; i += DCP_THREADS) {
        int ly, lx;
        if (i < 2 * DCP_RY * HW) {
          const int r = i / HW;
          ly = r < DCP_RY ? r : h + r;
          lx = i - r * HW;
        } else {
          const int j = i - 2 * DCP_RY * HW, r = j / DCP_SIDE, k = j - r * DCP_SIDE;
          ly = DCP_RY + r;
          lx = k < DCP_RX ? k : w + k;
        }
        int gy = y0 - DCP_RY + ly, gx = x0 - DCP_RX + lx;
        if (DCP_BC == DCP_BC_PERIODIC) {
          gy = dcp_wrap(gy, ny);
          gx = dcp_wrap(gx, nx);
        } else if ((unsigned)gy >= (unsigned)ny || (unsigned)gx >= (unsigned)nx) {
          continue;  // outside the array: stays 0
        }
        A[ly * DCP_PW + lx] = __ldcg(X + (long long)gy * nx + gx);
      }
    }
    __syncthreads();
    // border: cells within a radius of the tile's edge
    const int nb_cells = h * w - (ih > 0 && iw > 0 ? ih * iw : 0);
    for (int i = threadIdx.x; i < nb_cells; i += DCP_THREADS) {
      int ty, tx;
      dcp_border_cell(i, h, w, ih, iw, ty, tx);
      dcp_cell<S>(A, B, DCP_RY + ty, DCP_RX + tx, y0 + ty, x0 + tx, ny, nx, km);
    }
    __syncthreads();
    if (S + 1 < DCP_NSTEPS) {
      // publish this tile's border ring of step S + 1
      T* __restrict__ X = q.xb[(S + 1) & 1];
      for (int i = threadIdx.x; i < nb_cells; i += DCP_THREADS) {
        int ty, tx;
        dcp_border_cell(i, h, w, ih, iw, ty, tx);
        __stcg(X + (long long)(y0 + ty) * nx + (x0 + tx), B[(DCP_RY + ty) * DCP_PW + DCP_RX + tx]);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        dcp_st_release(q.flags + (tyi * q.s.tiles_x + txi), epoch * 64u + (unsigned)(S + 1));
      }
    }
    T* t = A;
    A = B;
    B = t;
    dcp_coop_steps<S + 1>(q, A, B, tyi, txi, h, w, epoch, km);
  }
}

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpCoopParams q) {
  extern __shared__ __align__(16) unsigned char dcp_smem[];
  __shared__ unsigned epoch_s;
  const DcpStParams& p = q.s;
  T* A = reinterpret_cast<T*>(dcp_smem);
  T* B = A + DCP_TILE_ELEMS;
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
  const int ny = p.ny, nx = p.nx;
  const int tyi = blockIdx.x / p.tiles_x, txi = blockIdx.x - tyi * p.tiles_x;
  const int y0 = tyi * DCP_TY, x0 = txi * DCP_TX;
  const int h = min(DCP_TY, ny - y0), w = min(DCP_TX, nx - x0);
  if (threadIdx.x == 0) epoch_s = *(volatile unsigned*)q.ctr;
  DcpGuard guard;
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
  // step 0's input: the tile and its halo (zero outside the array)
  for (int i = threadIdx.x; i < DCP_TILE_ELEMS; i += DCP_THREADS) {
    const int ly = i / DCP_PW, lx = i - ly * DCP_PW;
    int gy = y0 - DCP_RY + ly, gx = x0 - DCP_RX + lx;
    T v = (T)0;
    if (ly < h + 2 * DCP_RY && lx < w + 2 * DCP_RX) {
      const bool inside = (unsigned)gy < (unsigned)ny && (unsigned)gx < (unsigned)nx;
      if (DCP_BC == DCP_BC_PERIODIC) {
        gy = dcp_wrap(gy, ny);
        gx = dcp_wrap(gx, nx);
        v = dcp_input(p, sc, (long long)gy * nx + gx);
        if (DCP_GUARD) guard.see(v);
      } else if (inside) {
        v = dcp_input(p, sc, (long long)gy * nx + gx);
        if (DCP_GUARD) guard.see(v);
      }
    }
    A[i] = v;
    B[i] = (T)0;
  }
  __syncthreads();
  const unsigned epoch = epoch_s;
  dcp_coop_steps<0>(q, A, B, tyi, txi, h, w, epoch, km);

  // the tile after the last step: post maps, stores and reductions
  T acc[DCP_ARR(DCP_NRED)];
#pragma unroll
  for (int r = 0; r < DCP_NRED; ++r) acc[r] = dcp_red_init<T>(dcp_red_op(r));
  for (int i = threadIdx.x; i < h * w; i += DCP_THREADS) {
    const int ty = i / w, tx = i - ty * w;
    const long long gi = (long long)(y0 + ty) * nx + (x0 + tx);
    const T v = A[(ty + DCP_RY) * DCP_PW + tx + DCP_RX];
    T st[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
    dcp_post(p, sc, gi, v, st, rv);
#pragma unroll
    for (int s = 0; s < DCP_NSTORE; ++s) p.st[s][gi] = st[s];
#pragma unroll
    for (int r = 0; r < DCP_NRED; ++r)
      acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
  }
#if DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
#if DCP_GUARD
  guard.flush(p.guard);
#endif
  // the last CTA to finish advances the epoch for the next launch (every CTA
  // has read it by then)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(q.ctr + 1, 1u) == gridDim.x - 1) {
      q.ctr[1] = 0u;
      __threadfence();
      atomicAdd(q.ctr, 1u);
    }
  }
}
