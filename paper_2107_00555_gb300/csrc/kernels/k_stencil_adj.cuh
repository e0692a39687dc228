// k_stencil_adj.cuh -- skeleton of the time-tiled reverse pass of a 1-D /
// 2-D stencil chain.  The forward chain is u_{i+1} = E_i(z_i),
// z_i = S_i u_i (a weighted sum of shifted cells, then the step's epilogue
// maps E_i); its reverse step is  g_i = S_i^T (E_i'(z_i) * g_{i+1})  (the
// transposed stencil: the same weights at negated offsets).
//
// One launch runs DCP_K reverse steps.  It reads only u_t (a checkpoint
// the forward pass stored) and the cotangent g_{t+K}, and writes g_t:
//   1. stage u_t on the output tile plus a halo of 2 K r cells;
//   2. recompute the forward states u_{t+1} .. u_{t+K} in shared memory,
//      level i on the tile plus (2K - i) r ... grown back to i r from the
//      staging edge: every level keeps the cells the reverse steps need;
//   3. run the K reverse steps, the cotangent region shrinking by r per
//      step, the derivative map fused into each transposed sum.
// Device memory is therefore read twice and written once per K steps
// instead of three times per step, and the tape keeps every K-th state.
// Every forward level and reverse step does the same arithmetic, in the
// same order, as the per-step kernels, so the result is bit for bit that
// of the untiled reverse pass.
//
// Boundary rules at every level: ZERO -- cells outside the array are 0
// (states and cotangents); PERIODIC -- halo cells hold wrapped copies and
// evolve like the cells they copy.
//
// The generated prefix defines DCP_T, DCP_TX, DCP_TY, DCP_RX, DCP_RY, DCP_K,
// DCP_BC, DCP_THREADS, DCP_NEEDZ, DCP_KNAME, the multiplier table (DCP_NK,
// dcp_km) and, for every step S of the chunk,
//   T dcp_fsum<S>(const T* A, int c, km)   forward weighted sum at tile cell c
//   T dcp_fepi<S>(T z)                     forward epilogue maps
//   T dcp_bsum<S>(const T* A, int c, km)   transposed weighted sum
//   T dcp_vjp<S>(T g, T z, T u)            cotangent of z_S from the
//                                          cotangent g of u_{S+1} = E_S(z_S)
typedef DCP_T T;

#define DCP_BC_ZERO 0
#define DCP_BC_PERIODIC 1

constexpr int DCP_HX = 2 * DCP_K * DCP_RX;
constexpr int DCP_HY = 2 * DCP_K * DCP_RY;
constexpr int DCP_PW = DCP_TX + 2 * DCP_HX;  // pitch shared by every level
constexpr int DCP_PH = DCP_TY + 2 * DCP_HY;
constexpr int DCP_TILE_ELEMS = DCP_PW * DCP_PH;

typedef DcpStParamsT<T> DcpStParams;

__device__ __forceinline__ int dcp_wrap(int q, int n) {
  if ((unsigned)q < (unsigned)n) return q;
  int r = q % n;
  return r < 0 ? r + n : r;
}

// Applies f(c, inside) to every cell of the region m cells (in radii) in
// from the staging edge.
template <int M, class F>
__device__ __forceinline__ void dcp_region(int y0, int x0, int ny, int nx, F f) {
  constexpr int my = M * DCP_RY, mx = M * DCP_RX;
  constexpr int RH = DCP_PH - 2 * my, RW = DCP_PW - 2 * mx;
  for (int i = threadIdx.x; i < RH * RW; i += DCP_THREADS) {
    const int ly = my + i / RW, lx = mx + i % RW;
    const int gy = y0 + ly, gx = x0 + lx;
    const bool inside = DCP_BC == DCP_BC_PERIODIC ||
                        ((unsigned)gy < (unsigned)ny && (unsigned)gx < (unsigned)nx);
    f(ly * DCP_PW + lx, inside);
  }
}

// Forward level L = 1..K: u_L (and z_L when the reverse reads it) on the
// region L radii in.
template <int L>
__device__ __forceinline__ void dcp_forward(T* U, T* Z, int y0, int x0, int ny, int nx,
                                            const T (&km)[DCP_NK]) {
  if constexpr (L <= DCP_K) {
    const T* A = U + (L - 1) * DCP_TILE_ELEMS;
    T* B = U + L * DCP_TILE_ELEMS;
    T* ZB = Z + (L - 1) * DCP_TILE_ELEMS;
    dcp_region<L>(y0, x0, ny, nx, [&](int c, bool inside) {
      T z = (T)0, u = (T)0;
      if (inside) {
        z = dcp_fsum<L - 1>(A, c, km);
        u = dcp_fepi<L - 1>(z);
      }
      B[c] = u;
      if (DCP_NEEDZ) ZB[c] = z;
    });
    __syncthreads();
    dcp_forward<L + 1>(U, Z, y0, x0, ny, nx, km);
  }
}

// Reverse step producing g_J (J = K-1 .. 0) from h_{J+1} = E_J'(z_J) g_{J+1}
// in H.  For J > 0 the derivative map of step J-1 is applied on the spot,
// so D receives h_J; for J = 0 the cotangent g_t is written to `out`.
template <int J>
__device__ __forceinline__ void dcp_reverse(T* H, T* D, const T* U, const T* Z, int y0, int x0,
                                            int ny, int nx, int tyi, int txi,
                                            const T (&km)[DCP_NK], T* __restrict__ out) {
  if constexpr (J > 0) {
    const T* UJ = U + J * DCP_TILE_ELEMS;
    const T* ZJ = Z + (J - 1) * DCP_TILE_ELEMS;
    dcp_region<2 * DCP_K - J>(y0, x0, ny, nx, [&](int c, bool inside) {
      T h = (T)0;
      if (inside) h = dcp_vjp<J - 1>(dcp_bsum<J>(H, c, km), DCP_NEEDZ ? ZJ[c] : (T)0, UJ[c]);
      D[c] = h;
    });
    __syncthreads();
    dcp_reverse<J - 1>(D, H, U, Z, y0, x0, ny, nx, tyi, txi, km, out);
  } else {
    for (int i = threadIdx.x; i < DCP_TX * DCP_TY; i += DCP_THREADS) {
      const int ty = i / DCP_TX, tx = i - ty * DCP_TX;
      const int gy = tyi * DCP_TY + ty, gx = txi * DCP_TX + tx;
      if (gy >= ny || gx >= nx) continue;
      out[(long long)gy * nx + gx] = dcp_bsum<0>(H, (ty + DCP_HY) * DCP_PW + tx + DCP_HX, km);
    }
  }
}

// p.ld[0] = u_t, p.ld[1] = g_{t+K}, p.st[0] = g_t (all ny x nx, row-major).
extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpStParams p) {
  extern __shared__ __align__(16) unsigned char dcp_smem[];
  T* U = reinterpret_cast<T*>(dcp_smem);     // levels 0..K
  T* Z = U + (DCP_K + 1) * DCP_TILE_ELEMS;  // levels 1..K (DCP_NEEDZ)
  const int ny = p.ny, nx = p.nx;
  const int tyi = blockIdx.x / p.tiles_x, txi = blockIdx.x - tyi * p.tiles_x;
  const int y0 = tyi * DCP_TY - DCP_HY, x0 = txi * DCP_TX - DCP_HX;
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
  const T* __restrict__ u_in = p.ld[0];
  const T* __restrict__ g_in = p.ld[1];

  // 1. u_t on the whole staging area
  for (int i = threadIdx.x; i < DCP_TILE_ELEMS; i += DCP_THREADS) {
    const int ly = i / DCP_PW, lx = i - ly * DCP_PW;
    int gy = y0 + ly, gx = x0 + lx;
    T v = (T)0;
    if (DCP_BC == DCP_BC_PERIODIC) {
      v = u_in[(long long)dcp_wrap(gy, ny) * nx + dcp_wrap(gx, nx)];
    } else if ((unsigned)gy < (unsigned)ny && (unsigned)gx < (unsigned)nx) {
      v = u_in[(long long)gy * nx + gx];
    }
    U[i] = v;
  }
  __syncthreads();

  // 2. forward states u_{t+1} .. u_{t+K}
  dcp_forward<1>(U, Z, y0, x0, ny, nx, km);

  // 3. h_{t+K} = E_{K-1}'(z) g_{t+K} on the region K radii in, into level 0's
  //    buffer (u_t is no longer needed); the reverse steps then alternate
  //    between it and level K's buffer (u_{t+K} is needed only here)
  T* H = U;
  T* D = U + DCP_K * DCP_TILE_ELEMS;
  {
    const T* UK = U + DCP_K * DCP_TILE_ELEMS;
    const T* ZK = Z + (DCP_K - 1) * DCP_TILE_ELEMS;
    dcp_region<DCP_K>(y0, x0, ny, nx, [&](int c, bool inside) {
      T h = (T)0;
      if (inside) {
        const int ly = c / DCP_PW, lx = c - ly * DCP_PW;
        const int gy = dcp_wrap(y0 + ly, ny), gx = dcp_wrap(x0 + lx, nx);
        h = dcp_vjp<DCP_K - 1>(g_in[(long long)gy * nx + gx], DCP_NEEDZ ? ZK[c] : (T)0, UK[c]);
      }
      H[c] = h;
    });
  }
  __syncthreads();
  dcp_reverse<DCP_K - 1>(H, D, U, Z, y0, x0, ny, nx, tyi, txi, km, p.st[0]);
}
