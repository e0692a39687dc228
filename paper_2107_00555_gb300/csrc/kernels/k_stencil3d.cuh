// k_stencil3d.cuh -- skeleton of one step of a 3-D stencil (the 7-point
// heat-equation form of the paper's benchmarks), streamed through z: a CTA
// owns a DCP_TY x DCP_TX column of the grid over DCP_TZ consecutive planes
// and keeps the 2*RZ+1 planes it needs in a shared-memory ring, loading one
// new plane (with its x/y halo) per output plane.  Each input element is
// therefore read from device memory about (1 + 2*RZ/TZ) times per step and
// each output written once.  Step epilogue maps, a prologue on the input and
// post maps / reductions on the output are spliced in by the generator.
//
// The generated prefix defines DCP_T, DCP_TX, DCP_TY, DCP_TZ, DCP_RX,
// DCP_RY, DCP_RZ, DCP_BC, DCP_THREADS, DCP_KNAME, DCP_LAST, DCP_NLOAD,
// DCP_NPLOAD, DCP_NSTORE, DCP_NSCALAR, DCP_NRED, dcp_red_op(r) and
//   T    dcp_input(const DcpStParams& p, const T* sc, long long i)
//   T    dcp_sum3(const T* const* pl, int c)   weighted sum; pl[dz + RZ] = plane z + dz
//   T    dcp_epi3(T v)                         epilogue maps fused after the step
//   void dcp_post(const DcpStParams& p, const T* sc, long long i, T v, T* st, T* rv)
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)

#define DCP_BC_ZERO 0
#define DCP_BC_PERIODIC 1
#define DCP_BC_FIXED_RING 2

constexpr int DCP_PW = DCP_TX + 2 * DCP_RX;
constexpr int DCP_PH = DCP_TY + 2 * DCP_RY;
constexpr int DCP_PLANE = DCP_PW * DCP_PH;
constexpr int DCP_NP = 2 * DCP_RZ + 1;

typedef DcpStParamsT<T> DcpStParams;

__device__ __forceinline__ int dcp_wrap(int q, int n) {
  if ((unsigned)q < (unsigned)n) return q;
  int r = q % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ void dcp_load_plane(const DcpStParams& p, const T* sc, T* dst, int gz,
                                               int y0, int x0) {
  const int nz = p.nz, ny = p.ny, nx = p.nx;
  for (int i = threadIdx.x; i < DCP_PLANE; i += DCP_THREADS) {
    const int ly = i / DCP_PW, lx = i - ly * DCP_PW;
    int z = gz, y = y0 + ly, x = x0 + lx;
    T v = (T)0;
    if (DCP_BC == DCP_BC_PERIODIC) {
      z = dcp_wrap(z, nz);
      y = dcp_wrap(y, ny);
      x = dcp_wrap(x, nx);
      v = dcp_input(p, sc, ((long long)z * ny + y) * nx + x);
    } else if ((unsigned)z < (unsigned)nz && (unsigned)y < (unsigned)ny &&
               (unsigned)x < (unsigned)nx) {
      v = dcp_input(p, sc, ((long long)z * ny + y) * nx + x);
    }
    dst[i] = v;
  }
}

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpStParams p) {
  extern __shared__ __align__(16) unsigned char dcp_smem[];
  T* ring = reinterpret_cast<T*>(dcp_smem);
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
  const int nz = p.nz, ny = p.ny, nx = p.nx;
  const int tyi = blockIdx.x / p.tiles_x, txi = blockIdx.x - tyi * p.tiles_x;
  const int y0 = tyi * DCP_TY - DCP_RY, x0 = txi * DCP_TX - DCP_RX;
  const int z0 = blockIdx.y * DCP_TZ;
  const int z1 = min(z0 + DCP_TZ, nz);

  T acc[DCP_ARR(DCP_NRED)];
#pragma unroll
  for (int r = 0; r < DCP_NRED; ++r) acc[r] = dcp_red_init<T>(dcp_red_op(r));

  // ring slot of plane z: (z - z0 + RZ) mod NP
  for (int dz = -DCP_RZ; dz < DCP_RZ; ++dz)
    dcp_load_plane(p, sc, ring + ((dz + DCP_RZ) % DCP_NP) * DCP_PLANE, z0 + dz, y0, x0);
  for (int z = z0; z < z1; ++z) {
    dcp_load_plane(p, sc, ring + ((z - z0 + 2 * DCP_RZ) % DCP_NP) * DCP_PLANE, z + DCP_RZ, y0, x0);
    __syncthreads();
    const T* pl[DCP_NP];
#pragma unroll
    for (int j = 0; j < DCP_NP; ++j) pl[j] = ring + ((z - z0 + j) % DCP_NP) * DCP_PLANE;
    for (int i = threadIdx.x; i < DCP_TX * DCP_TY; i += DCP_THREADS) {
      const int ty = i / DCP_TX, tx = i - ty * DCP_TX;
      const int gy = tyi * DCP_TY + ty, gx = txi * DCP_TX + tx;
      if (gy >= ny || gx >= nx) continue;
      const int c = (ty + DCP_RY) * DCP_PW + tx + DCP_RX;
      T v;
      if (DCP_BC == DCP_BC_FIXED_RING &&
          (z < DCP_RZ || z >= nz - DCP_RZ || gy < DCP_RY || gy >= ny - DCP_RY || gx < DCP_RX ||
           gx >= nx - DCP_RX)) {
        v = dcp_epi3(pl[DCP_RZ][c]);  // ring cell keeps its value; epilogue still applies
      } else {
        v = dcp_epi3(dcp_sum3(pl, c));
      }
      const long long gi = ((long long)z * ny + gy) * nx + gx;
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
    __syncthreads();
  }
#if DCP_LAST && DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
}
