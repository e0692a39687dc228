// k_stencil3d.cuh -- skeleton of one step of a 3-D stencil (the 7-point
// heat-equation form of the paper's benchmarks), streamed through z: a CTA
// owns a DCP_TY x DCP_TX column of the grid over DCP_TZ consecutive planes
// and keeps the planes it reads in a shared-memory ring of 2*RZ+2 slots.
// While plane z is computed from the 2*RZ+1 planes around it, the loads of
// the next plane (with its x/y halo) are already in flight into registers;
// the one slot not being read receives them, so a single barrier per plane
// suffices.  Each input element is read from device memory about
// (1 + 2*RZ/TZ) times per step and each output written once.  Step epilogue
// maps, a prologue on the input and post maps / reductions on the output are
// spliced in by the generator.
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
constexpr int DCP_NP = 2 * DCP_RZ + 1;                                     // planes read per output plane
constexpr int DCP_NSLOT = DCP_NP + 1;                                      // ring slots
constexpr int DCP_LPT = (DCP_PLANE + DCP_THREADS - 1) / DCP_THREADS;       // plane elements per thread
constexpr int DCP_CPT = (DCP_TX * DCP_TY + DCP_THREADS - 1) / DCP_THREADS; // output cells per thread

typedef DcpStParamsT<T> DcpStParams;

__device__ __forceinline__ int dcp_wrap(int q, int n) {
  if ((unsigned)q < (unsigned)n) return q;
  int r = q % n;
  return r < 0 ? r + n : r;
}

// Plane gz of the CTA's column (with halo) into registers; off[k] is the
// in-plane offset of this thread's k-th element, -1 outside the array.
__device__ __forceinline__ void dcp_fetch_plane(const DcpStParams& p, const T* sc,
                                                const long long (&off)[DCP_LPT], int gz,
                                                T (&v)[DCP_LPT]) {
  int z = gz;
  bool zok = true;
  if (DCP_BC == DCP_BC_PERIODIC) z = dcp_wrap(gz, p.nz);
  else zok = (unsigned)gz < (unsigned)p.nz;
  const long long zb = (long long)z * p.ny * p.nx;
#pragma unroll
  for (int k = 0; k < DCP_LPT; ++k)
    v[k] = (zok && off[k] >= 0) ? dcp_input(p, sc, zb + off[k]) : (T)0;
}

__device__ __forceinline__ void dcp_store_plane(T* dst, const T (&v)[DCP_LPT]) {
#pragma unroll
  for (int k = 0; k < DCP_LPT; ++k) {
    const int i = threadIdx.x + k * DCP_THREADS;
    if (DCP_PLANE % DCP_THREADS == 0 || i < DCP_PLANE) dst[i] = v[k];
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

  // in-plane offsets of this thread's plane elements (the same for every plane)
  long long off[DCP_LPT];
#pragma unroll
  for (int k = 0; k < DCP_LPT; ++k) {
    const int i = threadIdx.x + k * DCP_THREADS;
    const int ly = i / DCP_PW, lx = i - ly * DCP_PW;
    int y = y0 + ly, x = x0 + lx;
    bool ok = i < DCP_PLANE;
    if (DCP_BC == DCP_BC_PERIODIC) {
      y = dcp_wrap(y, ny);
      x = dcp_wrap(x, nx);
    } else {
      ok = ok && (unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx;
    }
    off[k] = ok ? (long long)y * nx + x : -1;
  }

  // ring slot of plane z: (z - z0 + RZ) mod NSLOT
  T pf[DCP_LPT];
  for (int dz = -DCP_RZ; dz < DCP_RZ; ++dz) {
    dcp_fetch_plane(p, sc, off, z0 + dz, pf);
    dcp_store_plane(ring + ((dz + DCP_RZ) % DCP_NSLOT) * DCP_PLANE, pf);
  }
  dcp_fetch_plane(p, sc, off, z0 + DCP_RZ, pf);
  for (int z = z0; z < z1; ++z) {
    // plane z + RZ goes into the slot last read while computing plane z - 2,
    // which every thread finished before the previous barrier
    dcp_store_plane(ring + ((z - z0 + 2 * DCP_RZ) % DCP_NSLOT) * DCP_PLANE, pf);
    if (z + 1 < z1) dcp_fetch_plane(p, sc, off, z + DCP_RZ + 1, pf);
    __syncthreads();
    const T* pl[DCP_NP];
#pragma unroll
    for (int j = 0; j < DCP_NP; ++j) pl[j] = ring + ((z - z0 + j) % DCP_NSLOT) * DCP_PLANE;
#pragma unroll
    for (int k = 0; k < DCP_CPT; ++k) {
      const int i = threadIdx.x + k * DCP_THREADS;
      if ((DCP_TX * DCP_TY) % DCP_THREADS != 0 && i >= DCP_TX * DCP_TY) break;
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
  }
#if DCP_LAST && DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
}
