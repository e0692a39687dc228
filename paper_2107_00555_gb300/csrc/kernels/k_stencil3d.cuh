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
// With DCP_CX = 2 every thread computes two cells adjacent along x: rows of
// the plane are stored from an even offset DCP_AX, so each pair of cells and
// each pair of its neighbours is one aligned 2-element shared-memory load,
// and the two weighted sums are independent chains of FP64 operations.
//
// The generated prefix defines DCP_T, DCP_TX, DCP_TY, DCP_TZ, DCP_RX,
// DCP_RY, DCP_RZ, DCP_CX, DCP_AX, DCP_BC, DCP_THREADS, DCP_KNAME, DCP_LAST, DCP_GUARD,
// DCP_NLOAD, DCP_NPLOAD, DCP_NSTORE, DCP_NSCALAR, DCP_NRED, dcp_red_op(r) and
//   T    dcp_input(const DcpStParams& p, const T* sc, long long i)
//   void dcp_sum3(const T* const* pl, int c, T (&v)[DCP_CX], const T (&km)[DCP_NK])
//        (km: the multipliers of the sum, see dcp_load_multipliers)
//        weighted sums of cells c .. c+CX-1 of the plane ring; pl[dz + RZ] = plane z + dz
//   T    dcp_epi3(T v)                         epilogue maps fused after the step
//   void dcp_post(const DcpStParams& p, const T* sc, long long i, T v, T* st, T* rv)
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)

#define DCP_BC_ZERO 0
#define DCP_BC_PERIODIC 1
#define DCP_BC_FIXED_RING 2

constexpr int DCP_LW = DCP_TX + 2 * DCP_RX;                   // loaded row: tile + halo
constexpr int DCP_PW = DCP_TX + 2 * DCP_AX;                   // stored row (interior from DCP_AX)
constexpr int DCP_PH = DCP_TY + 2 * DCP_RY;
constexpr int DCP_PLANE = DCP_PW * DCP_PH;                    // stored plane
constexpr int DCP_PLANE_LD = DCP_LW * DCP_PH;                 // loaded plane
constexpr int DCP_NP = 2 * DCP_RZ + 1;                        // planes read per output plane
constexpr int DCP_NSLOT = DCP_NP + 1;                         // ring slots
constexpr int DCP_LPT = (DCP_PLANE_LD + DCP_THREADS - 1) / DCP_THREADS;  // plane elements per thread
constexpr int DCP_UNITS = DCP_TX * DCP_TY / DCP_CX;           // cell groups per plane
constexpr int DCP_CPT = (DCP_UNITS + DCP_THREADS - 1) / DCP_THREADS;   // cell groups per thread
static_assert(DCP_CX == 1 || (DCP_TX % 2 == 0 && DCP_AX % 2 == 0 && DCP_AX >= DCP_RX),
              "paired cells need an even row layout");

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

// Stores a fetched plane into its ring slot (the loads have arrived by now:
// with DCP_GUARD its values also enter the magnitude guard).
__device__ __forceinline__ void dcp_store_plane(T* dst, const T (&v)[DCP_LPT], DcpGuard& guard) {
#pragma unroll
  for (int k = 0; k < DCP_LPT; ++k) {
    if (DCP_GUARD) guard.see(v[k]);
    const int i = threadIdx.x + k * DCP_THREADS;
    if (DCP_PLANE_LD % DCP_THREADS == 0 || i < DCP_PLANE_LD) {
      const int ly = i / DCP_LW, lx = i - ly * DCP_LW;
      dst[ly * DCP_PW + (DCP_AX - DCP_RX) + lx] = v[k];
    }
  }
}

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpStParams p) {
  extern __shared__ __align__(16) unsigned char dcp_smem[];
  T* ring = reinterpret_cast<T*>(dcp_smem);
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
  T km[DCP_NK];
  dcp_load_multipliers(km, dcp_km);
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
    const int ly = i / DCP_LW, lx = i - ly * DCP_LW;
    int y = y0 + ly, x = x0 + lx;
    bool ok = i < DCP_PLANE_LD;
    if (DCP_BC == DCP_BC_PERIODIC) {
      y = dcp_wrap(y, ny);
      x = dcp_wrap(x, nx);
    } else {
      ok = ok && (unsigned)y < (unsigned)ny && (unsigned)x < (unsigned)nx;
    }
    off[k] = ok ? (long long)y * nx + x : -1;
  }

  // ring slot of plane z: (z - z0 + RZ) mod NSLOT
  DcpGuard guard;
  T pf[DCP_LPT];
  for (int dz = -DCP_RZ; dz < DCP_RZ; ++dz) {
    dcp_fetch_plane(p, sc, off, z0 + dz, pf);
    dcp_store_plane(ring + ((dz + DCP_RZ) % DCP_NSLOT) * DCP_PLANE, pf, guard);
  }
  dcp_fetch_plane(p, sc, off, z0 + DCP_RZ, pf);
  for (int z = z0; z < z1; ++z) {
    // plane z + RZ goes into the slot last read while computing plane z - 2,
    // which every thread finished before the previous barrier
    dcp_store_plane(ring + ((z - z0 + 2 * DCP_RZ) % DCP_NSLOT) * DCP_PLANE, pf, guard);
    if (z + 1 < z1) dcp_fetch_plane(p, sc, off, z + DCP_RZ + 1, pf);
    __syncthreads();
    const T* pl[DCP_NP];
#pragma unroll
    for (int j = 0; j < DCP_NP; ++j) pl[j] = ring + ((z - z0 + j) % DCP_NSLOT) * DCP_PLANE;
#pragma unroll
    for (int k = 0; k < DCP_CPT; ++k) {
      const int i = threadIdx.x + k * DCP_THREADS;
      if (DCP_UNITS % DCP_THREADS != 0 && i >= DCP_UNITS) break;
      const int ty = i / (DCP_TX / DCP_CX), tx = (i - ty * (DCP_TX / DCP_CX)) * DCP_CX;
      const int gy = tyi * DCP_TY + ty, gx = txi * DCP_TX + tx;
      if (gy >= ny || gx >= nx) continue;
      const int c = (ty + DCP_RY) * DCP_PW + tx + DCP_AX;
      T v[DCP_CX];
      dcp_sum3(pl, c, v, km);
#pragma unroll
      for (int j = 0; j < DCP_CX; ++j) {
        if (j > 0 && gx + j >= nx) break;
        if (DCP_BC == DCP_BC_FIXED_RING &&
            (z < DCP_RZ || z >= nz - DCP_RZ || gy < DCP_RY || gy >= ny - DCP_RY ||
             gx + j < DCP_RX || gx + j >= nx - DCP_RX)) {
          v[j] = dcp_epi3(pl[DCP_RZ][c + j]);  // ring cell keeps its value; epilogue still applies
        } else {
          v[j] = dcp_epi3(v[j]);
        }
        const long long gi = ((long long)z * ny + gy) * nx + gx + j;
#if DCP_LAST
        T st[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
        dcp_post(p, sc, gi, v[j], st, rv);
#pragma unroll
        for (int s = 0; s < DCP_NSTORE; ++s) p.st[s][gi] = st[s];
#pragma unroll
        for (int r = 0; r < DCP_NRED; ++r)
          acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
#else
        p.st[0][gi] = v[j];
#endif
      }
    }
  }
#if DCP_LAST && DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
#if DCP_GUARD
  guard.flush(p.guard);
#endif
}
