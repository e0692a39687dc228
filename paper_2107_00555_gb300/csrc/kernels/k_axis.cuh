// k_axis.cuh -- skeleton of a reduction along one axis (NumPy x.sum(axis=a);
// tiled write-conflict resolution with one partial per remaining index).
//
// The iteration space is viewed as (outer, R, inner), R the reduced axis.
// A CTA of DCP_THREADS threads covers TO outer indices x TI inner indices
// with TR threads along R (all powers of two, TO * TI * TR = DCP_THREADS,
// chosen by the host from the shape): consecutive threads run along the
// contiguous axis (inner, or R when inner == 1), so loads are coalesced.
// Each thread combines its elements r = r0 + tr, r0 + tr + TR, ... in index
// order, and the TR partial results are combined by a fixed tree (warp
// shuffles when the TR threads of an output share a warp, shared memory
// otherwise); a CTA owns one tile.  When the host splits R over S
// CTAs (few outputs, long axis) each split writes a partial and the last CTA
// of the tile to take a ticket combines the S partials, its TR threads per
// output taking every TR-th split in order, then the same tree.  No
// floating atomics, no waiting: the result depends only on the launch shape.
//
// Loads are 16-byte vectors of DCP_VEC elements along the contiguous axis
// when the shape and the buffers allow it: along inner (each thread then
// owns DCP_VEC adjacent outputs) or, for contiguous rows (inner == 1), along
// R (each thread combines DCP_VEC consecutive elements in order).
//
// The generated prefix defines DCP_T, DCP_THREADS, DCP_KNAME, DCP_NRED,
// DCP_NLOAD, DCP_NSCALAR, DCP_VEC, DCP_AXMODE (0: vectors along inner, 1:
// along R), dcp_red_op(r) and
//   void dcp_body(const T* ld, const T* sc, T* rv)
//        the reduced operands (prologue maps fused) from one element's loads
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)
typedef DcpAxParamsT<T> DcpAxParams;

constexpr int V = DCP_VEC;                   // elements per load
constexpr int VO = DCP_AXMODE == 0 ? V : 1;  // outputs per thread
constexpr int NL = DCP_ARR(DCP_NLOAD);
constexpr int NQ = DCP_ARR(DCP_NRED);
constexpr int UNR = V > 1 ? 2 : 4;           // loads in flight per thread and input

// The V consecutive elements of every input at flat index gi.
__device__ __forceinline__ void dcp_load_v(const DcpAxParams& p, long long gi, T (&ld)[NL][V]) {
#pragma unroll
  for (int l = 0; l < DCP_NLOAD; ++l) {
    if constexpr (V > 1) {
      DcpPack<T, V> pk;
      pk.u = dcp_ld_stream16(p.ld[l] + gi);
#pragma unroll
      for (int v = 0; v < V; ++v) ld[l][v] = pk.t[v];
    } else {
      ld[l][0] = p.ld[l][gi];
    }
  }
}

// Combine element v of a loaded vector into output slot `slot`.
__device__ __forceinline__ void dcp_acc_elem(const T (&ld)[NL][V], int v, const T* sc,
                                             T (&acc)[NQ * VO], int slot) {
  T l[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) l[k] = ld[k][v];
  T rv[NQ];
  dcp_body(l, sc, rv);
#pragma unroll
  for (int q = 0; q < DCP_NRED; ++q)
    acc[q * VO + slot] = dcp_red_comb(dcp_red_op(q), acc[q * VO + slot],
                                      dcp_red_lift(dcp_red_op(q), rv[q]));
}

// Combine the TR per-thread values of each output; valid where tr == 0.
// Value j of the array belongs to reduction j / VO.  buf holds N values of
// 8 bytes per thread (shared memory).
template <typename U, bool FIN, int N>
__device__ __forceinline__ void dcp_tree(U (&v)[N], U* buf, int TI, int TR, int t, int tr) {
  if (TI * TR <= 32) {
    for (int st = TR >> 1; st >= 1; st >>= 1) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const U w = __shfl_xor_sync(0xffffffffu, v[j], st * TI);
        if constexpr (FIN) v[j] = dcp_fin_comb(dcp_red_op(j / VO), v[j], w);
        else v[j] = dcp_red_comb(dcp_red_op(j / VO), v[j], w);
      }
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < N; ++j) buf[j * DCP_THREADS + t] = v[j];
  __syncthreads();
  for (int st = TR >> 1; st >= 1; st >>= 1) {
    if (tr < st) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const U w = buf[j * DCP_THREADS + t + st * TI];
        const U a = buf[j * DCP_THREADS + t];
        if constexpr (FIN) buf[j * DCP_THREADS + t] = dcp_fin_comb(dcp_red_op(j / VO), a, w);
        else buf[j * DCP_THREADS + t] = dcp_red_comb(dcp_red_op(j / VO), a, w);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < N; ++j) v[j] = buf[j * DCP_THREADS + t];
  __syncthreads();  // buf is reused by the next tree
}

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpAxParams p) {
  __shared__ __align__(8) unsigned char s_buf[NQ * VO * DCP_THREADS * 8];
  __shared__ bool s_last;
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int k = 0; k < DCP_NSCALAR; ++k) sc[k] = p.sc[k][0];
  const int t = threadIdx.x;
  const int TI = p.TI, TR = p.TR;
  const int ti = t & (TI - 1);
  const int tr = (t / TI) & (TR - 1);
  const int to = t / (TI * TR);
  const long long inner = p.inner;
  const long long nout = p.outer * inner;
  const int s = blockIdx.y;
  const long long r0 = (long long)s * p.rchunk;
  const long long r1 = min(p.R, r0 + p.rchunk);
  const long long tile = blockIdx.x;
  const long long ob = tile / p.ntiles, it = tile - ob * p.ntiles;
  const long long o = ob * p.TO + to;
  const long long i0 = (it * TI + ti) * VO;  // first output index along inner
  const bool active = o < p.outer && i0 < inner;

  T acc[NQ * VO];
#pragma unroll
  for (int j = 0; j < NQ * VO; ++j) acc[j] = dcp_red_init<T>(dcp_red_op(j / VO));
  if (active) {
    if constexpr (DCP_AXMODE == 0) {
      // rows r, r + TR, ... of V adjacent inner indices, in index order
      const long long base = o * p.R * inner + i0;
      long long r = r0 + tr;
      for (; r + (UNR - 1) * (long long)TR < r1; r += UNR * (long long)TR) {
        T ld[UNR][NL][V];
#pragma unroll
        for (int u = 0; u < UNR; ++u) dcp_load_v(p, base + (r + u * (long long)TR) * inner, ld[u]);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v) dcp_acc_elem(ld[u], v, sc, acc, v);
      }
      for (; r < r1; r += TR) {
        T ld[NL][V];
        dcp_load_v(p, base + r * inner, ld);
#pragma unroll
        for (int v = 0; v < V; ++v) dcp_acc_elem(ld, v, sc, acc, v);
      }
    } else {
      // contiguous row: vectors of V consecutive elements, TR*V apart
      const long long base = o * p.R;
      const long long step = (long long)TR * V;
      long long r = r0 + (long long)tr * V;
      for (; r + (UNR - 1) * step < r1; r += UNR * step) {
        T ld[UNR][NL][V];
#pragma unroll
        for (int u = 0; u < UNR; ++u) dcp_load_v(p, base + r + u * step, ld[u]);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v) dcp_acc_elem(ld[u], v, sc, acc, 0);
      }
      for (; r < r1; r += step) {
        T ld[NL][V];
        dcp_load_v(p, base + r, ld);
#pragma unroll
        for (int v = 0; v < V; ++v) dcp_acc_elem(ld, v, sc, acc, 0);
      }
    }
  }
  T* s_red = reinterpret_cast<T*>(s_buf);
  dcp_tree<T, false, NQ * VO>(acc, s_red, TI, TR, t, tr);
  const long long oi = o * inner + i0;
  if (p.S == 1) {
    if (tr == 0 && active) {
#pragma unroll
      for (int j = 0; j < NQ * VO; ++j)
        if (j / VO < DCP_NRED) p.out[j / VO][oi + j % VO] = acc[j];
    }
    return;
  }
  // R split over S CTAs: partials, then the tile's last CTA combines them
  if (tr == 0 && active) {
#pragma unroll
    for (int j = 0; j < NQ * VO; ++j)
      if (j / VO < DCP_NRED)
        p.partials[((long long)(j / VO) * p.S + s) * nout + oi + j % VO] = (F)acc[j];
  }
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned int prev = atomicAdd(p.tickets + tile, 1u);
    s_last = prev == (unsigned int)(p.S - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  F fin[NQ * VO];
#pragma unroll
  for (int j = 0; j < NQ * VO; ++j) {
    F v = (F)dcp_red_init<T>(dcp_red_op(j / VO));
    if (active && j / VO < DCP_NRED)
      for (int k = tr; k < p.S; k += TR)
        v = dcp_fin_comb(dcp_red_op(j / VO), v,
                         __ldcg(p.partials + ((long long)(j / VO) * p.S + k) * nout + oi + j % VO));
    fin[j] = v;
  }
  dcp_tree<F, true, NQ * VO>(fin, reinterpret_cast<F*>(s_buf), TI, TR, t, tr);
  if (tr == 0 && active) {
#pragma unroll
    for (int j = 0; j < NQ * VO; ++j)
      if (j / VO < DCP_NRED) p.out[j / VO][oi + j % VO] = (T)fin[j];
  }
  if (t == 0) p.tickets[tile] = 0u;  // ready for the next launch
}
