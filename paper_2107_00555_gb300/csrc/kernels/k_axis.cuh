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
// The generated prefix defines DCP_T, DCP_THREADS, DCP_KNAME, DCP_NRED,
// DCP_NSCALAR, dcp_red_op(r) and
//   void dcp_elem(const DcpAxParams& p, const T* sc, long long gi, T* rv)
//        the reduced operands (prologue maps fused) at flat index gi
typedef DCP_T T;
typedef typename DcpFin<T>::type F;
#define DCP_ARR(n) ((n) > 0 ? (n) : 1)
typedef DcpAxParamsT<T> DcpAxParams;

// Combine the TR per-thread values of each (outer, inner) index; the result
// is valid in the threads with tr == 0.  buf holds DCP_THREADS values of U
// per reduction (shared memory).
template <typename U, bool FIN>
__device__ __forceinline__ void dcp_tree(U (&v)[DCP_ARR(DCP_NRED)], U* buf, int TI, int TR, int t,
                                         int tr) {
  if (TI * TR <= 32) {
    for (int st = TR >> 1; st >= 1; st >>= 1) {
#pragma unroll
      for (int q = 0; q < DCP_NRED; ++q) {
        const U w = __shfl_xor_sync(0xffffffffu, v[q], st * TI);
        if constexpr (FIN) v[q] = dcp_fin_comb(dcp_red_op(q), v[q], w);
        else v[q] = dcp_red_comb(dcp_red_op(q), v[q], w);
      }
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < DCP_NRED; ++q) buf[q * DCP_THREADS + t] = v[q];
  __syncthreads();
  for (int st = TR >> 1; st >= 1; st >>= 1) {
    if (tr < st) {
#pragma unroll
      for (int q = 0; q < DCP_NRED; ++q) {
        const U w = buf[q * DCP_THREADS + t + st * TI];
        const U a = buf[q * DCP_THREADS + t];
        if constexpr (FIN) buf[q * DCP_THREADS + t] = dcp_fin_comb(dcp_red_op(q), a, w);
        else buf[q * DCP_THREADS + t] = dcp_red_comb(dcp_red_op(q), a, w);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < DCP_NRED; ++q) v[q] = buf[q * DCP_THREADS + t];
  __syncthreads();  // buf is reused by the next tree
}

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpAxParams p) {
  __shared__ __align__(8) unsigned char s_buf[DCP_ARR(DCP_NRED) * DCP_THREADS * 8];
  __shared__ bool s_last;
  T* s_red = reinterpret_cast<T*>(s_buf);
  F* s_fin = reinterpret_cast<F*>(s_buf);
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
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

  {
    const long long tile = blockIdx.x;
    const long long ob = tile / p.ntiles, it = tile - ob * p.ntiles;
    const long long o = ob * p.TO + to;
    const long long i = it * TI + ti;
    const bool active = o < p.outer && i < inner;
    T acc[DCP_ARR(DCP_NRED)];
#pragma unroll
    for (int q = 0; q < DCP_NRED; ++q) acc[q] = dcp_red_init<T>(dcp_red_op(q));
    if (active) {
      const long long base = o * p.R * inner + i;
      long long r = r0 + tr;
      // four elements in flight per thread, combined in index order
      for (; r + 3LL * TR < r1; r += 4LL * TR) {
        T v0[DCP_ARR(DCP_NRED)], v1[DCP_ARR(DCP_NRED)], v2[DCP_ARR(DCP_NRED)], v3[DCP_ARR(DCP_NRED)];
        dcp_elem(p, sc, base + r * inner, v0);
        dcp_elem(p, sc, base + (r + TR) * inner, v1);
        dcp_elem(p, sc, base + (r + 2LL * TR) * inner, v2);
        dcp_elem(p, sc, base + (r + 3LL * TR) * inner, v3);
#pragma unroll
        for (int q = 0; q < DCP_NRED; ++q) {
          const int op = dcp_red_op(q);
          acc[q] = dcp_red_comb(op, acc[q], dcp_red_lift(op, v0[q]));
          acc[q] = dcp_red_comb(op, acc[q], dcp_red_lift(op, v1[q]));
          acc[q] = dcp_red_comb(op, acc[q], dcp_red_lift(op, v2[q]));
          acc[q] = dcp_red_comb(op, acc[q], dcp_red_lift(op, v3[q]));
        }
      }
      for (; r < r1; r += TR) {
        T v[DCP_ARR(DCP_NRED)];
        dcp_elem(p, sc, base + r * inner, v);
#pragma unroll
        for (int q = 0; q < DCP_NRED; ++q)
          acc[q] = dcp_red_comb(dcp_red_op(q), acc[q], dcp_red_lift(dcp_red_op(q), v[q]));
      }
    }
    dcp_tree<T, false>(acc, s_red, TI, TR, t, tr);
    const long long oi = o * inner + i;
    if (p.S == 1) {
      if (tr == 0 && active) {
#pragma unroll
        for (int q = 0; q < DCP_NRED; ++q) p.out[q][oi] = acc[q];
      }
      return;
    }
    // R split over S CTAs: partials, then the tile's last CTA combines them
    if (tr == 0 && active) {
#pragma unroll
      for (int q = 0; q < DCP_NRED; ++q)
        p.partials[((long long)q * p.S + s) * nout + oi] = (F)acc[q];
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
    F fin[DCP_ARR(DCP_NRED)];
#pragma unroll
    for (int q = 0; q < DCP_NRED; ++q) {
      F v = (F)dcp_red_init<T>(dcp_red_op(q));
      if (active)
        for (int k = tr; k < p.S; k += TR)
          v = dcp_fin_comb(dcp_red_op(q), v, __ldcg(p.partials + ((long long)q * p.S + k) * nout + oi));
      fin[q] = v;
    }
    dcp_tree<F, true>(fin, s_fin, TI, TR, t, tr);
    if (tr == 0 && active) {
#pragma unroll
      for (int q = 0; q < DCP_NRED; ++q) p.out[q][oi] = (T)fin[q];
    }
    if (t == 0) p.tickets[tile] = 0u;  // ready for the next launch
  }
}
