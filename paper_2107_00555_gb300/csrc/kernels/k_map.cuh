// k_map.cuh -- skeleton of a fused map(+reduce) kernel: one pass over the
// iteration space, every fused elementwise op evaluated in registers, each
// loaded array read once and each stored array written once (Sec. 3.1
// greedy subgraph fusion; the reductions are the tiled write-conflict
// resolution epilogue).
//
// The generated prefix defines:
//   DCP_T, DCP_VEC (elements per 16-byte access, 1 = scalar path),
//   DCP_UNROLL, DCP_NLOAD, DCP_NSTORE, DCP_NSCALAR, DCP_NRED, DCP_THREADS,
//   DCP_KNAME and
//   dcp_body(const T* ld, const T* sc, T* st, T* rv): loads -> stores and
//   reduction inputs for one element.
//
// Memory access: a grid-stride loop over 16-byte vectors (float4 / double2 /
// int4 / longlong2 lanes), DCP_UNROLL vectors per array in flight per thread,
// streaming loads that bypass L1 and streaming stores; the ragged tail
// (n mod DCP_VEC elements) is done element by element.
typedef DCP_T T;
typedef typename DcpFin<T>::type F;

#define DCP_ARR(n) ((n) > 0 ? (n) : 1)

struct DcpMapParams {
  const T* ld[DCP_MAXIO];
  T* st[DCP_MAXIO];
  const T* sc[DCP_MAXIO];
  T* red_out[DCP_MAXIO];
  long long n;
  F* partials;
  unsigned int* ticket;
};

extern "C" __global__ void __launch_bounds__(DCP_THREADS) DCP_KNAME(const DcpMapParams p) {
  T sc[DCP_ARR(DCP_NSCALAR)];
#pragma unroll
  for (int i = 0; i < DCP_NSCALAR; ++i) sc[i] = p.sc[i][0];
  T acc[DCP_ARR(DCP_NRED)];
#pragma unroll
  for (int r = 0; r < DCP_NRED; ++r) acc[r] = dcp_red_init<T>(dcp_red_op(r));

  const long long tid = (long long)blockIdx.x * DCP_THREADS + threadIdx.x;
  const long long nthr = (long long)gridDim.x * DCP_THREADS;

#if DCP_VEC > 1
  typedef DcpPack<T, DCP_VEC> Pack;
  const long long nv = p.n / DCP_VEC;
  long long v = tid;
  for (; v + (DCP_UNROLL - 1) * nthr < nv; v += DCP_UNROLL * nthr) {
    Pack lv[DCP_UNROLL][DCP_ARR(DCP_NLOAD)];
#pragma unroll
    for (int u = 0; u < DCP_UNROLL; ++u)
#pragma unroll
      for (int l = 0; l < DCP_NLOAD; ++l)
        lv[u][l].u = dcp_ld_stream16(p.ld[l] + (v + u * nthr) * DCP_VEC);
#pragma unroll
    for (int u = 0; u < DCP_UNROLL; ++u) {
      Pack sv[DCP_ARR(DCP_NSTORE)];
#pragma unroll
      for (int j = 0; j < DCP_VEC; ++j) {
        T ld[DCP_ARR(DCP_NLOAD)], st[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
#pragma unroll
        for (int l = 0; l < DCP_NLOAD; ++l) ld[l] = lv[u][l].t[j];
        dcp_body(ld, sc, st, rv);
#pragma unroll
        for (int s = 0; s < DCP_NSTORE; ++s) sv[s].t[j] = st[s];
#pragma unroll
        for (int r = 0; r < DCP_NRED; ++r)
          acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
      }
#pragma unroll
      for (int s = 0; s < DCP_NSTORE; ++s) dcp_st_stream16(p.st[s] + (v + u * nthr) * DCP_VEC, sv[s].u);
    }
  }
  for (; v < nv; v += nthr) {
    Pack lv[DCP_ARR(DCP_NLOAD)], sv[DCP_ARR(DCP_NSTORE)];
#pragma unroll
    for (int l = 0; l < DCP_NLOAD; ++l) lv[l].u = dcp_ld_stream16(p.ld[l] + v * DCP_VEC);
#pragma unroll
    for (int j = 0; j < DCP_VEC; ++j) {
      T ld[DCP_ARR(DCP_NLOAD)], st[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
#pragma unroll
      for (int l = 0; l < DCP_NLOAD; ++l) ld[l] = lv[l].t[j];
      dcp_body(ld, sc, st, rv);
#pragma unroll
      for (int s = 0; s < DCP_NSTORE; ++s) sv[s].t[j] = st[s];
#pragma unroll
      for (int r = 0; r < DCP_NRED; ++r)
        acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
    }
#pragma unroll
    for (int s = 0; s < DCP_NSTORE; ++s) dcp_st_stream16(p.st[s] + v * DCP_VEC, sv[s].u);
  }
  const long long tail0 = nv * DCP_VEC;
#else
  const long long tail0 = 0;
#endif
  for (long long i = tail0 + tid; i < p.n; i += nthr) {
    T ld[DCP_ARR(DCP_NLOAD)], st[DCP_ARR(DCP_NSTORE)], rv[DCP_ARR(DCP_NRED)];
#pragma unroll
    for (int l = 0; l < DCP_NLOAD; ++l) ld[l] = p.ld[l][i];
    dcp_body(ld, sc, st, rv);
#pragma unroll
    for (int s = 0; s < DCP_NSTORE; ++s) p.st[s][i] = st[s];
#pragma unroll
    for (int r = 0; r < DCP_NRED; ++r)
      acc[r] = dcp_red_comb(dcp_red_op(r), acc[r], dcp_red_lift(dcp_red_op(r), rv[r]));
  }
#if DCP_NRED > 0
  dcp_reduce_epilogue<T, DCP_NRED, DCP_THREADS>(acc, p.red_out, p.partials, p.ticket);
#endif
}
