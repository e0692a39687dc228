/*
 * dcp oracle — plain, slow, single-threaded CPU reference for the fused
 * dataflow executor.  TEST INFRASTRUCTURE ONLY: it is called by tests/,
 * by the smoke check and by the CPU-baseline leg of the benchmark, never by
 * the product path.  It shares no code, header or constant with the CUDA
 * library and includes nothing from it.
 *
 * Every routine evaluates one NumPy-level operation of the program as a
 * plain loop in IEEE binary64 and materialises its whole output, which is
 * the unfused, op-at-a-time execution that the paper's translation starts
 * from (Sec. 2.3: one operation per SSA statement; Table 1: an assignment
 * becomes a map over the array with a tasklet per element).
 *
 * Build flags must keep binary64 semantics literal: -std=c11
 * -ffp-contract=off, no -ffast-math (no fused multiply-add, no
 * reassociation), so every sum below is evaluated exactly in the order
 * written.
 *
 * ORC_PARFOR / ORC_PARFOR2 mark the loops whose iterations write disjoint outputs (the
 * elementwise maps and the stencil step).  The checker build ignores it.  A
 * second build with -fopenmp, used only to time the oracle on every host
 * core, runs those loops in parallel; every output element is still the
 * same expression evaluated in the same order, so both builds give the
 * same bits.  Reductions and the transposed (scatter) step stay
 * sequential in both.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#define ORC_PARFOR _Pragma("omp parallel for schedule(static)")
#define ORC_PARFOR2 _Pragma("omp parallel for collapse(2) schedule(static)")
#else
#define ORC_PARFOR
#define ORC_PARFOR2
#endif

/* ---- operation codes (the oracle's own numbering) ---------------------- */
enum {
  ORC_NEG = 0, ORC_ABS, ORC_EXP, ORC_SIN, ORC_COS, ORC_TANH, ORC_SQRT, ORC_SQUARE,
  ORC_ADD, ORC_SUB, ORC_MUL, ORC_DIV, ORC_MAX, ORC_MIN,
  ORC_ADD_S, ORC_MUL_S, ORC_SUB_S, ORC_RSUB_S
};
enum { ORC_BC_ZERO = 0, ORC_BC_PERIODIC = 1, ORC_BC_FIXED_RING = 2 };
enum { ORC_RED_SUM = 0, ORC_RED_MAX = 1, ORC_RED_MIN = 2, ORC_RED_MAXABS = 3 };

/* Larger-of with NumPy's NaN propagation (np.maximum): NaN if either operand
 * is NaN, otherwise a when a > b, else b. */
static double orc_fmax_nan(double a, double b) {
  if (isnan(a) || isnan(b)) return NAN;
  return a > b ? a : b;
}
static double orc_fmin_nan(double a, double b) {
  if (isnan(a) || isnan(b)) return NAN;
  return a < b ? a : b;
}

/* ======================================================================= */
/* Elementwise maps, floating point (Sec. 2.3, Table 1: element-wise array  */
/* operations become map scopes with one tasklet per element).             */
/* y[i] = op(a[i], b[i])  or  op(a[i], imm).  Returns 0, or -1 on bad op.   */
/* ======================================================================= */
int orc_map_f(int op, int64_t n, const double* a, const double* b, double imm, double* y) {
  int64_t i;
  switch (op) {
    case ORC_NEG:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = -a[i]; } break;
    case ORC_ABS:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = fabs(a[i]); } break;
    case ORC_EXP:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = exp(a[i]); } break;
    case ORC_SIN:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = sin(a[i]); } break;
    case ORC_COS:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = cos(a[i]); } break;
    case ORC_TANH:   { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = tanh(a[i]); } break;
    case ORC_SQRT:   { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = sqrt(a[i]); } break;
    case ORC_SQUARE: { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] * a[i]; } break;
    case ORC_ADD:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] + b[i]; } break;
    case ORC_SUB:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] - b[i]; } break;
    case ORC_MUL:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] * b[i]; } break;
    case ORC_DIV:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] / b[i]; } break;
    case ORC_MAX:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = orc_fmax_nan(a[i], b[i]); } break;
    case ORC_MIN:    { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = orc_fmin_nan(a[i], b[i]); } break;
    case ORC_ADD_S:  { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] + imm; } break;
    case ORC_MUL_S:  { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] * imm; } break;
    case ORC_SUB_S:  { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = a[i] - imm; } break;
    case ORC_RSUB_S: { ORC_PARFOR for (i = 0; i < n; ++i) y[i] = imm - a[i]; } break;
    default: return -1;
  }
  return 0;
}

/* ======================================================================= */
/* Elementwise maps, integers.  NumPy integer arithmetic wraps modulo 2^bits */
/* (two's complement); values are carried in int64 and wrapped to `bits`    */
/* (32 or 64) after every operation.  Arithmetic is done on uint64_t so the */
/* wrap is defined behaviour in C.                                          */
/* ======================================================================= */
static int64_t orc_wrap(uint64_t v, int bits) {
  if (bits == 64) return (int64_t)v;
  uint64_t m = v & 0xffffffffull;
  return (m & 0x80000000ull) ? (int64_t)(m | 0xffffffff00000000ull) : (int64_t)m;
}

int orc_map_i(int op, int bits, int64_t n, const int64_t* a, const int64_t* b, int64_t imm,
              int64_t* y) {
  int64_t i;
  for (i = 0; i < n; ++i) {
    uint64_t x = (uint64_t)a[i];
    uint64_t z = b ? (uint64_t)b[i] : 0;
    uint64_t s = (uint64_t)imm;
    uint64_t r;
    switch (op) {
      case ORC_NEG:    r = 0 - x; break;
      case ORC_ABS:    r = (a[i] < 0) ? 0 - x : x; break;
      case ORC_SQUARE: r = x * x; break;
      case ORC_ADD:    r = x + z; break;
      case ORC_SUB:    r = x - z; break;
      case ORC_MUL:    r = x * z; break;
      case ORC_MAX:    r = (a[i] > b[i]) ? x : z; break;
      case ORC_MIN:    r = (a[i] < b[i]) ? x : z; break;
      case ORC_ADD_S:  r = x + s; break;
      case ORC_MUL_S:  r = x * s; break;
      case ORC_SUB_S:  r = x - s; break;
      case ORC_RSUB_S: r = s - x; break;
      default: return -1;
    }
    y[i] = orc_wrap(r, bits);
  }
  return 0;
}

/* ======================================================================= */
/* Stencils.  One step is a weighted sum of shifted slices of the input     */
/* (the jacobi_1d program of Sec. 2.2 and jacobi_2d of Sec. 4.3 both write  */
/* the new array as a sum of the old array at fixed offsets, times a        */
/* constant).  Here the general form                                        */
/*     out[p] = sum_k w_k * in[p + o_k]                                     */
/* is accumulated left to right in the listed point order, starting from   */
/* +0.0.  Arrays are row-major with the last axis contiguous; 1-D and 2-D   */
/* shapes are padded to (nz, ny, nx) with leading unit axes, offsets to     */
/* (dz, dy, dx) with leading zeros.                                         */
/*                                                                          */
/* Boundary readings:                                                       */
/*   ZERO        every cell is updated; reads outside the array give 0.    */
/*   PERIODIC    every cell is updated; reads wrap modulo the extent.       */
/*   FIXED_RING  only cells whose whole neighbourhood lies inside the array */
/*               are updated; the ring of width max|o| along each axis      */
/*               keeps its value (the paper's slice form B[1:-1] = ...).    */
/* A T-step stencil applies the step T times out of place (Jacobi ping-pong */
/* between two buffers, as the paper's programs alternate A and B).         */
/* ======================================================================= */
typedef struct {
  int64_t n[3];
  int npts;
  const int32_t* off; /* npts * 3, (dz, dy, dx) */
  const double* w;
  int bc;
  int64_t ring[3];
} orc_st;

static int orc_st_init(orc_st* s, int ndim, const int64_t* shape, int npts, const int32_t* offs,
                       const double* w, int bc, int32_t* off3) {
  int a, k;
  if (ndim < 1 || ndim > 3 || npts < 1) return -1;
  for (a = 0; a < 3; ++a) s->n[a] = 1;
  for (a = 0; a < ndim; ++a) s->n[3 - ndim + a] = shape[a];
  for (k = 0; k < npts; ++k) {
    for (a = 0; a < 3; ++a) off3[k * 3 + a] = 0;
    for (a = 0; a < ndim; ++a) off3[k * 3 + 3 - ndim + a] = offs[k * ndim + a];
  }
  s->npts = npts;
  s->off = off3;
  s->w = w;
  s->bc = bc;
  for (a = 0; a < 3; ++a) {
    int64_t r = 0;
    for (k = 0; k < npts; ++k) {
      int64_t o = off3[k * 3 + a] < 0 ? -(int64_t)off3[k * 3 + a] : off3[k * 3 + a];
      if (o > r) r = o;
    }
    s->ring[a] = r;
  }
  return 0;
}

static int64_t orc_mod(int64_t q, int64_t n) {
  int64_t r = q % n;
  return r < 0 ? r + n : r;
}

/* Value of `in` at (z, y, x) under the boundary rule for reads. */
static double orc_read(const orc_st* s, const double* in, int64_t z, int64_t y, int64_t x) {
  if (s->bc == ORC_BC_PERIODIC) {
    z = orc_mod(z, s->n[0]);
    y = orc_mod(y, s->n[1]);
    x = orc_mod(x, s->n[2]);
  } else if (z < 0 || z >= s->n[0] || y < 0 || y >= s->n[1] || x < 0 || x >= s->n[2]) {
    return 0.0;
  }
  return in[(z * s->n[1] + y) * s->n[2] + x];
}

static int orc_in_ring(const orc_st* s, int64_t z, int64_t y, int64_t x) {
  return z < s->ring[0] || z >= s->n[0] - s->ring[0] || y < s->ring[1] ||
         y >= s->n[1] - s->ring[1] || x < s->ring[2] || x >= s->n[2] - s->ring[2];
}

static void orc_stencil_step(const orc_st* s, const double* in, double* out) {
  ORC_PARFOR2
  for (int64_t z = 0; z < s->n[0]; ++z)
    for (int64_t y = 0; y < s->n[1]; ++y)
      for (int64_t x = 0; x < s->n[2]; ++x) {
        int64_t p = (z * s->n[1] + y) * s->n[2] + x;
        if (s->bc == ORC_BC_FIXED_RING && orc_in_ring(s, z, y, x)) {
          out[p] = in[p];
          continue;
        }
        double acc = 0.0;
        for (int k = 0; k < s->npts; ++k)
          acc += s->w[k] * orc_read(s, in, z + s->off[k * 3], y + s->off[k * 3 + 1],
                                    x + s->off[k * 3 + 2]);
        out[p] = acc;
      }
}

/* T-step stencil: out = S^T(u0).  Returns 0, -1 on bad arguments, -2 when
 * memory for the ping-pong buffer cannot be had. */
int orc_stencil_f(int ndim, const int64_t* shape, const double* u0, double* out, int npts,
                  const int32_t* offs, const double* w, int bc, int steps) {
  orc_st s;
  int32_t* off3 = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(npts > 0 ? npts : 1));
  int t, rc = 0;
  if (!off3) return -2;
  if (orc_st_init(&s, ndim, shape, npts, offs, w, bc, off3) != 0 || steps < 0) {
    free(off3);
    return -1;
  }
  int64_t n = s.n[0] * s.n[1] * s.n[2];
  double* tmp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!tmp) {
    free(off3);
    return -2;
  }
  memcpy(out, u0, sizeof(double) * (size_t)n);
  for (t = 0; t < steps; ++t) {
    orc_stencil_step(&s, out, tmp);
    memcpy(out, tmp, sizeof(double) * (size_t)n);
  }
  free(tmp);
  free(off3);
  return rc;
}

/* Transposed step (vector-Jacobian product of one step): the step is linear,
 * out = S in, so the adjoint is g_in += S^T g_out, computed by scattering each
 * output's weighted contribution back to the cells it read, through the same
 * boundary rule (a wrapped read scatters to the wrapped cell, a zero read
 * scatters nowhere, a kept ring cell passes its adjoint through). */
static void orc_stencil_step_T(const orc_st* s, const double* gout, double* gin) {
  int64_t z, y, x;
  int k;
  int64_t n = s->n[0] * s->n[1] * s->n[2];
  for (int64_t i = 0; i < n; ++i) gin[i] = 0.0;
  for (z = 0; z < s->n[0]; ++z)
    for (y = 0; y < s->n[1]; ++y)
      for (x = 0; x < s->n[2]; ++x) {
        int64_t p = (z * s->n[1] + y) * s->n[2] + x;
        if (s->bc == ORC_BC_FIXED_RING && orc_in_ring(s, z, y, x)) {
          gin[p] += gout[p];
          continue;
        }
        for (k = 0; k < s->npts; ++k) {
          int64_t qz = z + s->off[k * 3], qy = y + s->off[k * 3 + 1], qx = x + s->off[k * 3 + 2];
          if (s->bc == ORC_BC_PERIODIC) {
            qz = orc_mod(qz, s->n[0]);
            qy = orc_mod(qy, s->n[1]);
            qx = orc_mod(qx, s->n[2]);
          } else if (qz < 0 || qz >= s->n[0] || qy < 0 || qy >= s->n[1] || qx < 0 ||
                     qx >= s->n[2]) {
            continue;
          }
          gin[(qz * s->n[1] + qy) * s->n[2] + qx] += s->w[k] * gout[p];
        }
      }
}

/* g_in = (S^T)^steps g_out for a T-step stencil. */
int orc_stencil_vjp_f(int ndim, const int64_t* shape, const double* gout, double* gin, int npts,
                      const int32_t* offs, const double* w, int bc, int steps) {
  orc_st s;
  int32_t* off3 = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(npts > 0 ? npts : 1));
  int t;
  if (!off3) return -2;
  if (orc_st_init(&s, ndim, shape, npts, offs, w, bc, off3) != 0 || steps < 0) {
    free(off3);
    return -1;
  }
  int64_t n = s.n[0] * s.n[1] * s.n[2];
  double* tmp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!tmp) {
    free(off3);
    return -2;
  }
  memcpy(gin, gout, sizeof(double) * (size_t)n);
  for (t = 0; t < steps; ++t) {
    orc_stencil_step_T(&s, gin, tmp);
    memcpy(gin, tmp, sizeof(double) * (size_t)n);
  }
  free(tmp);
  free(off3);
  return 0;
}

/* Value of S^T(u0) at one cell p = (pz, py, px), computed only on the cone of
 * cells that can influence it: a box of half-width steps*max|o| around p in
 * unwrapped coordinates, shrinking by max|o| per step.  Under PERIODIC a box
 * cell takes the value of the wrapped cell (the periodic field lifted to the
 * infinite lattice evolves under the same stencil); under ZERO and
 * FIXED_RING cells outside the array hold 0 and are never updated.  Used to
 * check single outputs of grids too large for the full loop. */
double orc_stencil_point_f(int ndim, const int64_t* shape, const double* u0, int npts,
                           const int32_t* offs, const double* w, int bc, int steps,
                           const int64_t* p3, int* status) {
  orc_st s;
  int32_t off3[3 * 64];
  int a, k, t;
  *status = 0;
  if (npts > 64 || orc_st_init(&s, ndim, shape, npts, offs, w, bc, off3) != 0 || steps < 0) {
    *status = -1;
    return 0.0;
  }
  int64_t R[3], lo[3], b[3];
  for (a = 0; a < 3; ++a) {
    R[a] = (int64_t)steps * s.ring[a];
    lo[a] = p3[a] - R[a];
    b[a] = 2 * R[a] + 1;
  }
  int64_t nb = b[0] * b[1] * b[2];
  double* cur = (double*)malloc(sizeof(double) * (size_t)nb);
  double* nxt = (double*)malloc(sizeof(double) * (size_t)nb);
  if (!cur || !nxt) {
    free(cur);
    free(nxt);
    *status = -2;
    return 0.0;
  }
  for (int64_t i = 0; i < b[0]; ++i)
    for (int64_t j = 0; j < b[1]; ++j)
      for (int64_t l = 0; l < b[2]; ++l)
        cur[(i * b[1] + j) * b[2] + l] = orc_read(&s, u0, lo[0] + i, lo[1] + j, lo[2] + l);
  for (t = 1; t <= steps; ++t) {
    int64_t m[3];
    for (a = 0; a < 3; ++a) m[a] = (int64_t)t * s.ring[a];
    for (int64_t i = m[0]; i < b[0] - m[0]; ++i)
      for (int64_t j = m[1]; j < b[1] - m[1]; ++j)
        for (int64_t l = m[2]; l < b[2] - m[2]; ++l) {
          int64_t c = (i * b[1] + j) * b[2] + l;
          int64_t gz = lo[0] + i, gy = lo[1] + j, gx = lo[2] + l;
          if (bc != ORC_BC_PERIODIC &&
              (gz < 0 || gz >= s.n[0] || gy < 0 || gy >= s.n[1] || gx < 0 || gx >= s.n[2])) {
            nxt[c] = 0.0;
            continue;
          }
          if (bc == ORC_BC_FIXED_RING && orc_in_ring(&s, gz, gy, gx)) {
            nxt[c] = cur[c];
            continue;
          }
          double acc = 0.0;
          for (k = 0; k < npts; ++k) {
            int64_t q = ((i + off3[k * 3]) * b[1] + (j + off3[k * 3 + 1])) * b[2] +
                        (l + off3[k * 3 + 2]);
            acc += w[k] * cur[q];
          }
          nxt[c] = acc;
        }
    double* sw = cur;
    cur = nxt;
    nxt = sw;
  }
  double v = cur[(R[0] * b[1] + R[1]) * b[2] + R[2]];
  free(cur);
  free(nxt);
  return v;
}

/* ======================================================================= */
/* Reductions (write-conflict resolution, Sec. 2.3: a map whose iterations  */
/* all update one scalar, e.g. alpha += C[i, j]).                           */
/* ======================================================================= */

/* Sequential sum in flat index order. */
double orc_sum_seq(int64_t n, const double* y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += y[i];
  return s;
}

/* Sequential sum of magnitudes, the scale of the backward-stable bound on
 * any reassociated sum: |S_any_order - S_exact| <= (n-1) u sum|y_i|. */
double orc_sum_abs(int64_t n, const double* y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += fabs(y[i]);
  return s;
}

/* Exactly rounded sum (Shewchuk, "Adaptive precision floating-point
 * arithmetic and fast robust geometric predicates", 1997: the running sum is
 * kept as a non-overlapping expansion of doubles, each new term is added
 * with error-free two-sums, and the expansion is finally rounded once to the
 * nearest double, ties to even).  Non-finite inputs fall back to the plain
 * sequential sum, whose inf/NaN result is then the IEEE one. */
double orc_fsum(int64_t n, const double* y, int* status) {
  int cap = 64, len = 0;
  double* part = (double*)malloc(sizeof(double) * (size_t)cap);
  *status = 0;
  if (!part) {
    *status = -2;
    return 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    double x = y[i];
    if (!isfinite(x)) {
      free(part);
      return orc_sum_seq(n, y);
    }
    int j = 0;
    for (int k = 0; k < len; ++k) {
      double p = part[k];
      if (fabs(x) < fabs(p)) {
        double t = x;
        x = p;
        p = t;
      }
      double hi = x + p;
      double lo = p - (hi - x);
      if (lo != 0.0) part[j++] = lo;
      x = hi;
    }
    if (!isfinite(x)) { /* intermediate overflow: defer to IEEE */
      free(part);
      return orc_sum_seq(n, y);
    }
    if (j >= cap) {
      cap *= 2;
      double* np = (double*)realloc(part, sizeof(double) * (size_t)cap);
      if (!np) {
        free(part);
        *status = -2;
        return 0.0;
      }
      part = np;
    }
    if (x != 0.0) part[j++] = x; /* a zero component carries nothing */
    len = j;
  }
  /* Round the expansion: add terms from the most significant down until a
   * rounding error appears, then correct a half-way case using the sign of
   * the next lower term. */
  double hi = 0.0;
  if (len > 0) {
    int k = len - 1;
    hi = part[k];
    double lo = 0.0;
    while (k > 0) {
      double x = hi;
      double p = part[--k];
      hi = x + p;
      double yr = hi - x;
      lo = p - yr;
      if (lo != 0.0) break;
    }
    if (k > 0 && ((lo < 0.0 && part[k - 1] < 0.0) || (lo > 0.0 && part[k - 1] > 0.0))) {
      double t = lo * 2.0;
      double x = hi + t;
      double yr = x - hi;
      if (t == yr) hi = x;
    }
  }
  free(part);
  return hi;
}

/* MAX / MIN / MAXABS, NaN-propagating like np.max; *arg gets the first flat
 * index that attains the result (NaN: the first NaN).  n must be >= 1. */
int orc_reduce_ext_f(int red, int64_t n, const double* y, double* out, int64_t* arg) {
  if (n < 1) return -1;
  double best = (red == ORC_RED_MAXABS) ? fabs(y[0]) : y[0];
  int64_t bi = 0;
  for (int64_t i = 1; i < n && !isnan(best); ++i) {
    double v = (red == ORC_RED_MAXABS) ? fabs(y[i]) : y[i];
    int take;
    if (isnan(v)) take = 1;
    else if (red == ORC_RED_MIN) take = v < best;
    else if (red == ORC_RED_MAX || red == ORC_RED_MAXABS) take = v > best;
    else return -1;
    if (take) {
      best = v;
      bi = i;
    }
  }
  *out = best;
  *arg = bi;
  return 0;
}

/* Integer reductions: SUM wraps modulo 2^bits; MAX/MIN/MAXABS exact
 * (|INT_MIN| wraps to INT_MIN like np.abs). */
int orc_reduce_i(int red, int bits, int64_t n, const int64_t* y, int64_t* out) {
  if (red == ORC_RED_SUM) {
    uint64_t s = 0;
    for (int64_t i = 0; i < n; ++i) s += (uint64_t)y[i];
    *out = orc_wrap(s, bits);
    return 0;
  }
  if (n < 1) return -1;
  int64_t best = y[0];
  if (red == ORC_RED_MAXABS) best = orc_wrap(best < 0 ? 0 - (uint64_t)best : (uint64_t)best, bits);
  for (int64_t i = 1; i < n; ++i) {
    int64_t v = y[i];
    if (red == ORC_RED_MAXABS) v = orc_wrap(v < 0 ? 0 - (uint64_t)v : (uint64_t)v, bits);
    if (red == ORC_RED_MIN ? v < best : v > best) best = v;
  }
  *out = best;
  return 0;
}

/* Reduction along one axis (NumPy x.sum(axis=a) and friends: the
 * write-conflict resolution of Sec. 2.3 with one result per remaining index).
 * y is viewed as (outer, R, inner) in C order; out[o*inner + i] reduces the
 * R elements y[o, 0..R-1, i], gathered in index order, with the whole-array
 * routines above: SUM sequentially (fs and ab, when not NULL, receive the
 * exactly rounded sum and the magnitude sum of each output), MAX / MIN /
 * MAXABS with NaN propagation (R >= 1). */
int orc_reduce_axis_f(int red, int64_t outer, int64_t R, int64_t inner, const double* y,
                      double* out, double* fs, double* ab) {
  if (red != ORC_RED_SUM && R < 1) return -1;
  double* col = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
  if (!col) return -2;
  for (int64_t o = 0; o < outer; ++o)
    for (int64_t i = 0; i < inner; ++i) {
      const int64_t k = o * inner + i;
      for (int64_t r = 0; r < R; ++r) col[r] = y[(o * R + r) * inner + i];
      if (red == ORC_RED_SUM) {
        out[k] = orc_sum_seq(R, col);
        if (fs) {
          int st = 0;
          fs[k] = orc_fsum(R, col, &st);
          if (st) {
            free(col);
            return st;
          }
        }
        if (ab) ab[k] = orc_sum_abs(R, col);
      } else {
        int64_t arg = 0;
        int st = orc_reduce_ext_f(red, R, col, &out[k], &arg);
        if (st) {
          free(col);
          return st;
        }
      }
    }
  free(col);
  return 0;
}

/* Integer reduction along one axis (same view; SUM wraps modulo 2^bits). */
int orc_reduce_axis_i(int red, int bits, int64_t outer, int64_t R, int64_t inner,
                      const int64_t* y, int64_t* out) {
  if (red != ORC_RED_SUM && R < 1) return -1;
  int64_t* col = (int64_t*)malloc(sizeof(int64_t) * (size_t)(R > 0 ? R : 1));
  if (!col) return -2;
  for (int64_t o = 0; o < outer; ++o)
    for (int64_t i = 0; i < inner; ++i) {
      for (int64_t r = 0; r < R; ++r) col[r] = y[(o * R + r) * inner + i];
      int st = orc_reduce_i(red, bits, R, col, &out[o * inner + i]);
      if (st) {
        free(col);
        return st;
      }
    }
  free(col);
  return 0;
}

/* ======================================================================= */
/* Derivatives of the floating-point maps, for the reverse (adjoint) and     */
/* forward (tangent) passes of the unfused program.                         */
/* ======================================================================= */

/* Reverse: ga[i] += d y / d a * g[i], gb[i] += d y / d b * g[i].  y is the
 * forward output of the op.  MAX/MIN route the adjoint to the operand the
 * forward pass selected (ties and NaN: to b, the operand returned when
 * a > b is false).  ABS uses sign(a) with sign(0) = 0. */
int orc_map_vjp_f(int op, int64_t n, const double* a, const double* b, double imm,
                  const double* y, const double* g, double* ga, double* gb) {
  int64_t i;
  for (i = 0; i < n; ++i) {
    double gi = g[i];
    switch (op) {
      case ORC_NEG: ga[i] += -gi; break;
      case ORC_ABS: ga[i] += (a[i] > 0.0 ? gi : (a[i] < 0.0 ? -gi : 0.0)); break;
      case ORC_EXP: ga[i] += gi * y[i]; break;
      case ORC_SIN: ga[i] += gi * cos(a[i]); break;
      case ORC_COS: ga[i] += -gi * sin(a[i]); break;
      case ORC_TANH: ga[i] += gi * (1.0 - y[i] * y[i]); break;
      case ORC_SQRT: ga[i] += gi * (0.5 / y[i]); break;
      case ORC_SQUARE: ga[i] += gi * (2.0 * a[i]); break;
      case ORC_ADD: ga[i] += gi; gb[i] += gi; break;
      case ORC_SUB: ga[i] += gi; gb[i] += -gi; break;
      case ORC_MUL: ga[i] += gi * b[i]; gb[i] += gi * a[i]; break;
      case ORC_DIV: ga[i] += gi / b[i]; gb[i] += -gi * a[i] / (b[i] * b[i]); break;
      case ORC_MAX:
        if (a[i] > b[i]) ga[i] += gi; else gb[i] += gi;
        break;
      case ORC_MIN:
        if (a[i] < b[i]) ga[i] += gi; else gb[i] += gi;
        break;
      case ORC_ADD_S: ga[i] += gi; break;
      case ORC_MUL_S: ga[i] += gi * imm; break;
      case ORC_SUB_S: ga[i] += gi; break;
      case ORC_RSUB_S: ga[i] += -gi; break;
      default: return -1;
    }
  }
  (void)imm;
  return 0;
}

/* Forward: dy[i] = d y / d a * da[i] + d y / d b * db[i]. */
int orc_map_jvp_f(int op, int64_t n, const double* a, const double* b, double imm,
                  const double* y, const double* da, const double* db, double* dy) {
  int64_t i;
  for (i = 0; i < n; ++i) {
    switch (op) {
      case ORC_NEG: dy[i] = -da[i]; break;
      case ORC_ABS: dy[i] = a[i] > 0.0 ? da[i] : (a[i] < 0.0 ? -da[i] : 0.0); break;
      case ORC_EXP: dy[i] = y[i] * da[i]; break;
      case ORC_SIN: dy[i] = cos(a[i]) * da[i]; break;
      case ORC_COS: dy[i] = -sin(a[i]) * da[i]; break;
      case ORC_TANH: dy[i] = (1.0 - y[i] * y[i]) * da[i]; break;
      case ORC_SQRT: dy[i] = (0.5 / y[i]) * da[i]; break;
      case ORC_SQUARE: dy[i] = 2.0 * a[i] * da[i]; break;
      case ORC_ADD: dy[i] = da[i] + db[i]; break;
      case ORC_SUB: dy[i] = da[i] - db[i]; break;
      case ORC_MUL: dy[i] = b[i] * da[i] + a[i] * db[i]; break;
      case ORC_DIV: dy[i] = da[i] / b[i] - a[i] * db[i] / (b[i] * b[i]); break;
      case ORC_MAX: dy[i] = (a[i] > b[i]) ? da[i] : db[i]; break;
      case ORC_MIN: dy[i] = (a[i] < b[i]) ? da[i] : db[i]; break;
      case ORC_ADD_S: dy[i] = da[i]; break;
      case ORC_MUL_S: dy[i] = imm * da[i]; break;
      case ORC_SUB_S: dy[i] = da[i]; break;
      case ORC_RSUB_S: dy[i] = -da[i]; break;
      default: return -1;
    }
  }
  return 0;
}
