/*
 * dcp.h — C ABI of the fused dataflow executor for NumPy-style array programs
 * (Ziogas et al., "Productivity, Portability, Performance: Data-Centric
 * Python", SC'21).
 *
 * A program is built one NumPy-level operation per call, which is the SSA
 * form the paper's frontend produces (Sec. 2.3: the expression
 * `C[:] = alpha * A @ B + beta * C` becomes one single-operation statement
 * per temporary).  Data containers are typed, shaped arrays kept separate
 * from the computations that read and write them (Sec. 2, first tenet;
 * Sec. 2.2: symbolic shapes and NumPy dtypes).  Optimisation is applied to
 * the finished graph separately from the program text (Sec. 2.4: transforms
 * are applied to the SDFG, `sdfg.apply(...)`; Sec. 3.1: greedy subgraph
 * fusion, tiled write-conflict resolution, persistent transients), and the
 * compiled result is then called like a function on caller-owned buffers
 * (Sec. 3.3).
 *
 * Conventions for every entry point:
 *  - Return value: DCP_OK (0) or a negative dcp_status.  On error,
 *    dcp_last_error() returns a thread-local, human-readable message that
 *    stays valid until the next dcp_* call on the same thread.  No entry
 *    point aborts the process, throws, or prints.
 *  - Arrays are dense, row-major (C order, last axis contiguous).  Shapes
 *    have 0..4 axes (0 = scalar); stencils take 1..3 axes.
 *  - Handles: a dcp_graph owns its nodes, its intermediate (transient)
 *    device buffers, the compiled kernels and any adjoint tape; all are
 *    released by dcp_graph_destroy.  dcp_value handles are graph-local
 *    indices, valid only for the graph that returned them.
 *  - Buffers passed to dcp_run / dcp_run_adjoint are DEVICE pointers owned
 *    by the caller, contiguous, of the declared dtype and shape.  They may
 *    have any alignment; 16-byte aligned buffers take the vectorised path.
 *    Inputs are read only; outputs are fully overwritten.  Inputs and
 *    outputs must not overlap.
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default
 *    stream).  dcp_run* enqueue work asynchronously on it and return once
 *    the work is enqueued; the caller synchronises.  No kernel waits on
 *    another thread block, so no launch can hang on a lost peer; dcp_sync()
 *    reports asynchronous CUDA errors of the stream.
 *  - Thread safety: one graph must not be used by two threads at once;
 *    different graphs are independent.
 */
#ifndef DCP_H
#define DCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dcp_graph_s* dcp_graph;
typedef int32_t dcp_value;
typedef int32_t dcp_status;

enum {
  DCP_OK = 0,
  DCP_E_INVALID_ARG = -1, /* bad handle, pointer, count, op code or option */
  DCP_E_SHAPE = -2,       /* operand shapes disagree, or a shape is not allowed */
  DCP_E_DTYPE = -3,       /* operand dtypes disagree, or op not defined on dtype */
  DCP_E_UNSUPPORTED = -4, /* well-formed request outside what the library implements */
  DCP_E_OOM = -5,         /* device or host allocation failed (or budget exceeded) */
  DCP_E_CUDA = -6,        /* a CUDA runtime/driver call failed (message has detail) */
  DCP_E_COMPILE = -7,     /* run-time compilation of a fused kernel failed */
  DCP_E_TIMEOUT = -8,     /* a bounded device-side wait expired (cooperative stencil form;
                             reported by dcp_sync / dcp_run_host; results invalid) */
  DCP_E_STATE = -9        /* call not allowed in the graph's current state */
};

/* Element types of data containers (Sec. 2: NumPy-compatible dtypes). */
enum { DCP_F32 = 1, DCP_F64 = 2, DCP_I32 = 3, DCP_I64 = 4 };

/* Elementwise operations (one tasklet per element inside a map scope,
 * Sec. 2.3 / Table 1).  Unary ops take 1 operand; binary ops 2; the _S forms
 * take 1 operand and the immediate `imm`:
 *   ADD_S: x + imm   MUL_S: x * imm   SUB_S: x - imm   RSUB_S: imm - x.
 * Floating MAX/MIN return NaN when either operand is NaN (np.maximum),
 * otherwise a when a > b (resp. a < b), else b.  Integer ops wrap modulo
 * 2^bits like NumPy; EXP..SQRT and DIV are floating only (DCP_E_DTYPE). */
enum {
  DCP_NEG = 0, DCP_ABS = 1, DCP_EXP = 2, DCP_SIN = 3, DCP_COS = 4, DCP_TANH = 5,
  DCP_SQRT = 6, DCP_SQUARE = 7,
  DCP_ADD = 8, DCP_SUB = 9, DCP_MUL = 10, DCP_DIV = 11, DCP_MAX = 12, DCP_MIN = 13,
  DCP_ADD_S = 14, DCP_MUL_S = 15, DCP_SUB_S = 16, DCP_RSUB_S = 17
};

/* Stencil boundary rules (Sec. 2.2 jacobi_1d, Sec. 4.3 jacobi_2d):
 *   ZERO        every cell is updated; reads outside the array give 0.
 *   PERIODIC    every cell is updated; reads wrap modulo each extent.
 *   FIXED_RING  only cells whose whole neighbourhood lies inside the array
 *               are updated; the ring of width max|offset| per axis keeps
 *               its value (the paper's `B[1:-1] = ...` slice form). */
enum { DCP_BC_ZERO = 0, DCP_BC_PERIODIC = 1, DCP_BC_FIXED_RING = 2 };

/* Reductions (write-conflict resolution of a map into one scalar,
 * Sec. 2.3: `alpha += C[i, j]`).  MAX/MIN/MAXABS propagate NaN. */
enum { DCP_SUM = 0, DCP_MAX_R = 1, DCP_MIN_R = 2, DCP_MAXABS = 3 };

/* dcp_fuse flags (Sec. 3.1 auto-optimisation passes).  0 = op-by-op: one
 * kernel per operation, every intermediate materialised in device memory. */
enum {
  DCP_FUSE_MAPS = 1u << 0,     /* merge same-shape elementwise maps into one kernel */
  DCP_FUSE_SUBGRAPH = 1u << 1, /* reduce epilogues, map prologue/epilogue on stencils */
  DCP_TIME_TILE = 1u << 2,     /* several stencil steps per device-memory pass */
  DCP_BATCH = 1u << 3,         /* pack independent same-program stencils into one launch */
  DCP_AUTOTUNE = 1u << 4,      /* time candidate tile shapes / depths on first run */
  DCP_FUSE_ALL = (1u << 0) | (1u << 1) | (1u << 2)
};

/* dcp_set_option keys (overrides of the planner's choices; value < 0 resets). */
enum {
  DCP_OPT_TIME_TILE_DEPTH = 1, /* stencil steps per launch (>= 1) */
  DCP_OPT_TILE_X = 2,          /* stencil tile extent along x (multiple of 8) */
  DCP_OPT_TILE_Y = 3,          /* stencil tile extent along y */
  DCP_OPT_MAP_BLOCKS_PER_SM = 4, /* CTAs per SM for map/reduce kernels */
  DCP_OPT_USE_GRAPH = 5,       /* 1: replay a captured CUDA graph in dcp_run */
  DCP_OPT_STENCIL_KERNEL = 7,  /* 1-D / 2-D stencils: 0 shared-memory tiles, 1 warp stream,
                                  2 cooperative: every step in one launch, one tile per
                                  resident CTA, neighbour flags between steps (small grids) */
  DCP_OPT_HOST_ACCESS = 8,     /* dcp_run_host: 1 (default) kernels access page-locked host
                                  buffers directly, 0 always stage through device copies */
  DCP_OPT_STREAM_ROWS = 9,     /* warp-stream stencils: rows per work item (>= 1) */
  DCP_OPT_TILE_Z = 10,         /* 3-D stencils: planes per CTA (z chunk, 1..1024) */
  DCP_OPT_STREAM_PREFETCH = 11, /* warp-stream stencils: row windows requested ahead (1..4) */
  DCP_OPT_STREAM_THREADS = 12, /* warp-stream stencils: threads per CTA (32..1024, multiple of 32; default 64) */
  DCP_OPT_CELLS_PER_THREAD = 13, /* 3-D stencils: cells per thread along x (1 or 2) */
  DCP_OPT_MAP_UNROLL = 14,      /* map kernels: 16-byte vectors per array in flight per thread (1..8) */
  DCP_OPT_DEFERRED_WEIGHT = 15, /* stencils: 1 (default) deferred common weight where it applies,
                                   0 the plain weighted sum everywhere (set before dcp_fuse) */
  DCP_OPT_STREAM_MIN_CTAS = 16, /* warp-stream stencils: CTAs per SM the register budget must
                                   allow (1..32; default: the compiler's choice) */
  DCP_OPT_ADJOINT_DEPTH = 17    /* reverse pass of 1-D / 2-D stencil chains with step
                                   epilogues: k >= 1 runs k reverse steps per launch from every
                                   k-th state, recomputing the forward states in the tile; 0
                                   (default) one launch per step (0..64; set before dcp_fuse) */
};

/* ---- graph construction ------------------------------------------------ */

/* Creates an empty graph.  *out receives the handle (caller destroys it). */
dcp_status dcp_graph_create(dcp_graph* out);

/* Destroys a graph, freeing transients, tape, compiled modules and CUDA
 * graphs.  Waits for work this graph enqueued.  NULL is accepted. */
dcp_status dcp_graph_destroy(dcp_graph g);

/* Declares a program input container of `dtype` with `ndim` (0..4) axes of
 * extents shape[0..ndim-1] (each >= 0).  Inputs are bound to dcp_run's
 * `inputs` array in declaration order. */
dcp_status dcp_add_input(dcp_graph g, int32_t dtype, int32_t ndim, const int64_t* shape,
                         dcp_value* out);

/* Elementwise map (Sec. 2.3, Table 1): out = op(in[0] [, in[1]] [, imm]).
 * Operands share one dtype; shapes are equal, except that a binary operand
 * may be a 0-axis value (a scalar container, e.g. a reduction result), which
 * is broadcast.  The result has the operands' dtype and full shape. */
dcp_status dcp_add_map(dcp_graph g, int32_t op, int32_t n_in, const dcp_value* in, double imm,
                       dcp_value* out);

/* Iterated stencil (Sec. 2.2 jacobi_1d; Sec. 4.3 jacobi_2d): `steps`
 * out-of-place applications of out[p] = sum_k weights[k] * in[p + o_k],
 * o_k = offsets[k*ndim .. k*ndim+ndim-1] (axis order as the shape, last
 * axis contiguous), boundary rule `bc`.  Floating dtypes, 1..3 axes,
 * 1 <= npoints <= 32, |offset| <= 4 per axis, steps >= 0.  Rounding: each
 * step is one multiply and FMAs in point order, except on a deferred common
 * weight: a run of two or more steps with a zero or periodic boundary whose
 * weights are exact multiples of one weight f sums the exact ratios w_k / f
 * and applies f^m every m steps, m bounded so that the scaled state grows by
 * at most 2^32 (float64 only).  Such a run keeps finite results for inputs
 * up to the largest double over that growth (about 1.8e299 for the heat
 * step, 1.5e299 for the five-point average).  When the run
 * begins at the first step of its fused group (a stencil node's own steps,
 * or a chain of equal nodes), its first launch records the largest finite
 * |input| it reads, and dcp_sync (or dcp_run_host) returns
 * DCP_E_UNSUPPORTED when that exceeds the run's bound; a run that begins
 * after an epilogue map inside a group is not checked.
 * DCP_OPT_DEFERRED_WEIGHT = 0 selects the plain weighted sum throughout. */
dcp_status dcp_add_stencil(dcp_graph g, dcp_value in, int32_t npoints, const int32_t* offsets,
                           const double* weights, int32_t bc, int32_t steps, dcp_value* out);

/* Reduction of all elements of `in` into a 0-axis value of the same dtype
 * (Sec. 2.3 write-conflict resolution).  SUM of an empty array is 0; the
 * others need >= 1 element (DCP_E_SHAPE otherwise). */
dcp_status dcp_add_reduce(dcp_graph g, dcp_value in, int32_t red, dcp_value* out);

/* Reduction of `in` along one axis (NumPy `x.sum(axis=axis)`): the
 * write-conflict-resolution map of Sec. 2.3 / 3.1 whose result keeps one
 * partial per remaining index (e.g. the row or column sums of a matrix).
 *   axis   0 <= axis < ndim, or -ndim <= axis < 0 counted from the end
 *   out    value of the input's shape with `axis` removed (a 1-axis input
 *          gives a 0-axis value), same dtype
 * Each output is the reduction of the elements along the axis in index
 * order up to reassociation (floating sums); integer sums wrap; MAX/MIN
 * propagate NaN.  SUM along an empty axis gives 0; the others need the axis
 * to be non-empty (DCP_E_SHAPE otherwise).  Elementwise maps producing `in`
 * are fused into the reduction kernel.  dcp_run_adjoint does not support
 * programs containing axis reductions (DCP_E_UNSUPPORTED). */
dcp_status dcp_add_reduce_axis(dcp_graph g, dcp_value in, int32_t red, int32_t axis,
                               dcp_value* out);

/* Marks `v` as a program output; outputs bind to dcp_run's `outputs` array
 * in marking order.  An input may not be marked. */
dcp_status dcp_mark_output(dcp_graph g, dcp_value v);

/* ---- optimisation and execution ---------------------------------------- */

/* Freezes the graph and plans it under `flags` (Sec. 3.1): map fusion,
 * subgraph fusion, time tiling, batching; then generates and compiles one
 * kernel per fused group for sm_103a (Sec. 3.3).  *n_kernels_out (may be
 * NULL) receives the number of kernel launches one dcp_run makes.  Graph
 * mutation after dcp_fuse returns DCP_E_STATE.  Needs no GPU. */
dcp_status dcp_fuse(dcp_graph g, uint32_t flags, int32_t* n_kernels_out);

/* Runs the fused program on `cuda_stream`.  inputs[i] / outputs[j] are
 * device pointers in declaration / marking order.  Transient buffers are
 * allocated on the first run and reused.  With DCP_AUTOTUNE the first run
 * also times the candidate launch configurations of every stencil group (its
 * outputs are the program's; it synchronises the stream).  Asynchronous.
 * For tests, the environment variable DCP_FAULT=alloc (or =launch) makes the
 * next device allocation (kernel launch) fail with DCP_E_OOM (DCP_E_CUDA)
 * before any device work; the graph stays usable. */
dcp_status dcp_run(dcp_graph g, const void* const* inputs, void* const* outputs,
                   void* cuda_stream);

/* As dcp_run, but inputs and outputs are HOST pointers, and the call waits
 * for the stream before returning (then reporting what dcp_sync reports).
 * When every buffer is page-locked (cudaHostAlloc / cudaHostRegister) the
 * kernels read and write the host buffers directly; otherwise the inputs are
 * copied to graph-owned device staging buffers and the outputs copied back
 * (DCP_OPT_HOST_ACCESS). */
dcp_status dcp_run_host(dcp_graph g, const void* const* host_inputs, void* const* host_outputs,
                        void* cuda_stream);

/* Reverse pass (adjoint) of the program: each op's vector-Jacobian
 * product in reverse order, itself fused and run as a dataflow program.
 * out_grads[j] are device cotangents of the outputs (same dtype/shape;
 * 0-axis for reductions); in_grads[i] receive the input cotangents
 * (overwritten).  Floating programs; whole-array SUM reductions; zero and
 * periodic stencil boundaries (DCP_E_UNSUPPORTED otherwise); every map op
 * (max / min route a tie to the operand the forward pass returned).
 * Forward values the reverse rules read are kept on a tape: all of them
 * when they fit in `tape_budget_bytes`, otherwise every ceil(sqrt(S))-th
 * stencil state is kept and each segment recomputed (DCP_E_OOM if even that
 * does not fit).  With DCP_OPT_ADJOINT_DEPTH = k, 1-D / 2-D chains of
 * one-step stencils with epilogue maps run k reverse steps per launch,
 * recomputing each chunk's forward states from every k-th state (the tape
 * then keeps those only); the result is bit for bit that of one launch per
 * step.  Asynchronous on `cuda_stream`. */
dcp_status dcp_run_adjoint(dcp_graph g, const void* const* inputs, const void* const* out_grads,
                           void* const* in_grads, size_t tape_budget_bytes, void* cuda_stream);

/* Plans the reverse pass for `tape_budget_bytes` and compiles its kernels
 * without running it (no GPU needed; the paper compiles a program once and
 * then calls it, Sec. 2.4).  dcp_plan_info then lists the reverse pass's
 * launches; a later dcp_run_adjoint with the same budget reuses the plan.
 * DCP_E_OOM when even sqrt(T) checkpointing exceeds the budget. */
dcp_status dcp_prepare_adjoint(dcp_graph g, size_t tape_budget_bytes);

/* Waits for `cuda_stream` and reports asynchronous CUDA errors,
 * DCP_E_UNSUPPORTED when a deferred common-weight run of the last dcp_run
 * read an input above the magnitude it keeps finite (see dcp_add_stencil;
 * reported once), and DCP_E_TIMEOUT when a cooperative stencil launch gave
 * up waiting for a neighbouring tile (reported once). */
dcp_status dcp_sync(dcp_graph g, void* cuda_stream);

/* Overrides a planner choice (DCP_OPT_*).  Allowed before dcp_fuse (tile and
 * depth keys) or at any time (graph/limit keys). */
dcp_status dcp_set_option(dcp_graph g, int32_t key, int64_t value);

/* Writes a JSON description of the fused plan (groups, kernels, tiles,
 * transients, compile times) into buf (NUL-terminated, truncated to len).
 * *needed (may be NULL) receives the full length + 1. */
dcp_status dcp_plan_info(dcp_graph g, char* buf, size_t len, size_t* needed);

/* Whole-array reduction that allocates no device memory (the paper has no
 * counterpart; it serves callers that cannot allocate: a host application
 * whose pool allocator owns all device memory, an out-of-memory recovery
 * path, or a caller promised a fixed footprint).  Same result as a graph
 * input -> dcp_add_reduce -> output, up to summation order:
 *   in     device array of n elements of `dtype` (aligned to its size)
 *   n      0 <= n <= 2^31 elements; larger n returns DCP_E_INVALID_ARG
 *   red    DCP_SUM / DCP_MAX_R / DCP_MIN_R / DCP_MAXABS (not SUM: n >= 1)
 *   out    device pointer to one element of `dtype`, overwritten
 * Scratch is a fixed array inside the library (512 KiB + 256 B on every
 * device that calls it, kept until the process exits); it never calls
 * cudaMalloc or cudaFree.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress); make that first call outside any
 * CUDA stream capture.  Every call shares the one array, so calls whose
 * work overlaps on the GPU (different streams, no ordering between them)
 * race and give wrong results: order them on one stream.  Asynchronous on
 * `cuda_stream`. */
dcp_status dcp_reduce_noalloc(const void* in, int64_t n, int32_t dtype, int32_t red, void* out,
                              void* cuda_stream);

/* Measurement helper (not a program operation; the paper measures on other
 * hardware): the FP64 arithmetic rate of the current device, the roofline
 * denominator of the binary64 kernels, whose FP64 pipes bound them on GB300.
 * Every SM runs full-occupancy CTAs whose threads advance independent chains
 * of one operation (each with its own operand registers) for about `iters`
 * operations per thread and chain count; 4, 8 and 16 chains per thread are
 * each timed with CUDA events on `cuda_stream` after a shorter warm-up
 * launch, and the best rate is returned.
 *   op     0 = fused multiply-add, 1 = add, 2 = multiply, 3 = add issued as
 *          a fused multiply-add by a run-time 1.0 held in one register for
 *          all chains, 4 = the same with a register of 1.0 per chain (binary64)
 *   iters  1 .. 2^24 operations per chain (8192 runs for tens of ms on GB300)
 *   gops   receives 10^9 lane operations per second (a fused multiply-add
 *          counts once here; it is 2 flops)
 *   ms     (may be NULL) receives the best launch's duration
 * Synchronous: waits for the timed launches.  Allocates nothing (a fixed
 * 64-byte sink inside the library keeps the arithmetic live). */
dcp_status dcp_probe_fp64(int32_t op, int64_t iters, double* gops, double* ms, void* cuda_stream);

/* Thread-local message for the last failing call on this thread. */
const char* dcp_last_error(void);

/* Library version string. */
const char* dcp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DCP_H */
