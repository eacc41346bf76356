/*
 * legcheb.h -- C ABI of the GB300 fast multipole Legendre<->Chebyshev transform.
 *
 * The library computes the connection maps of Mortensen, "A faster multipole
 * Legendre-Chebyshev transform" (arXiv:2411.00033), Sec. 1, eq:directmv:
 *
 *   LC_L2C:  f_cheb = C^{-1} A f_leg        (Legendre -> Chebyshev coefficients)
 *   LC_C2L:  f_leg  = A^{-1} C f_cheb       (Chebyshev -> Legendre coefficients)
 *
 * with a_ij = Lambda((j-i)/2) Lambda((j+i)/2) for j >= i, j-i even, else 0
 * (eq:aij), Lambda(x) = Gamma(x+1/2)/Gamma(x+1) (eq:Lambda) and
 * C = diag(c_i pi/2), c_0 = 2, c_i = 1.  The C2L matrix has the entries
 * L(i,j) of eq:Lxymod, with entry (0,0) equal to 1.
 *
 * The execution stage follows Algorithm 4 (Sec. 4.1): a direct near-field
 * band (Step 6, Algorithm 1 restricted to the band), and the far-field
 * blocks of the level hierarchy of Sec. 3.1 applied through Chebyshev
 * expansions of order M = 18 (Steps 1-5), with the triangular translation
 * matrices B(0), B(1) of eq:wtk / Appendix A.3 moving expansions between
 * neighbouring levels, and the scaling C^{-1} (Step 7).
 *
 * Conventions shared by every call:
 *  - All device pointers are plain CUDA device addresses; the library never
 *    allocates device memory.  The caller provides a workspace for each plan
 *    (sized by lc_plan_workspace_size*) and keeps it alive, unmodified, until
 *    lc_destroy.  The plan object itself is host memory owned by the library.
 *  - Every call returns an lc_status; nothing aborts.  A CUDA error seen by a
 *    call is returned as LC_ERR_CUDA; asynchronous device faults surface at a
 *    later call or synchronisation.
 *  - Work is enqueued on the caller's stream; no call synchronises the host
 *    except where stated.  lc_execute and lc_adjoint neither allocate nor
 *    synchronise; they may fork independent kernels onto streams owned by
 *    the plan (at other priorities) and join them back (events) into the
 *    caller's stream before returning, so the caller sees ordinary stream
 *    order, also under stream capture.
 *  - One plan executes on one stream at a time: its intermediate arrays live
 *    in the plan workspace, so two executions of the same plan must not
 *    overlap on the device.
 *  - Input and output must not alias.  Inputs of length n are treated as
 *    zero-padded to the plan's internal length N >= n (Sec. 3.1,
 *    eq:numlevels); padding cannot change the first n outputs because A is
 *    upper triangular.
 */
#ifndef LEGCHEB_H
#define LEGCHEB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lc_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  LC_L2C = 0, /* f_cheb = C^{-1} A f_leg */
  LC_C2L = 1  /* f_leg  = A^{-1} C f_cheb */
} lc_direction;

typedef enum {
  /* FP64 in and out; every product and sum in FP64 on the FP64 pipe. */
  LC_F64 = 0,
  /* FP64 in and out, FP64-accurate; the block products run on the bf16 tensor
   * cores as exact 8-bit slice products with FP32 accumulation, recombined in
   * FP64 (split-precision tier). */
  LC_F64_SPLIT = 1,
  /* FP32 in and out; FP32 arithmetic (plan built in FP64, rounded once). */
  LC_F32 = 2,
  /* FP64 in and out, FP64-accurate; double-float (pairs of FP32) arithmetic
   * on the FP32 pipe for a single vector or small batches. */
  LC_F64_DF = 3
} lc_dtype;

typedef enum {
  LC_OK = 0,
  LC_ERR_INVALID_ARG = 1,         /* a size, enum, pointer or stride is invalid */
  LC_ERR_WORKSPACE_TOO_SMALL = 2, /* workspace bytes below lc_plan_workspace_size */
  LC_ERR_CUDA = 3,                /* a CUDA runtime call or launch failed */
  LC_ERR_DEVICE_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  LC_ERR_UNSUPPORTED = 5,         /* valid request the library does not implement */
  LC_ERR_HOST_ALLOC = 6           /* host memory for the plan object ran out */
} lc_status;

typedef struct lc_plan_s* lc_plan;

/* Plan options.  Defaults (lc_plan_options_default) follow the paper:
 * s_hat = 32 and s = ceil(n / 2^(L+2)) with L = ceil(log2(n/s_hat)) - 2
 * (eq:numlevels), so s lies in [s_hat/2, s_hat]. */
typedef struct {
  int32_t s_hat;   /* target leaf half-size (eq:numlevels); 4 <= s_hat <= 64 */
  int32_t fixed_s; /* > 0: use this s for every length (4 <= fixed_s <= 64); 0: paper rule */
  int32_t slices;  /* LC_F64_SPLIT: 8-bit slices per operand, 3..7, or 0 (default):
                    * 7 for n <= 1e5 (normwise relative error <= 1e-13),
                    * 6 above (<= 1e-12); for ragged plans n is the longest member */
  /* Testing only (0 in normal use).  Bit 0: the coupling kernel withholds
   * one of its bulk copies, so its bounded wait runs out and the execution
   * reports LC_ERR_DEVICE_TIMEOUT through lc_plan_check.  Bit 1 (split tier,
   * persistent schedule): one task waits for a write its row block never
   * receives; its bounded wait runs out, the launch aborts, and
   * lc_plan_check reports LC_ERR_DEVICE_TIMEOUT. */
  int32_t debug_flags;
  /* 1: the Chebyshev side holds values at the n Chebyshev-Gauss points
   * x_m = cos((m + 1/2) pi / n), m = 0 .. n-1, instead of Chebyshev
   * coefficients (Sec. 1: the Chebyshev-Legendre Galerkin use, point values
   * through fast cosine transforms).  LC_L2C then gives out_m = p(x_m) for
   * p = sum_j in_j P_j (Legendre synthesis on Chebyshev points); LC_C2L takes
   * in_m = p(x_m) and gives the Legendre coefficients of the degree < n
   * polynomial through those values.  The cosine transforms are FFTs of
   * length n: for powers of two, one CTA per vector up to n = 4096 and two
   * passes through a work array in the plan's workspace above; for other n,
   * Bluestein's chirp convolution through FFTs of the next power of two
   * m >= 2n - 1.  n must satisfy 2 <= n <= LC_VALUES_MAX_N (powers of two) or
   * 2 <= n <= LC_VALUES_MAX_N_ANY (others), the tier LC_F64, LC_F64_DF or LC_F64_SPLIT,
   * the plan uniform (not ragged); otherwise plan creation returns
   * LC_ERR_UNSUPPORTED.  lc_adjoint of such a plan returns
   * LC_ERR_UNSUPPORTED.  0 (default): coefficients. */
  int32_t values;
  /* 1: the nodal variant (eq:AijLag; the original method of Alpert and
   * Rokhlin that the paper's modal method replaces): every far-field block is
   * represented by the kernel's values at the M x M Chebyshev-Gauss node
   * pairs of the block with Lagrange bases instead of 2-D Chebyshev
   * coefficients, the leaf matrices hold the Lagrange basis at the leaf
   * points, and the level-to-level maps of Steps 2 and 4 are the two dense
   * M x M Lagrange interpolation matrices between a parent's and its
   * children's nodes instead of the triangular B(0), B(1).  The same linear
   * map to the same accuracy; planning skips the 2-D DCT, execution does
   * dense level maps.  LC_F64 and LC_F32 only (otherwise plan creation
   * returns LC_ERR_UNSUPPORTED).  0 (default): the modal method. */
  int32_t nodal;
  /* LC_F64_DF: 1 builds the tier's double-float A-hat by converting the FP64
   * plan's (eq:aklmore on the FP64 pipe); 0 (default) computes it in
   * double-float arithmetic on the FP32 pipe, about 10x faster on GB300,
   * for Legendre plans with s >= 10 (others always take the FP64 route).
   * The entries agree to a few units of 2^-48 of their matrix. */
  int32_t fp64_plan;
  int32_t reserved[1];
  /* Gegenbauer parameter a of the non-Chebyshev side (Conclusions: the
   * method carries over to Gegenbauer bases).  0 (default) or 0.5: Legendre,
   * P_j = C_j^(1/2).  Otherwise -1/2 < a <= LC_GEGENBAUER_MAX_ALPHA, a != 0:
   * LC_L2C maps coefficients of C_j^(a) to Chebyshev coefficients, with
   * entries (2/c_i) g_l g_m, g_k = (a)_k / k!, l = (j-i)/2, m = (j+i)/2 (the
   * generating function of C^(a) at x = cos t); LC_C2L is its inverse, with
   * entries (2i + 2a) j u_l w_m / (4a(a+1)), u_l = (-a)_l / l!,
   * w_m = (m-1)!/(a+2)_{m-1}, entry (0,0) = 1.  The far-field kernels are
   * the same products of Gamma ratios at real arguments, sampled through
   * their asymptotic series; every tier, adjoints, ragged plans and the
   * values option accept it.  Anything else returns LC_ERR_INVALID_ARG. */
  double alpha;
} lc_plan_options;
#define LC_GEGENBAUER_MAX_ALPHA 2.0
#define LC_VALUES_MAX_N 4194304
#define LC_VALUES_MAX_N_ANY 2097152

/* Fill *opt with the defaults above.  Returns LC_ERR_INVALID_ARG for NULL. */
lc_status lc_plan_options_default(lc_plan_options* opt);

/* Device bytes the caller must provide to lc_plan_create for a plan of
 * `batch` vectors of length n (n >= 1, batch >= 1).  The size covers the
 * plan tables (lambda, Vandermonde T, B, the N_c coefficient matrices A-hat
 * of eq:aklmore) and the per-vector level arrays w, c of Algorithm 4.
 * opt may be NULL (defaults). */
lc_status lc_plan_workspace_size(int64_t n, lc_direction direction, int64_t batch,
                                 lc_dtype dtype, size_t* bytes);
lc_status lc_plan_workspace_size_ex(int64_t n, lc_direction direction, int64_t batch,
                                    lc_dtype dtype, const lc_plan_options* opt,
                                    size_t* bytes);

/* Build a plan in `workspace` (device memory, 256-byte aligned, `bytes` >=
 * the size above) on `stream`: lambda by the tau series every 8th entry and
 * the recursion of eq:Lambdaint in between, T(sigma) of eq:Xs, B(0) exactly
 * (Appendix A.3), and A-hat for every submatrix by sampling the kernel
 * (A(x,y) for L2C, L(x,y) of eq:Lxymod for C2L) at M x M Chebyshev-Gauss
 * points and applying the 2-D DCT-II of eq:aklmore.  All in FP64 on the
 * GPU.  The plan is usable by later calls on the same stream (or after the
 * caller synchronises).  *out receives a host object freed by lc_destroy. */
lc_status lc_plan_create(lc_plan* out, int64_t n, lc_direction direction, int64_t batch,
                         lc_dtype dtype, void* workspace, size_t bytes, lc_stream stream);
lc_status lc_plan_create_ex(lc_plan* out, int64_t n, lc_direction direction, int64_t batch,
                            lc_dtype dtype, const lc_plan_options* opt, void* workspace,
                            size_t bytes, lc_stream stream);

/* Ragged batch: `count` transforms of lengths n[0..count-1] (host array,
 * each >= 1), packed back to back in input and output (member t starts at
 * sum_{u<t} n[u]).  All members share one coefficient table built for the
 * largest length with a fixed s (opt->fixed_s, default 32), since A-hat of a
 * submatrix depends only on its position in A (eq:globalij), so every
 * shorter plan is a corner of the largest one. */
lc_status lc_plan_workspace_size_ragged(const int64_t* n, int64_t count, lc_direction direction,
                                        lc_dtype dtype, const lc_plan_options* opt,
                                        size_t* bytes);
lc_status lc_plan_create_ragged(lc_plan* out, const int64_t* n, int64_t count,
                                lc_direction direction, lc_dtype dtype,
                                const lc_plan_options* opt, void* workspace, size_t bytes,
                                lc_stream stream);

/* Apply the plan's map to `batch` vectors (the plan's batch):
 *   out[b*out_batch_stride + i*out_elem_stride] = (map x_b)_i, i < n,
 *   x_b[j] = in[b*in_batch_stride + j*in_elem_stride].
 * Element type: double for LC_F64 / LC_F64_SPLIT / LC_F64_DF, float for
 * LC_F32.  Strides are in elements and may be any non-negative values that
 * keep the vectors disjoint in `out` (this is how fibres of a 2-D/3-D array
 * along any axis are transformed in place of a transpose).  For ragged plans
 * both batch strides must be 0 and both element strides 1 (packed layout).
 * Asynchronous on `stream`; no allocation, no host synchronisation. */
lc_status lc_execute(lc_plan plan, const void* in, void* out, int64_t in_batch_stride,
                     int64_t in_elem_stride, int64_t out_batch_stride,
                     int64_t out_elem_stride, lc_stream stream);

/* Apply the transpose of the plan's map (same layout rules as lc_execute):
 *   L2C plan: out = A^T C^{-1} in ;  C2L plan: out = (A^{-1} C)^T in.
 * Not in the paper: it runs Algorithm 4 backwards (C^{-1} first, leaf
 * restriction on the row side, upward pass over the row tree, A-hat
 * transposed, downward pass over the column tree, transposed band).
 * Every tier, uniform, strided and ragged plans alike. */
lc_status lc_adjoint(lc_plan plan, const void* in, void* out, int64_t in_batch_stride,
                     int64_t in_elem_stride, int64_t out_batch_stride,
                     int64_t out_elem_stride, lc_stream stream);

/* Two-level batches: vector b (0 <= b < the plan's batch) and its element j
 * are read from and written to
 *   in [(b / batch_inner) * in_outer_stride  + (b % batch_inner) * in_batch_stride  + j * in_elem_stride]
 *   out[(b / batch_inner) * out_outer_stride + (b % batch_inner) * out_batch_stride + j * out_elem_stride]
 * (strides in elements, all >= 0, 1 <= batch_inner <= batch; batch_inner
 * equal to the batch is lc_execute / lc_adjoint).  This reaches, in one call,
 * the fibres of a 3-D array along its middle axis (C order, shape (P, n, Q):
 * batch P*Q, batch_inner Q, batch stride 1, element stride Q, outer stride
 * n*Q), which no single batch stride can.  Ragged plans accept only
 * batch_inner = count with their packed layout.  Output strides that would
 * put two outputs on one address (a zero stride that is used) return
 * LC_ERR_INVALID_ARG. */
lc_status lc_execute_ex(lc_plan plan, const void* in, void* out, int64_t in_batch_stride,
                        int64_t in_elem_stride, int64_t out_batch_stride, int64_t out_elem_stride,
                        int64_t batch_inner, int64_t in_outer_stride, int64_t out_outer_stride,
                        lc_stream stream);
lc_status lc_adjoint_ex(lc_plan plan, const void* in, void* out, int64_t in_batch_stride,
                        int64_t in_elem_stride, int64_t out_batch_stride, int64_t out_elem_stride,
                        int64_t batch_inner, int64_t in_outer_stride, int64_t out_outer_stride,
                        lc_stream stream);

/* Device-side status of the plan's earlier executions.  Kernels that wait on
 * an asynchronous copy (mbarrier) give up after about one second, record the
 * failure in a status word of the workspace and exit.  This call
 * synchronises `stream`, returns LC_ERR_DEVICE_TIMEOUT if any such failure
 * was recorded since the last check (and clears it), else LC_OK. */
lc_status lc_plan_check(lc_plan plan, lc_stream stream);

/* Chunk geometry of the CUDA-core tiers (LC_F64, LC_F32, LC_F64_DF).  The
 * levels of Algorithm 4 are processed in subtrees, one CTA per subtree:
 * leaf_depth = levels the first upward chunk climbs from the leaves (and the
 * last downward chunk descends), chunk_depth = levels per coarser chunk;
 * leaf_depth 1..6, chunk_depth 1..8, defaults 4 and 4.  The results do not
 * depend on them. */
lc_status lc_plan_set_config(lc_plan plan, int32_t leaf_depth, int32_t chunk_depth);

/* Launch shape of the near-field band (Step 6) of single-vector plans on the
 * CUDA-core tiers: ctas = number of CTAs of the band kernel, each taking
 * groups of 16 strips of 2s rows in turn (0, the default: one CTA per
 * group; fewer leave SM room for the far-field chain that runs beside it);
 * after_leaf = 1 starts the band only after the leaf restriction and the
 * fine levels of Step 2, 0 (default) with them.  Results do not depend on
 * either.  LC_ERR_INVALID_ARG for a NULL plan, ctas < 0 or > 2^24, or
 * after_leaf not 0 or 1. */
lc_status lc_plan_set_band(lc_plan plan, int32_t ctas, int32_t after_leaf);

/* Schedule of the split-precision tier (LC_F64_SPLIT, uniform and ragged
 * batches).  persistent = 1 (the default): Steps 1-4 of Algorithm 4 -- leaf,
 * upward levels, coupling, downward levels -- run as ONE persistent kernel
 * launch whose CTAs draw tasks (a level, a segment, a tile of members) from
 * a device ticket counter; a task waits (bounded) only for the row blocks
 * it reads, counted by per-block write counters, so tasks of different
 * levels and member tiles overlap; the ticket order is a list schedule of
 * the task graph built at plan time (longest chain of dependants first).
 * The final stage (Steps 5-7) is the second launch.  persistent = 0 runs
 * one kernel launch per level (what lc_plan_set_timing breaks down per
 * kind).  Results are bitwise the same.  A failed bounded wait aborts the
 * execution and is reported by lc_plan_check.  LC_ERR_INVALID_ARG for a
 * NULL plan or a value other than 0 or 1; LC_ERR_UNSUPPORTED for other
 * tiers, or for persistent = 1 when the plan's task lists could not be
 * built (the plan then keeps the level launches). */
lc_status lc_plan_set_split_schedule(lc_plan plan, int32_t persistent);

/* Autotuner (not in the paper): time every candidate chunk geometry
 * (leaf_depth in {3,4,5} x chunk_depth in {3,4,6}) on the given input with
 * CUDA events on `stream` (synchronises it; `out` is overwritten, same layout
 * rules as lc_execute), keep the fastest in the plan, and cache it for this
 * process under the plan's shape (n, batch, L, s, dtype, direction); plans of
 * the same shape created later start from the cached choice.  Outputs may be
 * NULL.  Plans without a tunable geometry (split tier, ragged, L <= 1) return
 * LC_OK unchanged. */
lc_status lc_plan_autotune(lc_plan plan, const void* in, void* out, int64_t in_batch_stride,
                           int64_t in_elem_stride, int64_t out_batch_stride, int64_t out_elem_stride,
                           lc_stream stream, int32_t* leaf_depth, int32_t* chunk_depth, float* best_ms);

/* Free the host plan object.  The workspace stays the caller's. */
lc_status lc_destroy(lc_plan plan);

/* Static text for a status code (never NULL). */
const char* lc_status_string(lc_status status);

/* Plan geometry (Sec. 3.1): n, padded N, levels L, leaf half-size s,
 * expansion order M, number of submatrices N_c (eq:total_blocks_and_mats),
 * batch.  Any output pointer may be NULL. */
lc_status lc_plan_info(lc_plan plan, int64_t* n, int64_t* N, int32_t* L, int32_t* s,
                       int32_t* M, int64_t* n_c, int64_t* batch);

/* Copy plan tables to host memory for inspection (synchronises `stream`):
 * which = 0: lambda[N]; 1: T[2][s][M]; 2: B(0)[M][M]; 3: A-hat[N_c][M][M]
 * (row k = expansion in the row variable X, column l in Y, eq:Aij); C2L
 * plans: 4: u[N], 5: v[N].  Nodal plans: 1 holds the Lagrange basis at the
 * leaf points, 2 the level maps P(0), P(1) ([2][M][M]) and 3 the kernel at
 * the node pairs of each block (eq:AijLag).  LC_F64_DF plans: 6 copies the
 * compact double-float A-hat as raw FP32 words, two per double of dst
 * (N_c matrices of 436 (L2C) or 484 (C2L) words: the leading words of all
 * entries row-major, then the trailing words of the entries with
 * k + l <= 13 (L2C) or 16 (C2L), row by row); 3 returns LC_ERR_UNSUPPORTED
 * when that copy was built without the FP64 table (lc_plan_options.fp64_plan).
 * `count` is the capacity of dst in doubles; the number copied is returned
 * in *copied. */
lc_status lc_plan_table(lc_plan plan, int32_t which, double* dst, int64_t count,
                        int64_t* copied, lc_stream stream);

/* Number of kernels one lc_execute of this plan launches. */
lc_status lc_plan_launches(lc_plan plan, int32_t* launches);

/* Per-kernel timing with CUDA events (diagnostics, off by default).
 * slots > 0 creates slots x (launches + 1) events (host API, no device
 * memory); every later lc_execute / lc_adjoint records one event before
 * each of its kernels and one after the last, into the next slot (round
 * robin).  slots = 0 destroys the events and switches timing off.
 * Not for use while the stream is being captured into a CUDA graph. */
lc_status lc_plan_set_timing(lc_plan plan, int32_t slots);

/* Kernel durations (ms) of the execution recorded in `slot`; waits for its
 * events.  kinds[i] names kernel i: 0 leaf restriction (Step 1),
 * 1 upward pass (Step 2), 2 coupling (Step 3), 3 downward pass (Step 4),
 * 4 leaf spread (Step 5) + far/near sum + scaling, 5 input preparation,
 * 6 other, 7 near-field band (Steps 6-7; with the split tier, kind 4 also
 * covers the band).  ms and kinds may be NULL; *count receives the kernel
 * count.  With timing on, the kernels run one after another on the
 * caller's stream; without it they overlap on the plan's streams. */
lc_status lc_plan_get_timing(lc_plan plan, int32_t slot, float* ms, int32_t* kinds, int32_t capacity,
                             int32_t* count);

/* ---- Transform without any device allocation ------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory (a plugin inside an application whose memory
 * pool owns the device, a latency-critical loop that cannot afford the
 * device-wide synchronisation cudaMalloc may cause, a deployment that
 * reserves all memory at load time).  It computes the same maps as
 * lc_execute, out[b][i] = (M x_b)_i for i < n with M = C^{-1}A (LC_L2C) or
 * A^{-1}C (LC_C2L), FP64 in and out, by the direct O(n^2) sum over the whole
 * upper triangle.  Its scratch (the Lambda table) lives in a file-scope
 * __device__ array of LC_STATIC_MAX_N x 2 doubles (256 KiB) that every GPU
 * loading the library holds until the process exits; it calls no cudaMalloc
 * or cudaFree.
 *  - n > LC_STATIC_MAX_N (or n < 1, batch < 1, NULL or aliased pointers,
 *    negative strides, a zero output element stride with n > 1 or a zero
 *    output batch stride with batch > 1) returns LC_ERR_INVALID_ARG and
 *    launches nothing.
 *  - Pointers, strides and batch follow lc_execute; x and out are device
 *    memory of the caller.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (once per device, with that device current); make
 *    that first call before any stream capture begins.
 *  - All calls share the one array: calls whose executions overlap on the
 *    GPU (different streams, or concurrent host threads) race on it and give
 *    wrong results.  Calls ordered on one stream are safe; each call rewrites
 *    the part of the table it reads before reading it. */
#define LC_STATIC_MAX_N 16384
lc_status lc_direct_static(lc_direction direction, int64_t n, int64_t batch, const double* in, double* out,
                           int64_t in_batch_stride, int64_t in_elem_stride, int64_t out_batch_stride,
                           int64_t out_elem_stride, lc_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* LEGCHEB_H */
