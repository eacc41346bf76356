// lc_internal.cuh -- shared definitions of the GB300 Legendre<->Chebyshev library.
//
// Geometry (Sec. 3.1 of the paper): L levels gamma = 0..L-1, leaf half-size s,
// h_gamma = s 2^(L-gamma-1), N = s 2^(L+2) (eq:Ntot), b_gamma = 2^(gamma+1)-1
// blocks per level (eq:Nb), N_c = 3 (N/(2s) - L - 2) submatrices
// (eq:total_blocks_and_mats).
//
// Segment trees.  At level gamma the vectors are cut into segments of 2 h_gamma
// entries; segment g covers [2 h g, 2 h (g+1)).  The column blocks of eq:fgamma
// are the segments g = 2b+q+2 (so g >= 2) and the row blocks of eq:zgamma are
// v = 2b+p (so v < 2 b_gamma).  With this numbering the level links eq:flevels
// and eq:zlevels both become "parent = child / 2": f(gamma-1, G) is the union of
// f(gamma, 2G) and f(gamma, 2G+1), and likewise for z.  Submatrix (p, q) of
// block b couples row segment v = 2b+p with column segment g = 2b+q+2.
//
// Arrays w(gamma) and c(gamma) of Algorithm 4 are stored level after level,
// 2^(gamma+2) segments per level (including the two unused ones), each segment
// holding [sigma][k] for the two parities and k < M:
//   seg_offset(gamma) = 4 (2^gamma - 1), total 4 (2^L - 1) segments.
// A-hat(gamma, b, r) is stored at 3 (2^(gamma+1) - 2 - gamma) + 3 b + r.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/legcheb.h"

#define LC_M 18
#define LC_MAX_S 64
#define LC_EXP_CHUNK 2048  // elements per CTA of the double-float tier's exponent pre-pass

struct lc_geom {
  int64_t n;      // logical length (longest member for ragged plans)
  int64_t N;      // padded length s 2^(L+2), or n for direct-only plans
  int32_t L;      // number of levels; 0 means the whole triangle is near field
  int32_t s;      // leaf half-size h_(L-1)
  int64_t nc;     // submatrices
  int64_t nseg;   // segments over all levels, 4 (2^L - 1)
};

__host__ __device__ inline int64_t lc_seg_offset(int gamma) { return 4 * ((int64_t(1) << gamma) - 1); }
__host__ __device__ inline int64_t lc_ahat_offset(int gamma) {
  return 3 * ((int64_t(1) << (gamma + 1)) - 2 - gamma);
}

// Compact double-float A-hat.  Each M x M matrix keeps the FP32 leading
// words of all entries, row-major [k][l], followed by the FP32 trailing
// words of the entries with k + l <= head, row by row (row k holds
// l = 0 .. head - k).  The entries of A-hat are the 2-D Chebyshev
// coefficients of a kernel that is smooth across the well-separated blocks,
// so they fall off geometrically in k + l (by about 4x per step for L2C,
// 3x for C2L); beyond the head every entry is below 4e-9 of the matrix's
// largest for every leaf size s = 4..64 and level (2e-9 for s >= 5; tested),
// and its leading word alone is accurate to 2.4e-16 of that.  Gegenbauer
// kernels (lc_geg) reach 2.2e-8 past the head for -1/2 < a <= 2 (tested),
// so 2e-15 of the matrix.  Words per matrix: a multiple of 4 (16-byte
// bulk copies) with the 3 matrices of a block 28 (L2C) or 12 (C2L) words
// mod 32 apart, so that the blocks staged by one CTA start in distinct
// shared-memory banks.
__host__ __device__ constexpr int lc_dfa_head(int dir) { return dir == LC_L2C ? 13 : 16; }
__host__ __device__ constexpr int lc_dfa_words(int dir) { return dir == LC_L2C ? 436 : 484; }
__host__ __device__ constexpr int lc_dfa_rowstart(int k, int head) { return k * (head + 1) - k * (k - 1) / 2; }

// Memory layout of a batch (strides in elements).  Vector b, element j:
//   input  in[boff(b, ib, inner, iob) + j ie],
//   output out[boff(b, ob, inner, oob) + j oe],
// boff(b, stride, inner, outer) = (b / inner) outer + (b % inner) stride, or
// b stride when inner = 0 (one batch stride).  Two levels reach the fibres of
// a 3-D array along its middle axis in one call.
struct lc_layout {
  int64_t ib, ie, ob, oe;
  int64_t inner, iob, oob;
};
__host__ __device__ __forceinline__ int64_t lc_boff(int64_t b, int64_t stride, int64_t inner, int64_t outer) {
  return inner > 0 ? (b / inner) * outer + (b % inner) * stride : b * stride;
}

// Gegenbauer parameter a of a plan (lc_plan_options.alpha) and the constants
// its tables use.  Legendre plans (a = 1/2) keep on = 0 and the specialised
// Lambda routines.  Gamma(z + p)/Gamma(z + q) at real z is sampled through
// its asymptotic series in v = z + (p + q - 1)/2: v^(p-q) times a power
// series in 1/v^2 (even, because the Stirling expansions of the two log-Gamma
// terms cancel in every odd power); LC_GEG_TERMS + 1 coefficients after the
// argument is shifted to z >= 20 keep the truncation below 2e-18 for
// -1/2 < a <= 2.
#define LC_GEG_TERMS 8
struct lc_geg {
  int on;
  double alpha;
  double two_alpha;  // C2L row factor 2i + 2a (2i + 1 for Legendre)
  double c_lam;      // sqrt(pi) / Gamma(a): lambda_a(z) = c_lam Gamma(z+a)/Gamma(z+1)
  double c_u;        // Gamma(a) / (4 Gamma(-a)): u_a(z) = c_u Gamma(z-a)/Gamma(z+1)
  double u0;         // u_a(0) = Gamma(a)/4
  double v1;         // v_a(1) = 1/Gamma(a+2); v_a(m) = Gamma(m)/Gamma(m+a+1)
  double p_lam[LC_GEG_TERMS + 1];  // series of Gamma(z+a)/Gamma(z+1)
  double p_u[LC_GEG_TERMS + 1];    // series of Gamma(z-a)/Gamma(z+1)
  double p_v[LC_GEG_TERMS + 1];    // series of Gamma(z)/Gamma(z+a+1)
};

// Device views of a plan's tables, by element type.
template <typename R>
struct lc_tables {
  // Legendre: L2C lambda[N]; C2L u[N] = lambda_k / (1 - 2k).  Gegenbauer a:
  // L2C sqrt(pi) (a)_k / k! (so that the Legendre C^{-1} applies unchanged);
  // C2L u_k = Gamma(a)/4 (-a)_k / k!.
  const R* lam;
  // L2C: lam again; C2L: v[N] = 1 / (2m (2m+1) lambda_m) (Legendre) or
  // Gamma(m)/Gamma(m+a+1) (Gegenbauer), v[0] = 0.  C2L entries are
  // (2i + 2a) j u_k v_(i+k).
  const R* lam2;
  const R* T;     // [2][s][M]   T_k(-1 + (2m+sigma)/s)           (eq:Xs)
  const R* B;     // [M][M]      B(0), lower triangular           (eq:Tmap)
  const R* Ahat;  // [nc][M][M]
  R* W;           // [batch][nseg][2][M]   w of Algorithm 4
  R* Cc;          // [batch][nseg][2][M]   c of Algorithm 4
  int* err;       // device status word (bounded waits that ran out)
  int debug;      // lc_plan_options.debug_flags
};

struct lc_plan_s {
  lc_geom g;
  lc_direction dir;
  lc_dtype dtype;
  int64_t batch;
  lc_plan_options opt;
  lc_geg geg;
  int ragged;
  // FP64 tables (always built; they are the plan).
  double* lam;
  double* lam2;
  double* T;
  double* B;
  double* Ahat;
  double* W;
  double* Cc;
  // FP32 copies for LC_F32.
  float* lamf;
  float* lam2f;
  float* Tf;
  float* Bf;
  float* Ahatf;
  float* Wf;
  float* Ccf;
  // Double-float (hi, lo) copies for LC_F64_DF: stored as float2.
  void* df_lam;
  void* df_lam2;
  void* df_T;
  void* df_B;
  void* df_Ahat;
  int df_ahat_direct;    // df_Ahat built by the double-float plan kernel (no FP64 A-hat)
  int df_tables_direct;  // df_lam (df_lam2), df_T, df_B built at plan time in double-float (no FP64 lambda, u, v)
  void* df_W;
  void* df_Cc;
  // Per-vector exponents of the double-float tier and the pre-pass's
  // partial maxima / arrival counters (counters zeroed at plan time).
  int* xexp;
  int* xexp_part;
  unsigned* xexp_cnt;
  // Values at Chebyshev points (lc_values.cu): twiddle tables, and for C2L
  // plans a [batch][n] buffer for the Chebyshev coefficients of the input.
  void* val_tables;
  double* val_scratch;
  void* val_work;  // large n: the [batch][n] complex work array of the two FFT passes, exponents
  // Split tier data (see lc_split.cu).
  void* split;
  // Ragged members (host copies and device tables).
  int64_t count;
  int64_t* h_len;
  int64_t* h_off;
  void* ragged_dev;
  // Split tier schedule: 1 = one persistent launch (when its task lists
  // could be built), 0 = level-by-level launches; CTAs of the persistent launch.
  int split_sched;
  int split_grid;
  size_t bytes_used;
  int* err;  // device status word in the workspace
  // Side stream and fork/join events used to overlap independent kernels of
  // one execution (host objects; created at plan time).
  cudaStream_t side;    // coarse-level chain (highest priority)
  cudaStream_t fine;    // far-field chain of the fine levels (next priority)
  cudaStream_t nearst;  // near-field band (lowest priority)
  cudaEvent_t ev_fork, ev_join, ev_start, ev_near, ev_done;
  // Chunk geometry of the CUDA-core tiers (lc_plan_autotune / lc_plan_set_config).
  int leaf_depth, chunk_depth;
  // Single-vector band launch (lc_plan_set_band): CTAs of k_near (0: one per
  // group of strips) and whether it starts after the first up chunk.
  int band_ctas, band_after_leaf;
  // Optional per-kernel timing (lc_plan_set_timing).
  int timing_slots;
  int timing_stride;       // events per slot
  cudaEvent_t* events;     // [slots][stride]
  int32_t* kinds;          // [slots][stride]
  int* marks;              // events recorded per slot
  int64_t exec_counter;
  int cur_slot;
};

// Timing marks: call lc_timer_begin once per execution, lc_timer_mark before
// each kernel (with its kind) and lc_timer_end after the last one.
enum { LC_K_LEAF = 0, LC_K_UP = 1, LC_K_COUPLE = 2, LC_K_DOWN = 3, LC_K_FINAL = 4, LC_K_PREP = 5, LC_K_OTHER = 6,
       LC_K_NEAR = 7 };
inline void lc_timer_begin(lc_plan_s* p) {
  if (p->timing_slots <= 0) return;
  p->cur_slot = int(p->exec_counter++ % p->timing_slots);
  p->marks[p->cur_slot] = 0;
}
inline void lc_timer_mark(lc_plan_s* p, cudaStream_t st, int kind) {
  if (p->timing_slots <= 0) return;
  int& m = p->marks[p->cur_slot];
  if (m >= p->timing_stride - 1) return;
  cudaEventRecord(p->events[p->cur_slot * p->timing_stride + m], st);
  p->kinds[p->cur_slot * p->timing_stride + m] = kind;
  ++m;
}
inline void lc_timer_end(lc_plan_s* p, cudaStream_t st) {
  if (p->timing_slots <= 0) return;
  int& m = p->marks[p->cur_slot];
  cudaEventRecord(p->events[p->cur_slot * p->timing_stride + m], st);
  p->kinds[p->cur_slot * p->timing_stride + m] = -1;
  ++m;
}

// ---- programmatic dependent launch -------------------------------------------
// A kernel launched with cudaLaunchAttributeProgrammaticStreamSerialization
// may be scheduled while its predecessor in the stream is still running;
// lc_grid_wait() returns once the predecessor has completed and its memory
// is visible, so such a kernel calls it before it reads or writes data other
// kernels share (plan tables and the caller's input only before).
// lc_grid_trigger() lets the successor be scheduled once every CTA of this
// grid has called it or exited.  Both are no-ops without the attribute.
__device__ __forceinline__ void lc_grid_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void lc_grid_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ---- error helpers ---------------------------------------------------------
#define LC_CUDA_TRY(expr)                        \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return LC_ERR_CUDA;   \
  } while (0)
#define LC_LAUNCH_CHECK() LC_CUDA_TRY(cudaGetLastError())

// ---- geometry / plan helpers (lc_plan.cu) -----------------------------------
lc_status lc_compute_geometry(int64_t n, const lc_plan_options* opt, int fixed_default, lc_geom* g);

// ---- execution entry points (lc_exec.cu) ------------------------------------
lc_status lc_exec_cuda_cores(lc_plan p, const void* in, void* out, const lc_layout& lay, cudaStream_t st,
                             int adjoint);
int lc_exec_cuda_cores_launches(const lc_plan_s* p);

// ---- double-float tier (lc_df.cu) -------------------------------------------
lc_status lc_df_prepare(lc_plan p, cudaStream_t st);
lc_status lc_exec_df(lc_plan p, const void* in, void* out, const lc_layout& lay, cudaStream_t st, int adjoint);
size_t lc_df_bytes(const lc_geom& g, int64_t batch);

// ---- split tier (lc_split.cu) ------------------------------------------------
size_t lc_split_bytes(const lc_plan_s* p);
lc_status lc_split_prepare(lc_plan p, char* base, size_t bytes, cudaStream_t st);
lc_status lc_exec_split(lc_plan p, const void* in, void* out, const lc_layout& lay, cudaStream_t st,
                        int adjoint);
int lc_exec_split_launches(const lc_plan_s* p);
bool lc_split_persistent(const lc_plan_s* p);
void lc_split_release(lc_plan p);

// ---- values at Chebyshev points (lc_values.cu) -------------------------------
bool lc_values_supported(int64_t n);
size_t lc_values_table_bytes(int64_t n);
size_t lc_values_work_bytes(int64_t n, int64_t batch);
int lc_values_launches(const lc_plan_s* p);
lc_status lc_values_prepare(lc_plan p, cudaStream_t st);
lc_status lc_values_synth(lc_plan p, double* out, const lc_layout& lay, cudaStream_t st);
lc_status lc_values_analysis(lc_plan p, const double* in, const lc_layout& lay, double* scratch, cudaStream_t st);

// ---- autotuning cache (lc_tune.cu) ------------------------------------------
void lc_tune_apply_cached(lc_plan p);
