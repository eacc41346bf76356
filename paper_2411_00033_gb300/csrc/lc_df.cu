// lc_df.cu -- LC_F64_DF: FP64 input and output, Algorithm 4 in double-float
// arithmetic on the FP32 pipe (the kernels of lc_exec_kernels.cuh with
// R = lc_df).  Each vector is scaled by a power of two that brings its
// largest entry into [1, 2) before the double-float arithmetic (exponents
// from k_vec_exponent) and scaled back exactly in the FP64 Step 7.  The plan tables are rounded once from the FP64 plan to
// double-float pairs; A-hat keeps the trailing FP32 word only where the
// entry needs it (the compact layout of lc_internal.cuh).
#include "lc_df.cuh"
#include "lc_exec_kernels.cuh"

namespace lc_exec {
template <>
struct lc_io<lc_df> {
  typedef double type;
};
template <>
__device__ __forceinline__ lc_df lc_ld_in<lc_df, double>(const double* p, int e) {
  return lc_df_from_double_s(*p, e);
}
// Step 7 in FP64: each double-float word is brought back to FP64 exactly
// (times 2^e, undoing the scaling), and the near- and far-field parts are
// summed in FP64: their leading words in FP64, their trailing words (each
// below 2^-24 of its leading word) summed in FP32 first -- an error below
// 2^-48 of those small words -- then added in FP64.
template <>
__device__ __forceinline__ double lc_out1<lc_df, double>(const lc_df& v, int e) {
  return lc_f2d_s(v.hi, e) + lc_f2d_s(v.lo, e);
}
template <>
__device__ __forceinline__ double lc_out2<lc_df, double>(const lc_df& far, const lc_df& near, int e) {
  return (lc_f2d_s(far.hi, e) + lc_f2d_s(near.hi, e)) + lc_f2d_s(far.lo + near.lo, e);
}
template <>
__device__ __forceinline__ double lc_out_acc<lc_df, double>(double acc, const lc_df& v, int e) {
  return (acc + lc_f2d_s(v.hi, e)) + lc_f2d_s(v.lo, e);
}
// The band kernel scales its operand tile by the tile's own exponent.
template <>
struct local_scale<lc_df, double> { static constexpr bool value = true; };
template <>
__device__ __forceinline__ lc_df lc_from_double<lc_df>(double x) { return lc_df_from_double(x); }
template <>
__device__ __forceinline__ lc_df cinv<lc_df>(int64_t i) {
  // 1/pi and 2/pi as double-floats
  return i == 0 ? lc_df(0.31830987334251404f, 1.2841276486597053e-08f)
                : lc_df(0.6366197466850281f, 2.5682552973194106e-08f);
}
// Lean accumulation: the product's error terms and the TwoSum error are
// gathered in acc.lo without renormalising; finish() normalises once.
template <>
__device__ __forceinline__ lc_df acc2<lc_df>(const lc_df& acc, const lc_df& a, const lc_df& b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float t = (acc.hi - (s - bb)) + (p - bb);
  return lc_df(s, acc.lo + (t + e));
}
template <>
__device__ __forceinline__ lc_df acc3<lc_df>(const lc_df& acc, const lc_df& a, const lc_df& b, const lc_df& c) {
  const float p1 = a.hi * b.hi;
  float e1 = fmaf(a.hi, b.hi, -p1);
  e1 = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e1));
  const float p2 = p1 * c.hi;
  float e2 = fmaf(p1, c.hi, -p2);
  e2 = fmaf(p1, c.lo, fmaf(e1, c.hi, e2));
  const float s = acc.hi + p2;
  const float bb = s - acc.hi;
  const float t = (acc.hi - (s - bb)) + (p2 - bb);
  return lc_df(s, acc.lo + (t + e2));
}
template <>
__device__ __forceinline__ lc_df finish<lc_df>(const lc_df& acc) {
  return lc_df_fast2(acc.hi, acc.lo);
}
template <>
struct compact_ahat<lc_df> { static constexpr bool value = true; };
}  // namespace lc_exec

using namespace lc_exec;

namespace {
__global__ void k_d2df(int64_t n, const double* __restrict__ a, lc_df* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double x = a[i];
    const float h = float(x);
    b[i] = lc_df(h, float(x - double(h)));
  }
}
// A-hat for the double-float tier in the compact layout of lc_internal.cuh:
// one thread per entry of the FP64 table (row-major [m][k][l]); the spare
// words at the end of each matrix are zeroed.
__global__ void k_d2df_compact(int64_t nm, int head, int words, const double* __restrict__ a,
                               float* __restrict__ b) {
  const int used = LC_M * LC_M + lc_dfa_rowstart(head + 1, head);
  const int64_t total = nm * LC_M * LC_M;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = i / (LC_M * LC_M);
    const int r = int(i % (LC_M * LC_M));
    const int k = r / LC_M, l = r % LC_M;
    const double x = a[i];
    const float h = float(x);
    float* d = b + m * words;
    d[r] = h;
    if (k + l <= head) d[LC_M * LC_M + lc_dfa_rowstart(k, head) + l] = float(x - double(h));
    if (r < words - used) d[used + r] = 0.0f;
  }
}
unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 65535 * 16) b = 65535 * 16;
  return unsigned(b);
}
}  // namespace

size_t lc_df_bytes(const lc_geom&, int64_t) { return 0; }

lc_status lc_df_prepare(lc_plan p, cudaStream_t st) {
  const lc_geom& g = p->g;
  if (!p->df_tables_direct) {  // else lambda (u, v), T and B were built in double-float
    k_d2df<<<blocks_for(g.N), 256, 0, st>>>(g.N, p->lam, static_cast<lc_df*>(p->df_lam));
    if (p->dir == LC_C2L) k_d2df<<<blocks_for(g.N), 256, 0, st>>>(g.N, p->lam2, static_cast<lc_df*>(p->df_lam2));
    k_d2df<<<1, 256, 0, st>>>(int64_t(2) * g.s * LC_M, p->T, static_cast<lc_df*>(p->df_T));
    k_d2df<<<1, 256, 0, st>>>(LC_M * LC_M, p->B, static_cast<lc_df*>(p->df_B));
  }
  if (g.nc > 0 && !p->df_ahat_direct)
    k_d2df_compact<<<blocks_for(g.nc * LC_M * LC_M), 256, 0, st>>>(
        g.nc, lc_dfa_head(p->dir), lc_dfa_words(p->dir), p->Ahat, static_cast<float*>(p->df_Ahat));
  LC_LAUNCH_CHECK();
  return LC_OK;
}

lc_status lc_exec_df(lc_plan p, const void* in, void* out, const lc_layout& lay, cudaStream_t st, int adjoint) {
  if (p->ragged) return LC_ERR_UNSUPPORTED;
  Args<lc_df> a;
  a.in = static_cast<const double*>(in);
  a.out = static_cast<double*>(out);
  a.ib = lay.ib; a.ie = lay.ie; a.ob = lay.ob; a.oe = lay.oe;
  a.inner = lay.inner; a.iob = lay.iob; a.oob = lay.oob;
  a.n = p->g.n; a.N = p->g.N; a.L = p->g.L; a.s = p->g.s; a.nseg = p->g.nseg;
  a.batch = p->batch; a.dir = int(p->dir);
  a.two_alpha = p->geg.two_alpha;
  a.nodal = 0;
  a.trigger = 0;
  a.t = lc_tables<lc_df>{static_cast<const lc_df*>(p->df_lam), static_cast<const lc_df*>(p->df_lam2),
                         static_cast<const lc_df*>(p->df_T), static_cast<const lc_df*>(p->df_B),
                         static_cast<const lc_df*>(p->df_Ahat), static_cast<lc_df*>(p->df_W),
                         static_cast<lc_df*>(p->df_Cc), p->err, p->opt.debug_flags};
  a.xe = p->xexp;
  a.xe_part = p->xexp_part;
  a.xe_cnt = p->xexp_cnt;
  return run<lc_df>(p, a, st, adjoint);
}
