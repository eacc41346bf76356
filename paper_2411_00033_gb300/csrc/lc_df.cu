// lc_df.cu -- LC_F64_DF: FP64 input and output, Algorithm 4 in double-float
// arithmetic on the FP32 pipe (the kernels of lc_exec_kernels.cuh with
// R = lc_df).  The plan tables are rounded once from the FP64 plan to
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
__device__ __forceinline__ lc_df lc_ld<lc_df, double>(const double* p) {
  return lc_df_from_double(*p);
}
template <>
__device__ __forceinline__ void lc_st<lc_df, double>(double* p, const lc_df& v) {
  *p = lc_df_to_double(v);
}
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
  k_d2df<<<blocks_for(g.N), 256, 0, st>>>(g.N, p->lam, static_cast<lc_df*>(p->df_lam));
  if (p->dir == LC_C2L) k_d2df<<<blocks_for(g.N), 256, 0, st>>>(g.N, p->lam2, static_cast<lc_df*>(p->df_lam2));
  k_d2df<<<1, 256, 0, st>>>(int64_t(2) * g.s * LC_M, p->T, static_cast<lc_df*>(p->df_T));
  k_d2df<<<1, 256, 0, st>>>(LC_M * LC_M, p->B, static_cast<lc_df*>(p->df_B));
  if (g.nc > 0)
    k_d2df_compact<<<blocks_for(g.nc * LC_M * LC_M), 256, 0, st>>>(
        g.nc, lc_dfa_head(p->dir), lc_dfa_words(p->dir), p->Ahat, static_cast<float*>(p->df_Ahat));
  LC_LAUNCH_CHECK();
  return LC_OK;
}

lc_status lc_exec_df(lc_plan p, const void* in, void* out, int64_t ib, int64_t ie, int64_t ob, int64_t oe,
                     cudaStream_t st, int adjoint) {
  if (p->ragged) return LC_ERR_UNSUPPORTED;
  Args<lc_df> a;
  a.in = static_cast<const double*>(in);
  a.out = static_cast<double*>(out);
  a.ib = ib; a.ie = ie; a.ob = ob; a.oe = oe;
  a.n = p->g.n; a.N = p->g.N; a.L = p->g.L; a.s = p->g.s; a.nseg = p->g.nseg;
  a.batch = p->batch; a.dir = int(p->dir);
  a.t = lc_tables<lc_df>{static_cast<const lc_df*>(p->df_lam), static_cast<const lc_df*>(p->df_lam2),
                         static_cast<const lc_df*>(p->df_T), static_cast<const lc_df*>(p->df_B),
                         static_cast<const lc_df*>(p->df_Ahat), static_cast<lc_df*>(p->df_W),
                         static_cast<lc_df*>(p->df_Cc), p->err, p->opt.debug_flags};
  return run<lc_df>(p, a, st, adjoint);
}
