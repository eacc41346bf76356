// lc_values.cu -- values at Chebyshev points: the Legendre synthesis on the
// n Chebyshev-Gauss points x_m = cos((m + 1/2) pi / n) (an L2C plan with the
// option `values`: out = p(x_m) for p = sum_j f_j P_j) and its inverse (a C2L
// plan with `values`: in = p(x_m), out = the Legendre coefficients of the
// degree < n polynomial through them).  Sec. 1 of the paper motivates the
// transform by exactly this use: Chebyshev coefficients reach point values
// through fast cosine transforms.
//
// The cosine transforms, for n a power of two:
//   synthesis  v_m = sum_k c_k cos(pi k (2m+1) / (2n))         (after L2C)
//   analysis   c_k = (2/n)/(1 + [k = 0]) sum_m v_m cos(...)    (before C2L)
// each through one complex FFT of length n (Makhoul's reordering: the even
// entries of v in order, then the odd ones reversed, and a shift by
// exp(i pi k / (2n))).  One CTA takes one whole vector: it stages it in shared
// memory and runs a radix-2 FFT there.  The synthesis works in double-float
// arithmetic on the FP32 pipe, on a copy scaled by the power of two of the
// vector's largest entry (scaled back exactly); the analysis works in FP64,
// since C2L, which follows it, grows the rounding noise that a transform of
// point values leaves on every coefficient (double-float left 2.7e-13 at
// n = 4096).  Twiddles are built in FP64 at plan time.
#include "lc_df.cuh"
#include "lc_internal.cuh"

namespace {

// Complex numbers in double-float (the synthesis) and in FP64 (the
// analysis: its result feeds C2L, whose growth on the noise floor of a
// transform of point values needs the FP64 rounding level).
struct __align__(16) cdf {
  lc_df re, im;
};
struct __align__(16) cd {
  double re, im;
};
__device__ __forceinline__ cdf cmul(const cdf& a, const cdf& b) {
  return cdf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cdf cadd(const cdf& a, const cdf& b) { return cdf{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cdf csub(const cdf& a, const cdf& b) { return cdf{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd cmul(const cd& a, const cd& b) {
  return cd{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cd cadd(const cd& a, const cd& b) { return cd{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd csub(const cd& a, const cd& b) { return cd{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ void conj_inplace(cdf& w) { w.im = -w.im; }
__device__ __forceinline__ void conj_inplace(cd& w) { w.im = -w.im; }
__device__ __forceinline__ lc_df df_of(double x) {
  const float h = float(x);
  return lc_df(h, float(x - double(h)));
}

// tw[t] = exp(-2 pi i t / n), t < n/2; sh[k] = exp(i pi k / (2n)), k < n: in
// FP64 (tw64, sh64) and rounded to double-float (tw, sh).
__global__ void k_values_tables(int n, cdf* __restrict__ tw, cdf* __restrict__ sh, cd* __restrict__ tw64,
                                cd* __restrict__ sh64) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    if (t < n / 2) {
      const double c = cospi(2.0 * t / n), s = -sinpi(2.0 * t / n);
      tw[t] = cdf{df_of(c), df_of(s)};
      tw64[t] = cd{c, s};
    }
    const double c = cospi(0.5 * t / n), s = sinpi(0.5 * t / n);
    sh[t] = cdf{df_of(c), df_of(s)};
    sh64[t] = cd{c, s};
  }
}

// Unbiased exponent of |x| (subnormals normalised), or kNone for 0, inf, NaN.
constexpr int kNone = -(1 << 20);
__device__ __forceinline__ int exponent_of(double x) {
  const uint64_t u = __double_as_longlong(x);
  const int E = int((u >> 52) & 0x7ff);
  const uint64_t m = u & ((uint64_t(1) << 52) - 1);
  if (E == 2047) return kNone;
  if (E == 0) return m ? 1 - (__clzll(m) - 11) - 1023 : kNone;
  return E - 1023;
}

// In-place radix-2 FFT of the n = 2^logn points in x (loaded in bit-reversed
// order); inverse != 0 uses exp(+2 pi i t / n) and no 1/n.
template <typename C>
__device__ __forceinline__ void fft(C* x, int n, int logn, const C* __restrict__ tw, int inverse) {
  for (int st = 0; st < logn; ++st) {
    const int h = 1 << st;
    for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
      const int pos = j & (h - 1);
      const int i0 = ((j >> st) << (st + 1)) + pos, i1 = i0 + h;
      C w = tw[pos << (logn - 1 - st)];
      if (inverse) conj_inplace(w);
      const C a = x[i0], t = cmul(w, x[i1]);
      x[i0] = cadd(a, t);
      x[i1] = csub(a, t);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int block_max(int v, int* red) {
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int r = kNone;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) r = max(r, red[w]);
  __syncthreads();
  return r;
}

// Synthesis: the Chebyshev coefficients c of each vector (at io, layout
// ob/oe/inner/oob) become their values at the Chebyshev-Gauss points, in
// place, in double-float arithmetic on a copy scaled by the power of two of
// the vector's largest entry.
__global__ void __launch_bounds__(256) k_values_synth(int n, int logn, int64_t batch, double* io, int64_t ob,
                                                     int64_t oe, int64_t inner, int64_t oob,
                                                     const cdf* __restrict__ tw, const cdf* __restrict__ sh) {
  extern __shared__ __align__(16) unsigned char smem[];
  cdf* x = reinterpret_cast<cdf*>(smem);                                   // [n]
  double* raw = reinterpret_cast<double*>(smem + size_t(n) * sizeof(cdf));  // [n]
  __shared__ int red[32];
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    double* s = io + lc_boff(b, ob, inner, oob);
    __syncthreads();  // shared memory of the previous vector is free
    int m = kNone;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double v = s[j * oe];
      raw[j] = v;
      m = max(m, exponent_of(v));
    }
    const int emax = block_max(m, red);
    const int e = emax == kNone ? 0 : emax;  // the vector is c 2^-e: largest entry in [1, 2)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      // Y_k = 1/2 exp(i pi k/(2n)) (a_k c_k - i c_(n-k)), a_0 = 2, c_n = 0
      const lc_df P = lc_df_from_double_s(raw[j], e) * lc_df(j == 0 ? 1.0f : 0.5f, 0.0f);
      const lc_df Q = j == 0 ? lc_df(0.0f, 0.0f) : lc_df_from_double_s(raw[n - j], e) * lc_df(0.5f, 0.0f);
      const cdf w = sh[j];
      const int r = int(__brev(unsigned(j)) >> (32 - logn));
      x[r] = cdf{P * w.re + Q * w.im, P * w.im - Q * w.re};
    }
    __syncthreads();
    fft(x, n, logn, tw, 1);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int yi = (j & 1) ? n - 1 - (j >> 1) : (j >> 1);  // even entries in order, odd ones reversed
      s[j * oe] = lc_df_to_double_s(x[yi].re, e);
    }
  }
}

// Analysis: the values of each vector (at src, layout ib/ie/inner/iob)
// become Chebyshev coefficients in dst[b n + k], in FP64 arithmetic.
__global__ void __launch_bounds__(256) k_values_analysis(int n, int logn, int64_t batch, const double* src,
                                                        int64_t ib, int64_t ie, int64_t inner, int64_t iob,
                                                        double* dst, const cd* __restrict__ tw,
                                                        const cd* __restrict__ sh) {
  extern __shared__ __align__(16) unsigned char smem[];
  cd* x = reinterpret_cast<cd*>(smem);  // [n]
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    const double* s = src + lc_boff(b, ib, inner, iob);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const int yi = (j & 1) ? n - 1 - (j >> 1) : (j >> 1);  // even entries in order, odd ones reversed
      x[int(__brev(unsigned(yi)) >> (32 - logn))] = cd{s[j * ie], 0.0};
    }
    __syncthreads();
    fft(x, n, logn, tw, 0);
    double* o = dst + b * int64_t(n);
    const double two_n = 2.0 / double(n);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const cd w = sh[k];  // X_k = Re(exp(-i pi k/(2n)) Y_k)
      const double X = fma(x[k].re, w.re, x[k].im * w.im);
      o[k] = X * (k == 0 ? 0.5 * two_n : two_n);
    }
  }
}

size_t values_smem(int n) { return size_t(n) * (sizeof(cdf) + sizeof(double)) + 16; }
size_t analysis_smem(int n) { return size_t(n) * sizeof(cd) + 16; }

int log2_exact(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return (int64_t(1) << l) == n ? l : -1;
}

unsigned values_grid(int64_t batch) {
  const int64_t g = batch < 152 * 16 ? batch : 152 * 16;
  return unsigned(g > 0 ? g : 1);
}

// ---------------------------------------------------------------- large n
// Above kSmallN one vector no longer fits one CTA's shared memory; its FFT of
// length n = n1 n2 runs in two passes through a [n2][n1] work array
// (the four-step FFT): with k = k1 + n1 k2 and j = j2 + n2 j1,
//   A_j = sum_k1 W_n1^(j1 k1) [ W_n^(j2 k1) sum_k2 W_n2^(j2 k2) a_k ],
// (W_m = exp(-+2 pi i / m)).  The column pass takes kTW consecutive k1 and
// every k2 (coalesced rows of kTW entries), runs the kTW FFTs of length n2,
// applies the twiddles W_n^(j2 k1) and stores row j2 of the work array; the
// row pass takes one row j2, runs the FFT of length n1 over k1 and writes the
// outputs j = j2 + n2 j1.  The pre- and post-processing of the small kernels
// (Makhoul's reordering, the half-sample shift) ride in the two passes.
constexpr int kSmallN = 4096;
constexpr int kTW = 8;  // columns per CTA of the column pass

struct Split {
  int n1, n2, log1, log2;
};
Split split_of(int64_t n) {
  Split q;
  q.n1 = int(n / 16 < 8192 ? n / 16 : 8192);
  q.n2 = int(n / q.n1);
  q.log1 = log2_exact(q.n1);
  q.log2 = log2_exact(q.n2);
  return q;
}
__device__ __forceinline__ cdf cneg(const cdf& a) { return cdf{-a.re, -a.im}; }
__device__ __forceinline__ cd cneg(const cd& a) { return cd{-a.re, -a.im}; }
// W_n^t = exp(-2 pi i t / n), 0 <= t < n, from the half-circle table
template <typename C>
__device__ __forceinline__ C tw_full(const C* __restrict__ tw, int64_t t, int64_t half) {
  return t < half ? tw[t] : cneg(tw[t - half]);
}
__device__ __forceinline__ int bitrev(int k, int logm) { return int(__brev(unsigned(k)) >> (32 - logm)); }

// count independent radix-2 FFTs of length L = 2^logL at x + f L (each loaded
// in bit-reversed order); roots W_L^t = tw[t * tstride] (tw: the table of W_n).
template <typename C>
__device__ __forceinline__ void fft_multi(C* x, int count, int L, int logL, const C* __restrict__ tw, int64_t tstride,
                                          int inverse) {
  const int per = L >> 1;
  for (int st = 0; st < logL; ++st) {
    const int h = 1 << st;
    for (int u = threadIdx.x; u < count * per; u += blockDim.x) {
      const int f = u >> (logL - 1), j = u & (per - 1);
      const int pos = j & (h - 1);
      const int i0 = ((j >> st) << (st + 1)) + pos, i1 = i0 + h;
      C w = tw[int64_t(pos << (logL - 1 - st)) * tstride];
      if (inverse) conj_inplace(w);
      C* y = x + f * L;
      const C a = y[i0], t = cmul(w, y[i1]);
      y[i0] = cadd(a, t);
      y[i1] = csub(a, t);
    }
    __syncthreads();
  }
}

// Largest exponent of each vector of Chebyshev coefficients (the synthesis
// scales by it): CTA (x, b) takes 4096 entries of vector b; xe[b] starts at
// the memset pattern 0x80808080 (below every exponent).
__global__ void __launch_bounds__(256) k_vsyn_exp(int64_t n, int64_t batch, const double* io, int64_t ob, int64_t oe,
                                                 int64_t inner, int64_t oob, int* __restrict__ xe) {
  __shared__ int red[32];
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const double* s = io + lc_boff(b, ob, inner, oob);
    int m = kNone;
    const int64_t j0 = int64_t(blockIdx.x) * 4096;
    for (int u = 0; u < 16; ++u) {
      const int64_t j = j0 + u * 256 + threadIdx.x;
      if (j < n) m = max(m, exponent_of(s[j * oe]));
    }
    m = block_max(m, red);
    if (threadIdx.x == 0 && m > kNone) atomicMax(xe + b, m);
  }
}

__device__ __forceinline__ int vec_e(const int* xe, int64_t b) {
  const int v = xe[b];
  return v <= kNone ? 0 : v;
}

// Synthesis, column pass: Y_k = 1/2 exp(i pi k/(2n)) (a_k c_k - i c_(n-k))
// from the coefficients (scaled by 2^-e), inverse FFTs over k2, twiddles,
// rows j2 of the work array T[b][n2][n1].
__global__ void __launch_bounds__(256) k_vsyn_cols(int n, int n1, int n2, int log2, int64_t batch, const double* io,
                                                  int64_t ob, int64_t oe, int64_t inner, int64_t oob,
                                                  const int* __restrict__ xe, cdf* __restrict__ T,
                                                  const cdf* __restrict__ tw, const cdf* __restrict__ sh) {
  extern __shared__ __align__(16) unsigned char smem[];
  cdf* x = reinterpret_cast<cdf*>(smem);  // [kTW][n2]
  const int c0 = blockIdx.x * kTW;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const double* s = io + lc_boff(b, ob, inner, oob);
    const int e = vec_e(xe, b);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTW * n2; idx += blockDim.x) {
      const int tc = idx & (kTW - 1), k2 = idx / kTW;
      const int64_t k = c0 + tc + int64_t(n1) * k2;
      const lc_df P = lc_df_from_double_s(s[k * oe], e) * lc_df(k == 0 ? 1.0f : 0.5f, 0.0f);
      const lc_df Q = k == 0 ? lc_df(0.0f, 0.0f) : lc_df_from_double_s(s[(n - k) * oe], e) * lc_df(0.5f, 0.0f);
      const cdf w = sh[k];
      x[tc * n2 + bitrev(k2, log2)] = cdf{P * w.re + Q * w.im, P * w.im - Q * w.re};
    }
    __syncthreads();
    fft_multi(x, kTW, n2, log2, tw, n / n2, 1);
    cdf* Tb = T + b * int64_t(n);
    for (int idx = threadIdx.x; idx < kTW * n2; idx += blockDim.x) {
      const int tc = idx & (kTW - 1), j2 = idx / kTW;
      const int k1 = c0 + tc;
      cdf w = tw_full(tw, int64_t(j2) * k1, n / 2);
      conj_inplace(w);
      Tb[int64_t(j2) * n1 + k1] = cmul(w, x[tc * n2 + j2]);
    }
  }
}

// Synthesis, row pass: FFT over k1 of row j2, then out_j = Re A_(j2 + n2 j1)
// 2^e at the position j of Makhoul's reordering (even j in order, odd reversed).
__global__ void __launch_bounds__(256) k_vsyn_rows(int n, int n1, int n2, int log1, int64_t batch, double* io,
                                                  int64_t ob, int64_t oe, int64_t inner, int64_t oob,
                                                  const int* __restrict__ xe, const cdf* __restrict__ T,
                                                  const cdf* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  cdf* x = reinterpret_cast<cdf*>(smem);  // [n1]
  const int j2 = blockIdx.x;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    double* s = io + lc_boff(b, ob, inner, oob);
    const int e = vec_e(xe, b);
    const cdf* row = T + b * int64_t(n) + int64_t(j2) * n1;
    __syncthreads();
    for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) x[bitrev(k1, log1)] = row[k1];
    __syncthreads();
    fft_multi(x, 1, n1, log1, tw, n / n1, 1);
    for (int j1 = threadIdx.x; j1 < n1; j1 += blockDim.x) {
      const int64_t i = j2 + int64_t(n2) * j1;
      const int64_t j = i < n / 2 ? 2 * i : 2 * (n - 1 - i) + 1;
      s[j * oe] = lc_df_to_double_s(x[j1].re, e);
    }
  }
}

// Analysis, column pass (FP64): x_k = v at the position of Makhoul's
// reordering, forward FFTs over k2, twiddles, rows j2 of T[b][n2][n1].
__global__ void __launch_bounds__(256) k_vana_cols(int n, int n1, int n2, int log2, int64_t batch, const double* src,
                                                  int64_t ib, int64_t ie, int64_t inner, int64_t iob,
                                                  cd* __restrict__ T, const cd* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem[];
  cd* x = reinterpret_cast<cd*>(smem);  // [kTW][n2]
  const int c0 = blockIdx.x * kTW;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const double* s = src + lc_boff(b, ib, inner, iob);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTW * n2; idx += blockDim.x) {
      const int tc = idx & (kTW - 1), k2 = idx / kTW;
      const int64_t k = c0 + tc + int64_t(n1) * k2;
      const int64_t j = k < n / 2 ? 2 * k : 2 * (n - 1 - k) + 1;  // x_k = v_j
      x[tc * n2 + bitrev(k2, log2)] = cd{s[j * ie], 0.0};
    }
    __syncthreads();
    fft_multi(x, kTW, n2, log2, tw, n / n2, 0);
    cd* Tb = T + b * int64_t(n);
    for (int idx = threadIdx.x; idx < kTW * n2; idx += blockDim.x) {
      const int tc = idx & (kTW - 1), j2 = idx / kTW;
      const int k1 = c0 + tc;
      Tb[int64_t(j2) * n1 + k1] = cmul(tw_full(tw, int64_t(j2) * k1, n / 2), x[tc * n2 + j2]);
    }
  }
}

// Analysis, row pass: FFT over k1 of row j2, then
// X_i = Re(exp(-i pi i/(2n)) Y_i) 2/n (halved at i = 0) into dst[b n + i].
__global__ void __launch_bounds__(256) k_vana_rows(int n, int n1, int n2, int log1, int64_t batch,
                                                  const cd* __restrict__ T, double* __restrict__ dst,
                                                  const cd* __restrict__ tw, const cd* __restrict__ sh) {
  extern __shared__ __align__(16) unsigned char smem[];
  cd* x = reinterpret_cast<cd*>(smem);  // [n1]
  const int j2 = blockIdx.x;
  const double two_n = 2.0 / double(n);
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const cd* row = T + b * int64_t(n) + int64_t(j2) * n1;
    __syncthreads();
    for (int k1 = threadIdx.x; k1 < n1; k1 += blockDim.x) x[bitrev(k1, log1)] = row[k1];
    __syncthreads();
    fft_multi(x, 1, n1, log1, tw, n / n1, 0);
    double* o = dst + b * int64_t(n);
    for (int j1 = threadIdx.x; j1 < n1; j1 += blockDim.x) {
      const int64_t i = j2 + int64_t(n2) * j1;
      const cd w = sh[i];
      const double X = fma(x[j1].re, w.re, x[j1].im * w.im);
      o[i] = X * (i == 0 ? 0.5 * two_n : two_n);
    }
  }
}

unsigned batch_grid(int64_t batch) { return unsigned(batch < 65535 ? batch : 65535); }

}  // namespace

bool lc_values_supported(int64_t n) { return n >= 2 && n <= LC_VALUES_MAX_N && log2_exact(n) > 0; }

size_t lc_values_table_bytes(int64_t n) { return size_t(n) * 3 / 2 * (sizeof(cdf) + sizeof(cd)); }

size_t lc_values_work_bytes(int64_t n, int64_t batch) {
  if (n <= kSmallN) return 0;
  return size_t(batch) * size_t(n) * sizeof(cd) + size_t(batch) * sizeof(int) + 256;
}

int lc_values_launches(const lc_plan_s* p) {
  if (p->g.n <= kSmallN) return 1;
  return p->dir == LC_L2C ? 3 : 2;
}

namespace {
struct Tables {
  cdf *tw, *sh;
  cd *tw64, *sh64;
};
Tables tables_of(const lc_plan_s* p) {
  const int64_t n = p->g.n;
  cdf* t = static_cast<cdf*>(p->val_tables);
  cd* t64 = reinterpret_cast<cd*>(t + n * 3 / 2);
  return Tables{t, t + n / 2, t64, t64 + n / 2};
}
}  // namespace

lc_status lc_values_prepare(lc_plan p, cudaStream_t st) {
  const int n = int(p->g.n);
  const Tables t = tables_of(p);
  k_values_tables<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, t.tw, t.sh, t.tw64, t.sh64);
  LC_LAUNCH_CHECK();
  if (n > kSmallN) {
    const Split q = split_of(n);
    const int cols = int(size_t(kTW) * q.n2 * sizeof(cd)), rows = int(size_t(q.n1) * sizeof(cd));
    const void* fc[2] = {reinterpret_cast<const void*>(k_vsyn_cols), reinterpret_cast<const void*>(k_vana_cols)};
    const void* fr[2] = {reinterpret_cast<const void*>(k_vsyn_rows), reinterpret_cast<const void*>(k_vana_rows)};
    for (int k = 0; k < 2; ++k) {
      if (cols > 44 * 1024) LC_CUDA_TRY(cudaFuncSetAttribute(fc[k], cudaFuncAttributeMaxDynamicSharedMemorySize, cols));
      if (rows > 44 * 1024) LC_CUDA_TRY(cudaFuncSetAttribute(fr[k], cudaFuncAttributeMaxDynamicSharedMemorySize, rows));
    }
    return LC_OK;
  }
  if (values_smem(n) > 44 * 1024)
    LC_CUDA_TRY(cudaFuncSetAttribute(k_values_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, int(values_smem(n))));
  if (analysis_smem(n) > 44 * 1024)
    LC_CUDA_TRY(
        cudaFuncSetAttribute(k_values_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, int(analysis_smem(n))));
  return LC_OK;
}

lc_status lc_values_synth(lc_plan p, double* out, const lc_layout& lay, cudaStream_t st) {
  const int n = int(p->g.n);
  const Tables t = tables_of(p);
  if (n > kSmallN) {
    const Split q = split_of(n);
    cd* T = static_cast<cd*>(p->val_work);
    int* xe = reinterpret_cast<int*>(T + size_t(p->batch) * size_t(n));
    LC_CUDA_TRY(cudaMemsetAsync(xe, 0x80, size_t(p->batch) * sizeof(int), st));
    const unsigned gy = batch_grid(p->batch);
    k_vsyn_exp<<<dim3(unsigned((n + 4095) / 4096), gy), 256, 0, st>>>(n, p->batch, out, lay.ob, lay.oe, lay.inner,
                                                                    lay.oob, xe);
    LC_LAUNCH_CHECK();
    k_vsyn_cols<<<dim3(unsigned(q.n1 / kTW), gy), 256, size_t(kTW) * q.n2 * sizeof(cdf), st>>>(
        n, q.n1, q.n2, q.log2, p->batch, out, lay.ob, lay.oe, lay.inner, lay.oob, xe, reinterpret_cast<cdf*>(T), t.tw,
        t.sh);
    LC_LAUNCH_CHECK();
    k_vsyn_rows<<<dim3(unsigned(q.n2), gy), 256, size_t(q.n1) * sizeof(cdf), st>>>(
        n, q.n1, q.n2, q.log1, p->batch, out, lay.ob, lay.oe, lay.inner, lay.oob, xe, reinterpret_cast<cdf*>(T), t.tw);
    LC_LAUNCH_CHECK();
    return LC_OK;
  }
  k_values_synth<<<values_grid(p->batch), 256, values_smem(n), st>>>(n, log2_exact(n), p->batch, out, lay.ob, lay.oe,
                                                                     lay.inner, lay.oob, t.tw, t.sh);
  LC_LAUNCH_CHECK();
  return LC_OK;
}

lc_status lc_values_analysis(lc_plan p, const double* in, const lc_layout& lay, double* scratch, cudaStream_t st) {
  const int n = int(p->g.n);
  const Tables t = tables_of(p);
  if (n > kSmallN) {
    const Split q = split_of(n);
    cd* T = static_cast<cd*>(p->val_work);
    const unsigned gy = batch_grid(p->batch);
    k_vana_cols<<<dim3(unsigned(q.n1 / kTW), gy), 256, size_t(kTW) * q.n2 * sizeof(cd), st>>>(
        n, q.n1, q.n2, q.log2, p->batch, in, lay.ib, lay.ie, lay.inner, lay.iob, T, t.tw64);
    LC_LAUNCH_CHECK();
    k_vana_rows<<<dim3(unsigned(q.n2), gy), 256, size_t(q.n1) * sizeof(cd), st>>>(n, q.n1, q.n2, q.log1, p->batch, T,
                                                                                scratch, t.tw64, t.sh64);
    LC_LAUNCH_CHECK();
    return LC_OK;
  }
  k_values_analysis<<<values_grid(p->batch), 256, analysis_smem(n), st>>>(n, log2_exact(n), p->batch, in, lay.ib,
                                                                          lay.ie, lay.inner, lay.iob, scratch,
                                                                          t.tw64, t.sh64);
  LC_LAUNCH_CHECK();
  return LC_OK;
}
