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

// --------------------------------------------------- other lengths n
// For n not a power of two the FFT of length n is Bluestein's: with
// zeta = exp(i pi / n) and jk = (j^2 + k^2 - (j-k)^2)/2,
//   sum_k a_k exp(+-2 pi i jk/n) = zeta^(+-j^2) sum_k (a_k zeta^(+-k^2)) zeta^(-+(j-k)^2),
// a convolution, computed as a circular one of power-of-two length m >= 2n-1
// by two FFTs of length m (four-step, through the work arrays) and the
// pointwise product with the FFT of the chirp sequence, made at plan time.
// chirp[t] = zeta^(t^2), the angle reduced exactly (t^2 mod 2n) in integers.
int64_t blu_m(int64_t n) {
  int64_t m = 256;
  while (m < 2 * n - 1) m <<= 1;
  return m;
}
__global__ void k_blu_tables(int n, int m, cdf* __restrict__ twm, cd* __restrict__ twm64, cdf* __restrict__ sh,
                             cd* __restrict__ sh64, cdf* __restrict__ ch, cd* __restrict__ ch64) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m / 2 || t < n; t += gridDim.x * blockDim.x) {
    if (t < m / 2) {
      const double c = cospi(2.0 * t / m), si = -sinpi(2.0 * t / m);
      twm[t] = cdf{df_of(c), df_of(si)};
      twm64[t] = cd{c, si};
    }
    if (t < n) {
      const double c = cospi(0.5 * t / n), si = sinpi(0.5 * t / n);
      sh[t] = cdf{df_of(c), df_of(si)};
      sh64[t] = cd{c, si};
      const int64_t q = (int64_t(t) * t) % (2 * int64_t(n));  // zeta^(t^2) = exp(i pi q / n)
      const double cc = cospi(double(q) / n), ss = sinpi(double(q) / n);
      ch[t] = cdf{df_of(cc), df_of(ss)};
      ch64[t] = cd{cc, ss};
    }
  }
}
// The chirp sequence of the synthesis's convolution, b_t = zeta^(-t^2) for
// |t| < n, placed circularly in [0, m) (FP64).
__global__ void k_blu_bc(int n, int m, const cd* __restrict__ ch64, cd* __restrict__ bc) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    const int u = t < n ? t : (m - t < n ? m - t : -1);
    bc[t] = u < 0 ? cd{0.0, 0.0} : cd{ch64[u].re, -ch64[u].im};
  }
}
__global__ void k_d2df_c(int count, const cd* __restrict__ a, cdf* __restrict__ b) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
    b[t] = cdf{df_of(a[t].re), df_of(a[t].im)};
}

// FFT of length m (four-step) over work arrays in natural order: the column
// pass reads src[b][m], runs the m2-point FFTs over k2, applies the
// twiddles and writes rows j2 of T[b][m2][m1].
template <typename C>
__global__ void __launch_bounds__(256) k_cf_cols(int m, int m1, int m2, int logm2, int64_t batch,
                                                const C* __restrict__ src, C* __restrict__ T,
                                                const C* __restrict__ tw, int inverse) {
  extern __shared__ __align__(16) unsigned char smem[];
  C* x = reinterpret_cast<C*>(smem);  // [kTW][m2]
  const int c0 = blockIdx.x * kTW;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const C* sb = src + b * int64_t(m);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTW * m2; idx += blockDim.x) {
      const int tc = idx & (kTW - 1), k2 = idx / kTW;
      x[tc * m2 + bitrev(k2, logm2)] = sb[c0 + tc + int64_t(m1) * k2];
    }
    __syncthreads();
    fft_multi(x, kTW, m2, logm2, tw, m / m2, inverse);
    C* Tb = T + b * int64_t(m);
    for (int idx = threadIdx.x; idx < kTW * m2; idx += blockDim.x) {
      const int tc = idx & (kTW - 1), j2 = idx / kTW;
      const int k1 = c0 + tc;
      C w = tw_full(tw, int64_t(j2) * k1, m / 2);
      if (inverse) conj_inplace(w);
      Tb[int64_t(j2) * m1 + k1] = cmul(w, x[tc * m2 + j2]);
    }
  }
}

// Row pass: the m1-point FFT of row j2, then, for the outputs j = j2 + m2 j1,
// mode 0: dst[b][j] = y * Bh[j] (the convolution's pointwise product; conj_b:
// the analysis's filter conj(Bh[(m - j) mod m])); mode 1: dst[b][j] = y (the
// plan-time FFT of the chirp sequence).
template <typename C>
__global__ void __launch_bounds__(256) k_cf_rows(int m, int m1, int m2, int logm1, int64_t batch,
                                                const C* __restrict__ T, C* __restrict__ dst,
                                                const C* __restrict__ tw, int inverse, int mode,
                                                const C* __restrict__ Bh, int conj_b) {
  extern __shared__ __align__(16) unsigned char smem[];
  C* x = reinterpret_cast<C*>(smem);  // [m1]
  const int j2 = blockIdx.x;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const C* row = T + b * int64_t(m) + int64_t(j2) * m1;
    __syncthreads();
    for (int k1 = threadIdx.x; k1 < m1; k1 += blockDim.x) x[bitrev(k1, logm1)] = row[k1];
    __syncthreads();
    fft_multi(x, 1, m1, logm1, tw, m / m1, inverse);
    C* db = dst + b * int64_t(m);
    for (int j1 = threadIdx.x; j1 < m1; j1 += blockDim.x) {
      const int64_t j = j2 + int64_t(m2) * j1;
      C y = x[j1];
      if (mode == 0) {
        C f = conj_b ? Bh[(m - j) & (m - 1)] : Bh[j];
        if (conj_b) conj_inplace(f);
        y = cmul(y, f);
      }
      db[j] = y;
    }
  }
}

// Synthesis, Bluestein input: a_k = Y_k chirp[k] (k < n; 0 up to m), Y_k from
// the coefficients as in k_values_synth (scaled by the vector's 2^-e).
__global__ void __launch_bounds__(256) k_blu_pre_syn(int n, int m, int64_t batch, const double* io, int64_t ob,
                                                    int64_t oe, int64_t inner, int64_t oob,
                                                    const int* __restrict__ xe, const cdf* __restrict__ sh,
                                                    const cdf* __restrict__ ch, cdf* __restrict__ A) {
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const double* s = io + lc_boff(b, ob, inner, oob);
    const int e = vec_e(xe, b);
    cdf* Ab = A + b * int64_t(m);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
      cdf v{lc_df(0.0f, 0.0f), lc_df(0.0f, 0.0f)};
      if (k < n) {
        const lc_df P = lc_df_from_double_s(s[int64_t(k) * oe], e) * lc_df(k == 0 ? 1.0f : 0.5f, 0.0f);
        const lc_df Q =
            k == 0 ? lc_df(0.0f, 0.0f) : lc_df_from_double_s(s[int64_t(n - k) * oe], e) * lc_df(0.5f, 0.0f);
        const cdf w = sh[k];
        v = cmul(cdf{P * w.re + Q * w.im, P * w.im - Q * w.re}, ch[k]);
      }
      Ab[k] = v;
    }
  }
}
// Synthesis output: x_j = chirp[j] conv_j / m, out at Makhoul's position of j.
__global__ void __launch_bounds__(256) k_blu_post_syn(int n, int m, int64_t batch, const cdf* __restrict__ conv,
                                                     const cdf* __restrict__ ch, const int* __restrict__ xe,
                                                     double* io, int64_t ob, int64_t oe, int64_t inner,
                                                     int64_t oob) {
  const lc_df inv_m(1.0f / float(m), 0.0f);  // m a power of two: exact
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    double* s = io + lc_boff(b, ob, inner, oob);
    const int e = vec_e(xe, b);
    const cdf* cb = conv + b * int64_t(m);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      const cdf x = cmul(ch[j], cb[j]);
      const int64_t o = j < (n + 1) / 2 ? 2 * int64_t(j) : 2 * int64_t(n - 1 - j) + 1;
      s[o * oe] = lc_df_to_double_s(x.re * inv_m, e);
    }
  }
}
// Analysis, Bluestein input: a_j = x_j conj(chirp[j]), x_j = v at Makhoul's
// position of j (FP64).
__global__ void __launch_bounds__(256) k_blu_pre_ana(int n, int m, int64_t batch, const double* src, int64_t ib,
                                                    int64_t ie, int64_t inner, int64_t iob,
                                                    const cd* __restrict__ ch64, cd* __restrict__ A) {
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const double* s = src + lc_boff(b, ib, inner, iob);
    cd* Ab = A + b * int64_t(m);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
      cd v{0.0, 0.0};
      if (j < n) {
        const int64_t o = j < (n + 1) / 2 ? 2 * int64_t(j) : 2 * int64_t(n - 1 - j) + 1;
        const double x = s[o * ie];
        v = cd{x * ch64[j].re, -x * ch64[j].im};
      }
      Ab[j] = v;
    }
  }
}
// Analysis output: X_k = conj(chirp[k]) conv_k / m, then the coefficient
// Re(exp(-i pi k/(2n)) X_k) 2/n (halved at k = 0) into dst[b n + k].
__global__ void __launch_bounds__(256) k_blu_post_ana(int n, int m, int64_t batch, const cd* __restrict__ conv,
                                                     const cd* __restrict__ ch64, const cd* __restrict__ sh64,
                                                     double* __restrict__ dst) {
  const double inv_m = 1.0 / double(m), two_n = 2.0 / double(n);
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const cd* cb = conv + b * int64_t(m);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
      const cd c{ch64[k].re, -ch64[k].im};
      const cd X = cmul(c, cb[k]);
      const cd w = sh64[k];
      const double v = fma(X.re, w.re, X.im * w.im) * inv_m;
      dst[b * int64_t(n) + k] = v * (k == 0 ? 0.5 * two_n : two_n);
    }
  }
}

unsigned batch_grid(int64_t batch) { return unsigned(batch < 65535 ? batch : 65535); }

}  // namespace

namespace {
bool pow2(int64_t n) { return log2_exact(n) > 0; }
}  // namespace

bool lc_values_supported(int64_t n) {
  return n >= 2 && n <= LC_VALUES_MAX_N && (pow2(n) || n <= LC_VALUES_MAX_N_ANY);
}

size_t lc_values_table_bytes(int64_t n) {
  if (pow2(n)) return size_t(n) * 3 / 2 * (sizeof(cdf) + sizeof(cd));
  const int64_t m = blu_m(n);  // twiddles of m, shift and chirp of n, the chirp's FFT
  return size_t(m / 2 + 2 * n + m) * (sizeof(cdf) + sizeof(cd));
}

size_t lc_values_work_bytes(int64_t n, int64_t batch) {
  if (pow2(n)) {
    if (n <= kSmallN) return 0;
    return size_t(batch) * size_t(n) * sizeof(cd) + size_t(batch) * sizeof(int) + 256;
  }
  const int64_t m = blu_m(n);  // two complex arrays of m per vector (at least two for the plan-time FFT)
  const int64_t b = batch > 1 ? batch : 1;
  return size_t(2 * b) * size_t(m) * sizeof(cd) + size_t(batch) * sizeof(int) + 256;
}

int lc_values_launches(const lc_plan_s* p) {
  if (!pow2(p->g.n)) return p->dir == LC_L2C ? 7 : 6;
  if (p->g.n <= kSmallN) return 1;
  return p->dir == LC_L2C ? 3 : 2;
}

namespace {
struct Tables {
  cdf *tw, *sh;
  cd *tw64, *sh64;
  cdf *ch, *Bh;    // Bluestein: chirp[n], FFT of the chirp sequence [m]
  cd *ch64, *Bh64;
  int64_t m;       // Bluestein length (0 for powers of two)
};
Tables tables_of(const lc_plan_s* p) {
  const int64_t n = p->g.n;
  cdf* t = static_cast<cdf*>(p->val_tables);
  if (pow2(n)) {
    cd* t64 = reinterpret_cast<cd*>(t + n * 3 / 2);
    return Tables{t, t + n / 2, t64, t64 + n / 2, nullptr, nullptr, nullptr, nullptr, 0};
  }
  const int64_t m = blu_m(n), per = m / 2 + 2 * n + m;
  cd* t64 = reinterpret_cast<cd*>(t + per);
  return Tables{t,           t + m / 2,           t64,       t64 + m / 2, t + m / 2 + n, t + m / 2 + 2 * n,
                t64 + m / 2 + n, t64 + m / 2 + 2 * n, m};
}
// The two-pass FFT of length m over work arrays (Bluestein's convolutions).
template <typename C>
lc_status cf_fft(int64_t m, int64_t batch, const C* src, C* T, C* dst, const C* tw, int inverse, int mode,
                 const C* Bh, int conj_b, cudaStream_t st) {
  const Split q = split_of(m);
  const unsigned gy = batch_grid(batch);
  k_cf_cols<C><<<dim3(unsigned(q.n1 / kTW), gy), 256, size_t(kTW) * q.n2 * sizeof(C), st>>>(
      int(m), q.n1, q.n2, q.log2, batch, src, T, tw, inverse);
  LC_LAUNCH_CHECK();
  k_cf_rows<C><<<dim3(unsigned(q.n2), gy), 256, size_t(q.n1) * sizeof(C), st>>>(int(m), q.n1, q.n2, q.log1, batch, T,
                                                                              dst, tw, inverse, mode, Bh, conj_b);
  LC_LAUNCH_CHECK();
  return LC_OK;
}
lc_status cf_smem(int64_t m) {
  const Split q = split_of(m);
  const int cols = int(size_t(kTW) * q.n2 * sizeof(cd)), rows = int(size_t(q.n1) * sizeof(cd));
  const void* fc[2] = {reinterpret_cast<const void*>(k_cf_cols<cdf>), reinterpret_cast<const void*>(k_cf_cols<cd>)};
  const void* fr[2] = {reinterpret_cast<const void*>(k_cf_rows<cdf>), reinterpret_cast<const void*>(k_cf_rows<cd>)};
  for (int k = 0; k < 2; ++k) {
    if (cols > 44 * 1024) LC_CUDA_TRY(cudaFuncSetAttribute(fc[k], cudaFuncAttributeMaxDynamicSharedMemorySize, cols));
    if (rows > 44 * 1024) LC_CUDA_TRY(cudaFuncSetAttribute(fr[k], cudaFuncAttributeMaxDynamicSharedMemorySize, rows));
  }
  return LC_OK;
}
unsigned grid_1d(int64_t work) {
  const int64_t g = (work + 255) / 256;
  return unsigned(g < 4096 ? g : 4096);
}
}  // namespace

lc_status lc_values_prepare(lc_plan p, cudaStream_t st) {
  const int n = int(p->g.n);
  const Tables t = tables_of(p);
  if (t.m) {  // Bluestein: tables, then the FFT of the chirp sequence (FP64, once)
    const int m = int(t.m);
    k_blu_tables<<<grid_1d(m > 2 * n ? m : 2 * n), 256, 0, st>>>(n, m, t.tw, t.tw64, t.sh, t.sh64, t.ch, t.ch64);
    LC_LAUNCH_CHECK();
    lc_status e = cf_smem(m);
    if (e != LC_OK) return e;
    cd* A = static_cast<cd*>(p->val_work);
    cd* T = A + m;
    k_blu_bc<<<grid_1d(m), 256, 0, st>>>(n, m, t.ch64, A);
    LC_LAUNCH_CHECK();
    e = cf_fft<cd>(m, 1, A, T, t.Bh64, t.tw64, 0, 1, nullptr, 0, st);
    if (e != LC_OK) return e;
    k_d2df_c<<<grid_1d(m), 256, 0, st>>>(m, t.Bh64, t.Bh);
    LC_LAUNCH_CHECK();
    return LC_OK;
  }
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
  if (t.m) {  // Bluestein: a = Y chirp, conv = IFFT(FFT(a) FFT(b)) / m, x = chirp conv
    const int64_t m = t.m;
    cdf* A = static_cast<cdf*>(p->val_work);
    cdf* T = A + p->batch * m;
    int* xe = reinterpret_cast<int*>(static_cast<cd*>(p->val_work) + 2 * (p->batch > 1 ? p->batch : 1) * m);
    const unsigned gy = batch_grid(p->batch);
    LC_CUDA_TRY(cudaMemsetAsync(xe, 0x80, size_t(p->batch) * sizeof(int), st));
    k_vsyn_exp<<<dim3(unsigned((n + 4095) / 4096), gy), 256, 0, st>>>(n, p->batch, out, lay.ob, lay.oe, lay.inner,
                                                                    lay.oob, xe);
    LC_LAUNCH_CHECK();
    k_blu_pre_syn<<<dim3(grid_1d(m), gy), 256, 0, st>>>(n, int(m), p->batch, out, lay.ob, lay.oe, lay.inner, lay.oob,
                                                       xe, t.sh, t.ch, A);
    LC_LAUNCH_CHECK();
    lc_status e = cf_fft<cdf>(m, p->batch, A, T, A, t.tw, 0, 0, t.Bh, 0, st);
    if (e != LC_OK) return e;
    e = cf_fft<cdf>(m, p->batch, A, T, A, t.tw, 1, 1, nullptr, 0, st);
    if (e != LC_OK) return e;
    k_blu_post_syn<<<dim3(grid_1d(n), gy), 256, 0, st>>>(n, int(m), p->batch, A, t.ch, xe, out, lay.ob, lay.oe,
                                                        lay.inner, lay.oob);
    LC_LAUNCH_CHECK();
    return LC_OK;
  }
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
  if (t.m) {  // Bluestein, FP64: a = x conj(chirp), conv with conj(b), X = conj(chirp) conv
    const int64_t m = t.m;
    cd* A = static_cast<cd*>(p->val_work);
    cd* T = A + p->batch * m;
    const unsigned gy = batch_grid(p->batch);
    k_blu_pre_ana<<<dim3(grid_1d(m), gy), 256, 0, st>>>(n, int(m), p->batch, in, lay.ib, lay.ie, lay.inner, lay.iob,
                                                       t.ch64, A);
    LC_LAUNCH_CHECK();
    lc_status e = cf_fft<cd>(m, p->batch, A, T, A, t.tw64, 0, 0, t.Bh64, 1, st);
    if (e != LC_OK) return e;
    e = cf_fft<cd>(m, p->batch, A, T, A, t.tw64, 1, 1, nullptr, 0, st);
    if (e != LC_OK) return e;
    k_blu_post_ana<<<dim3(grid_1d(n), gy), 256, 0, st>>>(n, int(m), p->batch, A, t.ch64, t.sh64, scratch);
    LC_LAUNCH_CHECK();
    return LC_OK;
  }
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
