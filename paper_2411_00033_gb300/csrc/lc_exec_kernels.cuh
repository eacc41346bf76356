// lc_exec_kernels.cuh -- Algorithm 4 on the CUDA cores, templated on the
// arithmetic type R (double, float, or the double-float pair of lc_df.cuh).
//
// Forward pass for one vector f of length n (zero beyond n), per parity sigma:
//   leaf    w(L-1, g) = T(sigma)^T f^sigma(segment g)           Step 1, eq:wMM
//   up      w(gamma-1, G) = B(0) w(gamma, 2G) + B(1) w(gamma, 2G+1)
//                                                               Step 2, eq:wtk, Alg. a.1
//   couple  c(gamma, v) = sum_{(p,q)} A-hat(gamma, b, r) w(gamma, g)   Step 3
//   down    c(gamma+1, v) += B(v mod 2)^T c(gamma, v/2)         Step 4
//   final   z_i = T(sigma) c(L-1, v) + sum_{band} a_ij f_j, then C^{-1}
//                                                               Steps 5-7
// Segment numbering: see lc_internal.cuh.  The band of row i is
// j in [i, min(N, 2s(floor(i/2s)+2))), j - i even: the part of the upper
// triangle that no submatrix of eq:globalij covers.
//
// The transposed pass runs the same kernels with the roles of row and column
// segments exchanged (leaf restriction over row segments, the row tree
// upwards, A-hat transposed, the column tree downwards, spread over column
// segments, transposed band).
#pragma once
#include "lc_internal.cuh"

namespace lc_exec {


constexpr int kSegs = 4;                 // segments per CTA in leaf/up/down kernels
constexpr int kThreadsSeg = 2 * LC_M;    // (sigma, k) pairs per segment
constexpr int kCoupleSegs = 8;
constexpr int kFinalThreads = 128;

// Element conversions between the I/O type and the arithmetic type R.
template <typename R, typename IO>
__device__ __forceinline__ R lc_ld(const IO* p) { return R(*p); }
template <typename R, typename IO>
__device__ __forceinline__ void lc_st(IO* p, const R& v) { *p = IO(v); }

template <typename R>
struct lc_io { typedef R type; };

template <typename R>
struct Args {
  const typename lc_io<R>::type* in;
  typename lc_io<R>::type* out;
  int64_t ib, ie, ob, oe;
  int64_t n, N;
  int L, s;
  int64_t nseg;
  int64_t batch;
  int dir;
  lc_tables<R> t;
};

template <typename R>
__device__ __forceinline__ R cinv(int64_t i) {
  return i == 0 ? R(0.31830988618379067154) : R(0.63661977236758134308);  // 1/pi, 2/pi
}
template <typename R>
__device__ __forceinline__ R negate(const R& v) { return -v; }

// Leaf restriction (Step 1) over segments [lo, hi) of the leaf level.
// scale_rows: multiply the input by C^{-1} first (transposed L2C pass).
template <typename R>
__global__ void k_leaf(Args<R> a, int64_t lo, int64_t hi, int scale_rows) {
  extern __shared__ unsigned char smem_raw[];
  R* Ts = reinterpret_cast<R*>(smem_raw);               // [2][s][M]
  R* fs = Ts + 2 * a.s * LC_M;                           // [kSegs][2s]
  const int s = a.s, L = a.L;
  for (int i = threadIdx.x; i < 2 * s * LC_M; i += blockDim.x) Ts[i] = a.t.T[i];
  const int64_t g0 = lo + int64_t(blockIdx.x) * kSegs;
  const int seg = threadIdx.x / kThreadsSeg;
  const int sigma = (threadIdx.x % kThreadsSeg) / LC_M;
  const int k = threadIdx.x % LC_M;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    __syncthreads();
    for (int i = threadIdx.x; i < kSegs * 2 * s; i += blockDim.x) {
      const int64_t g = g0 + i / (2 * s);
      const int64_t j = g * 2 * s + i % (2 * s);
      R v = R(0);
      if (g < hi && j < a.n) {
        v = lc_ld<R>(a.in + b * a.ib + j * a.ie);
        if (scale_rows) v *= cinv<R>(j);
      }
      fs[i] = v;
    }
    __syncthreads();
    const int64_t g = g0 + seg;
    if (seg < kSegs && g < hi) {
      const R* fseg = fs + seg * 2 * s;
      R acc = R(0);
      for (int m = 0; m < s; ++m) acc = fma(fseg[2 * m + sigma], Ts[(sigma * s + m) * LC_M + k], acc);
      a.t.W[((b * a.nseg) + lc_seg_offset(L - 1) + g) * (2 * LC_M) + sigma * LC_M + k] = acc;
    }
  }
}

// Upward pass (Step 2): level gc -> gc-1 for parents P in [lo, hi):
//   w(gc-1, P) = B(0) w(gc, 2P) + B(1) w(gc, 2P+1), by Algorithm a.1:
//   z0 = w_left + w_right, z1 = w_left - w_right,
//   out_k = sum_{j<=k} b_kj z_{(k-j) mod 2, j}.
template <typename R>
__global__ void k_up(Args<R> a, int gc, int64_t lo, int64_t hi) {
  __shared__ R Bs[LC_M * LC_M];
  __shared__ R z[kSegs][2][2][LC_M];  // [seg][z0/z1][sigma][j]
  for (int i = threadIdx.x; i < LC_M * LC_M; i += blockDim.x) Bs[i] = a.t.B[i];
  const int seg = threadIdx.x / kThreadsSeg;
  const int sigma = (threadIdx.x % kThreadsSeg) / LC_M;
  const int k = threadIdx.x % LC_M;
  const int64_t P = lo + int64_t(blockIdx.x) * kSegs + seg;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    __syncthreads();
    if (seg < kSegs && P < hi) {
      const R* wc = a.t.W + ((b * a.nseg) + lc_seg_offset(gc) + 2 * P) * (2 * LC_M);
      const R l = wc[sigma * LC_M + k], r = wc[2 * LC_M + sigma * LC_M + k];
      z[seg][0][sigma][k] = l + r;
      z[seg][1][sigma][k] = l - r;
    }
    __syncthreads();
    if (seg < kSegs && P < hi) {
      R acc = R(0);
      for (int j = 0; j <= k; ++j) acc = fma(Bs[k * LC_M + j], z[seg][(k - j) & 1][sigma][j], acc);
      a.t.W[((b * a.nseg) + lc_seg_offset(gc - 1) + P) * (2 * LC_M) + sigma * LC_M + k] = acc;
    }
  }
}

// Coupling (Step 3), all levels in one launch.  Forward: one output row
// segment v per group of 18 threads:
//   v even: c = A-hat(b,0) w(2b+2) + A-hat(b,1) w(2b+3);  v odd: c = A-hat(b,2) w(2b+3).
// Transposed: one output column segment g:
//   g even: c = A-hat(b,0)^T w(2b), b = (g-2)/2;
//   g odd:  c = A-hat(b,1)^T w(2b) + A-hat(b,2)^T w(2b+1), b = (g-3)/2.
template <typename R, bool kAdj>
__global__ void k_couple(Args<R> a) {
  const int seg = threadIdx.x / LC_M;
  const int k = threadIdx.x % LC_M;
  const int64_t t = int64_t(blockIdx.x) * kCoupleSegs + seg;
  if (seg >= kCoupleSegs || t >= a.nseg) return;
  int gamma = 0;
  while (gamma + 1 < a.L && t >= lc_seg_offset(gamma + 1)) ++gamma;
  const int64_t v = t - lc_seg_offset(gamma);
  const int64_t nrow = (int64_t(4) << gamma) - 2;  // 2 b_gamma
  const int64_t aoff = lc_ahat_offset(gamma);
  const R* Ah = a.t.Ahat;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    const R* Wl = a.t.W + ((b * a.nseg) + lc_seg_offset(gamma)) * (2 * LC_M);
    R* Cl = a.t.Cc + ((b * a.nseg) + lc_seg_offset(gamma)) * (2 * LC_M);
    R c0 = R(0), c1 = R(0);
    if (!kAdj) {
      if (v >= nrow) continue;
      const int64_t bb = v >> 1;
      if ((v & 1) == 0) {
        const R* A0 = Ah + (aoff + 3 * bb + 0) * (LC_M * LC_M) + k * LC_M;
        const R* A1 = Ah + (aoff + 3 * bb + 1) * (LC_M * LC_M) + k * LC_M;
        const R* w0 = Wl + (v + 2) * (2 * LC_M);
        const R* w1 = Wl + (v + 3) * (2 * LC_M);
        for (int l = 0; l < LC_M; ++l) {
          c0 = fma(A0[l], w0[l], c0);
          c1 = fma(A0[l], w0[LC_M + l], c1);
          c0 = fma(A1[l], w1[l], c0);
          c1 = fma(A1[l], w1[LC_M + l], c1);
        }
      } else {
        const R* A2 = Ah + (aoff + 3 * bb + 2) * (LC_M * LC_M) + k * LC_M;
        const R* w0 = Wl + (v + 2) * (2 * LC_M);
        for (int l = 0; l < LC_M; ++l) {
          c0 = fma(A2[l], w0[l], c0);
          c1 = fma(A2[l], w0[LC_M + l], c1);
        }
      }
    } else {
      const int64_t g = v;
      if (g < 2) continue;
      if ((g & 1) == 0) {
        const int64_t bb = (g - 2) >> 1;
        const R* A0 = Ah + (aoff + 3 * bb + 0) * (LC_M * LC_M) + k;
        const R* w0 = Wl + (2 * bb) * (2 * LC_M);
        for (int l = 0; l < LC_M; ++l) {
          c0 = fma(A0[l * LC_M], w0[l], c0);
          c1 = fma(A0[l * LC_M], w0[LC_M + l], c1);
        }
      } else {
        const int64_t bb = (g - 3) >> 1;
        const R* A1 = Ah + (aoff + 3 * bb + 1) * (LC_M * LC_M) + k;
        const R* A2 = Ah + (aoff + 3 * bb + 2) * (LC_M * LC_M) + k;
        const R* w0 = Wl + (2 * bb) * (2 * LC_M);
        const R* w1 = Wl + (2 * bb + 1) * (2 * LC_M);
        for (int l = 0; l < LC_M; ++l) {
          c0 = fma(A1[l * LC_M], w0[l], c0);
          c1 = fma(A1[l * LC_M], w0[LC_M + l], c1);
          c0 = fma(A2[l * LC_M], w1[l], c0);
          c1 = fma(A2[l * LC_M], w1[LC_M + l], c1);
        }
      }
    }
    Cl[v * (2 * LC_M) + k] = c0;
    Cl[v * (2 * LC_M) + LC_M + k] = c1;
  }
}

// Downward pass (Step 4): level gp -> gp+1 for children v in [lo, hi):
//   c(gp+1, v) += B(v mod 2)^T c(gp, v/2), with b(1)_jk = (-1)^(j-k) b(0)_jk.
template <typename R>
__global__ void k_down(Args<R> a, int gp, int64_t lo, int64_t hi) {
  __shared__ R Bs[LC_M * LC_M];
  __shared__ R par[kSegs][2][LC_M];
  for (int i = threadIdx.x; i < LC_M * LC_M; i += blockDim.x) Bs[i] = a.t.B[i];
  const int seg = threadIdx.x / kThreadsSeg;
  const int sigma = (threadIdx.x % kThreadsSeg) / LC_M;
  const int k = threadIdx.x % LC_M;
  const int64_t v = lo + int64_t(blockIdx.x) * kSegs + seg;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    __syncthreads();
    if (seg < kSegs && v < hi)
      par[seg][sigma][k] = a.t.Cc[((b * a.nseg) + lc_seg_offset(gp) + (v >> 1)) * (2 * LC_M) + sigma * LC_M + k];
    __syncthreads();
    if (seg < kSegs && v < hi) {
      R acc = R(0);
      const bool odd = (v & 1) != 0;
      for (int j = k; j < LC_M; ++j) {
        const R bjk = Bs[j * LC_M + k];
        acc = fma((odd && ((j - k) & 1)) ? negate(bjk) : bjk, par[seg][sigma][j], acc);
      }
      a.t.Cc[((b * a.nseg) + lc_seg_offset(gp + 1) + v) * (2 * LC_M) + sigma * LC_M + k] += acc;
    }
  }
}

// Steps 5-7 for the forward pass: one thread per output row i < n.
template <typename R>
__global__ void k_final(Args<R> a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int s = a.s, L = a.L;
  const int64_t two_s = 2 * int64_t(s);
  const int64_t v = i / two_s;
  const int l = int(i - v * two_s);
  const int m = l >> 1, sigma = l & 1;
  const int64_t nleaf_rows = (int64_t(2) << L) - 2;
  const int64_t end = (L > 0) ? min(a.n, two_s * (v + 2)) : a.n;
  const R* Trow = a.t.T + (sigma * s + m) * LC_M;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    const typename lc_io<R>::type* f = a.in + b * a.ib;
    R far = R(0);
    if (L > 0 && v < nleaf_rows) {
      const R* c = a.t.Cc + ((b * a.nseg) + lc_seg_offset(L - 1) + v) * (2 * LC_M) + sigma * LC_M;
      for (int k = 0; k < LC_M; ++k) far = fma(c[k], Trow[k], far);
    }
    R near = R(0);
    R res;
    if (a.dir == LC_L2C) {
      // a_{i,i+2k} = lambda_k lambda_{i+k}   (eq:hik)
      int64_t kk = 0;
      for (int64_t j = i; j < end; j += 2, ++kk) near = fma(a.t.lam[kk] * a.t.lam2[i + kk], lc_ld<R>(f + j * a.ie), near);
      res = cinv<R>(i) * (far + near);
    } else {
      // L(i, i+2k) = (2i+1)(i+2k) u_k v_{i+k}; L(0,0) = 1   (eq:Lxymod)
      int64_t kk = 0;
      for (int64_t j = i; j < end; j += 2, ++kk)
        near = fma(a.t.lam[kk] * a.t.lam2[i + kk], R(j) * lc_ld<R>(f + j * a.ie), near);
      near *= R(2 * i + 1);
      if (i == 0) near += lc_ld<R>(f);
      res = far + near;
    }
    lc_st<R>(a.out + b * a.ob + i * a.oe, res);
  }
}

// Transposed Steps 7-5: one thread per output column j < n:
//   g_j = [spread of c over column segment j/2s] + sum_{band rows i of column j} M_ij r_i
// with r scaled by C^{-1} for L2C.  Band rows of column j: i <= j, same
// parity, floor(i/2s) >= floor(j/2s) - 1.
template <typename R>
__global__ void k_final_adj(Args<R> a) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const int s = a.s, L = a.L;
  const int64_t two_s = 2 * int64_t(s);
  const int64_t g = j / two_s;
  const int l = int(j - g * two_s);
  const int m = l >> 1, sigma = l & 1;
  int64_t start = (L > 0) ? max(int64_t(0), two_s * (g - 1)) : 0;
  if ((start & 1) != (j & 1)) ++start;
  const R* Trow = a.t.T + (sigma * s + m) * LC_M;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    const typename lc_io<R>::type* r = a.in + b * a.ib;
    R far = R(0);
    if (L > 0 && g >= 2) {
      const R* c = a.t.Cc + ((b * a.nseg) + lc_seg_offset(L - 1) + g) * (2 * LC_M) + sigma * LC_M;
      for (int k = 0; k < LC_M; ++k) far = fma(c[k], Trow[k], far);
    }
    R near = R(0);
    if (a.dir == LC_L2C) {
      for (int64_t i = start; i <= j; i += 2) {
        const int64_t k = (j - i) >> 1;
        near = fma(a.t.lam[k] * a.t.lam2[i + k], cinv<R>(i) * lc_ld<R>(r + i * a.ie), near);
      }
    } else {
      for (int64_t i = start; i <= j; i += 2) {
        const int64_t k = (j - i) >> 1;
        near = fma(a.t.lam[k] * a.t.lam2[i + k], R(2 * i + 1) * lc_ld<R>(r + i * a.ie), near);
      }
      near *= R(j);
      if (j == 0) near += lc_ld<R>(r);
    }
    lc_st<R>(a.out + b * a.ob + j * a.oe, far + near);
  }
}

template <typename R>
lc_status run(lc_plan_s* p, Args<R> a, cudaStream_t st, int adjoint) {
  const int L = a.L, s = a.s;
  lc_timer_begin(p);
  const int gy = int(a.batch < 65535 ? a.batch : 65535);
  if (L > 0) {
    // leaf restriction: column segments [2, 2^(L+1)) forward, row segments [0, 2^(L+1)-2) transposed
    const int64_t lo = adjoint ? 0 : 2;
    const int64_t hi = adjoint ? ((int64_t(2) << L) - 2) : (int64_t(2) << L);
    const size_t sm = (size_t(2) * s * LC_M + kSegs * 2 * s) * sizeof(R);
    dim3 grid(unsigned((hi - lo + kSegs - 1) / kSegs), gy);
    lc_timer_mark(p, st, LC_K_LEAF);
    k_leaf<R><<<grid, kSegs * kThreadsSeg, sm, st>>>(a, lo, hi, (adjoint && a.dir == LC_L2C) ? 1 : 0);
    LC_LAUNCH_CHECK();
    for (int gc = L - 1; gc >= 1; --gc) {
      // parents at level gc-1: [2, 2^(gc+1)) forward (column tree), [0, 2^(gc+1)-2) transposed (row tree)
      const int64_t plo = adjoint ? 0 : 2;
      const int64_t phi = adjoint ? ((int64_t(2) << gc) - 2) : (int64_t(2) << gc);
      dim3 g2(unsigned((phi - plo + kSegs - 1) / kSegs), gy);
      lc_timer_mark(p, st, LC_K_UP);
      k_up<R><<<g2, kSegs * kThreadsSeg, 0, st>>>(a, gc, plo, phi);
      LC_LAUNCH_CHECK();
    }
    dim3 g3(unsigned((a.nseg + kCoupleSegs - 1) / kCoupleSegs), gy);
    lc_timer_mark(p, st, LC_K_COUPLE);
    if (adjoint)
      k_couple<R, true><<<g3, kCoupleSegs * LC_M, 0, st>>>(a);
    else
      k_couple<R, false><<<g3, kCoupleSegs * LC_M, 0, st>>>(a);
    LC_LAUNCH_CHECK();
    for (int gp = 0; gp + 1 <= L - 1; ++gp) {
      // children at level gp+1: [0, 2^(gp+3)-4) forward (row tree), [4, 2^(gp+3)) transposed (column tree)
      const int64_t clo = adjoint ? 4 : 0;
      const int64_t chi = adjoint ? (int64_t(8) << gp) : ((int64_t(8) << gp) - 4);
      dim3 g4(unsigned((chi - clo + kSegs - 1) / kSegs), gy);
      lc_timer_mark(p, st, LC_K_DOWN);
      k_down<R><<<g4, kSegs * kThreadsSeg, 0, st>>>(a, gp, clo, chi);
      LC_LAUNCH_CHECK();
    }
  }
  dim3 g5(unsigned((a.n + kFinalThreads - 1) / kFinalThreads), gy);
  lc_timer_mark(p, st, LC_K_FINAL);
  if (adjoint)
    k_final_adj<R><<<g5, kFinalThreads, 0, st>>>(a);
  else
    k_final<R><<<g5, kFinalThreads, 0, st>>>(a);
  LC_LAUNCH_CHECK();
  lc_timer_end(p, st);
  return LC_OK;
}

}  // namespace lc_exec
