// lc_plan.cu -- plan geometry, FP64 plan builder kernels and the C ABI front door.
//
// Plan contents (all computed in FP64 on the GPU):
//   lambda_i = Lambda(i), i < N: every 8th value from the tau series (eq:tau,
//       Lambda(z) = tau(z+1/4)/sqrt(z+1/4)), the 7 in between by the
//       recursion Lambda(i) = Lambda(i-1)(i-1/2)/i (eq:Lambdaint); the first
//       24 values by the recursion from Lambda(0) = sqrt(pi)  (Sec. 4.3).
//   T(sigma)_{mk} = T_k(-1 + (2m+sigma)/s)  (eq:Xs), by the three-term recurrence.
//   B(0)_{kj}: T_k((Y-1)/2) = sum_j b_kj T_j(Y)  (eq:Tmap).  Built exactly from
//       the Chebyshev recurrence T_{k+1}(u) = 2u T_k(u) - T_{k-1}(u) with
//       u = (Y-1)/2 and Y T_j = (T_{j+1} + T_{j-1})/2; every entry is a dyadic
//       rational, so FP64 holds it exactly (Appendix A.3 gives the same matrix
//       as W^{-1} V(0) W).  B(1) differs only in the sign of odd diagonals.
//   A-hat(gamma,b,r): the kernel A(x,y) = Lambda((y-x)/2) Lambda((y+x)/2)
//       (Sec. 3.2) or, for C2L, L(x,y) of eq:Lxymod, sampled at M x M
//       Chebyshev-Gauss points of the submatrix domain (eq:Xfromx) and
//       transformed with the 2-D DCT-II of eq:aklmore.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lc_df.cuh"
#include "lc_internal.cuh"

// ------------------------------------------------------------------ Lambda --
// Lambda(z) for real z > 0 via the tau series (eq:tau).  The series reaches
// machine precision for z > 19.88; below 20 the argument is first shifted up
// with Lambda(z) = Lambda(z+1) (z+1)/(z+1/2), which follows from
// Gamma(x+1) = x Gamma(x).
__device__ double lc_Lambda(double z) {
  double f = 1.0;
  while (z < 20.0) {
    f *= (z + 1.0) / (z + 0.5);
    z += 1.0;
  }
  const double y = z + 0.25;
  const double x = 1.0 / (y * y);
  const double tau =
      1.0 + x * (-1.0 / 64.0 + x * (21.0 / 8192.0 + x * (-671.0 / 524288.0 + x * (180323.0 / 134217728.0))));
  return f * tau / sqrt(y);
}

// The same series for the kernel samples inside A-hat (entries needed to a
// block-relative 1e-14, not to a few ulp): one reciprocal square root gives
// both y^(-1/2) and x = y^(-2), instead of two divisions and a square root,
// and the series keeps only the terms it needs at z: the paper notes that 4,
// 3 or 2 terms reach machine precision above z = 40, 134 or 1844 (Sec. 4.3).
__device__ __forceinline__ double tau_terms(double z, double x) {
  if (z > 1844.0) return 1.0 + x * (-1.0 / 64.0);
  if (z > 134.0) return 1.0 + x * (-1.0 / 64.0 + x * (21.0 / 8192.0));
  if (z > 40.0) return 1.0 + x * (-1.0 / 64.0 + x * (21.0 / 8192.0 + x * (-671.0 / 524288.0)));
  return 1.0 + x * (-1.0 / 64.0 + x * (21.0 / 8192.0 + x * (-671.0 / 524288.0 + x * (180323.0 / 134217728.0))));
}
__device__ double lc_Lambda_sample(double z) {
  double f = 1.0;
  while (z < 20.0) {
    f *= (z + 1.0) / (z + 0.5);
    z += 1.0;
  }
  const double y = z + 0.25;
  const double r = rsqrt(y);
  const double r2 = r * r;
  return f * tau_terms(z, r2 * r2) * r;
}

// 1 / (w (w + 1) Lambda(w/2)), the factor of L(x, y) (eq:Lxymod) that depends
// on w = x + y, without a division.  With z = w/2 and y = z + 1/4:
// w (w + 1) = 4 (y^2 - 1/16), and 1/Lambda(z) = y^(1/2) / tau(y^(-2)); so the
// factor is y^(-3/2) / 4 times Q(x) = (1/tau(x)) (1/(1 - x/16)), x = y^(-2),
// whose power series (the reciprocal of eq:tau's series times a geometric
// series, truncated at x^4 like eq:tau) has the dyadic coefficients below and
// the same accuracy as eq:tau: 2e-16 relative at z = 19.88, with 4, 3 or 2
// terms enough above z = 40, 134 or 1844 (checked at 40 digits).  Below
// z = 20 the argument is shifted up as in lc_Lambda, with one division.
__device__ double lc_c2l_wfactor(double w) {
  double z = 0.5 * w;
  if (z < 20.0) return 1.0 / (w * (w + 1.0) * lc_Lambda_sample(z));
  const double y = z + 0.25;
  const double r = rsqrt(y);
  const double r2 = r * r;
  const double x = r2 * r2;
  double q;
  if (z > 1844.0) q = 1.0 + x * (5.0 / 64.0);
  else if (z > 134.0) q = 1.0 + x * (5.0 / 64.0 + x * (21.0 / 8192.0));
  else if (z > 40.0) q = 1.0 + x * (5.0 / 64.0 + x * (21.0 / 8192.0 + x * (715.0 / 524288.0)));
  else q = 1.0 + x * (5.0 / 64.0 + x * (21.0 / 8192.0 + x * (715.0 / 524288.0 + x * (-162877.0 / 134217728.0))));
  return 0.25 * r2 * r * q;
}

__global__ void k_plan_lambda(int64_t N, double* __restrict__ lam) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i0 = 8 * t;
  if (i0 >= N) return;
  double v;
  int64_t start;
  if (i0 < 24) {
    v = 1.7724538509055160273;  // Lambda(0) = Gamma(1/2) = sqrt(pi)
    for (int64_t i = 1; i <= i0; ++i) v *= (double(2 * i - 1) / double(2 * i));
    start = i0;
  } else {
    v = lc_Lambda(double(i0));
    start = i0;
  }
  lam[start] = v;
  for (int64_t i = start + 1; i < start + 8 && i < N; ++i) {
    v *= (double(2 * i - 1) / double(2 * i));
    lam[i] = v;
  }
}

// C2L near-field tables: L(i, i+2k) = (2i+1)(i+2k) u_k v_{i+k} with
// u_k = Lambda(k)/(1-2k) and v_m = 1/(2m(2m+1) Lambda(m)) -- a factorisation
// of eq:Lxymod at x = i, y = i + 2k.  v_0 = 0; entry (0,0) = 1 is added
// separately.  Input: lambda in v (overwritten in place).
// One division per m: with d = 2m(2m+1) lambda_m and q = 1 / ((1-2m) d),
// u_m = lambda_m d q and v_m = (1-2m) q (a few ulp).
__global__ void k_plan_c2l_tables(int64_t N, double* __restrict__ u, double* __restrict__ v) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const double l = v[m];
  if (m == 0) {
    u[0] = l;
    v[0] = 0.0;
    return;
  }
  const double one_m = double(1 - 2 * m);
  const double d = double(2 * m) * double(2 * m + 1) * l;
  const double q = 1.0 / (one_m * d);
  u[m] = l * d * q;
  v[m] = one_m * q;
}

// ------------------------------------------------------------- Gegenbauer --
// Gamma(z + p)/Gamma(z + q) for real z with z + min(p, q) > 0: shifted up to
// z >= 20 by Gamma(x+1) = x Gamma(x), then v^(p-q) times the series pc in
// x = 1/v^2, v = z + (p + q - 1)/2 (lc_geg).
__device__ double lc_gratio(double z, double pa, double qb, const double* pc) {
  double f = 1.0;
  for (int it = 0; it < 64 && z < 20.0; ++it) {
    f *= (z + qb) / (z + pa);
    z += 1.0;
  }
  const double v = z + 0.5 * (pa + qb - 1.0);
  const double x = 1.0 / (v * v);
  double q = pc[LC_GEG_TERMS];
  for (int j = LC_GEG_TERMS - 1; j >= 0; --j) q = fma(q, x, pc[j]);
  return f * q * pow(v, pa - qb);
}
__device__ __forceinline__ double lc_geg_lam(const lc_geg& G, double z) {
  return G.c_lam * lc_gratio(z, G.alpha, 1.0, G.p_lam);
}
__device__ __forceinline__ double lc_geg_u(const lc_geg& G, double z) {
  return G.c_u * lc_gratio(z, -G.alpha, 1.0, G.p_u);
}
__device__ __forceinline__ double lc_geg_v(const lc_geg& G, double z) {
  return lc_gratio(z, 0.0, G.alpha + 1.0, G.p_v);
}

// Near-field tables of a Gegenbauer plan, 8 consecutive indices per thread:
// the first from the series (from the start value below index 24), the rest
// by the ratio recursions g_k = g_(k-1) (k-1+a)/k, u_k = u_(k-1) (k-1-a)/k,
// v_m = v_(m-1) (m-1)/(m+a).  L2C: lam = sqrt(pi) g; C2L: lam = u, lam2 = v.
__global__ void k_plan_geg_tables(int64_t N, int dir, lc_geg G, double* __restrict__ lam,
                                  double* __restrict__ lam2) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t i0 = 8 * t;
  if (i0 >= N) return;
  const double a = G.alpha;
  const double ua = dir == LC_L2C ? a : -a;  // g or u recursion
  double x;
  int64_t k = 0;
  if (i0 < 24) {
    x = dir == LC_L2C ? 1.7724538509055160273 : G.u0;
    for (k = 1; k <= i0; ++k) x *= (double(k - 1) + ua) / double(k);
  } else {
    x = dir == LC_L2C ? lc_geg_lam(G, double(i0)) : lc_geg_u(G, double(i0));
  }
  lam[i0] = x;
  for (k = i0 + 1; k < i0 + 8 && k < N; ++k) {
    x *= (double(k - 1) + ua) / double(k);
    lam[k] = x;
  }
  if (dir == LC_L2C) return;
  double v;
  if (i0 < 24) {
    v = G.v1;
    for (k = 2; k <= i0; ++k) v *= double(k - 1) / (double(k) + a);
  } else {
    v = lc_geg_v(G, double(i0));
  }
  lam2[i0] = i0 == 0 ? 0.0 : v;
  for (k = i0 + 1; k < i0 + 8 && k < N; ++k) {
    if (k >= 2) v *= double(k - 1) / (double(k) + a);
    lam2[k] = v;
  }
}

__device__ __forceinline__ void plan_T_row(int t, int s, double* __restrict__ T) {
  const int sigma = t / s, m = t % s;
  const double X = -1.0 + double(2 * m + sigma) / double(s);
  double* row = T + (size_t(sigma) * s + m) * LC_M;
  double t0 = 1.0, t1 = X;
  row[0] = t0;
  row[1] = t1;
  for (int k = 2; k < LC_M; ++k) {
    const double t2 = 2.0 * X * t1 - t0;
    row[k] = t2;
    t0 = t1;
    t1 = t2;
  }
}

// B(0) by the exact row recurrence (M^2 work).  One warp: row k+1 from rows k and k-1, entry i per lane (rows are
// independent across i, sequential in k).
__device__ __forceinline__ void plan_B_warp(int i, double* __restrict__ B) {
  for (int t = i; t < LC_M * LC_M; t += 32) B[t] = 0.0;
  __syncwarp();
  if (i == 0) {
    B[0] = 1.0;          // T_0(u) = 1
    B[LC_M + 0] = -0.5;  // T_1(u) = u = Y/2 - 1/2
    B[LC_M + 1] = 0.5;
  }
  __syncwarp();
  for (int k = 1; k + 1 < LC_M; ++k) {
    const double* bk = B + k * LC_M;
    const double* bm = B + (k - 1) * LC_M;
    double* bn = B + (k + 1) * LC_M;
    if (i <= k + 1) {
      // Y * T_k(u) expanded in T_j(Y): T_0 -> T_1, T_j -> (T_{j+1} + T_{j-1})/2.
      double y = 0.0;
      if (i == 1) y += bk[0];
      if (i >= 2) y += 0.5 * bk[i - 1];
      if (i + 1 <= k) y += 0.5 * bk[i + 1];
      // T_{k+1}(u) = (Y - 1) T_k(u) - T_{k-1}(u)
      const double own = (i <= k) ? bk[i] : 0.0;
      const double prev = (i <= k - 1) ? bm[i] : 0.0;
      bn[i] = y - own - prev;
    }
    __syncwarp();
  }
}

// Nodal variant (eq:AijLag): Lagrange basis l_k(X) of the M Chebyshev-Gauss
// nodes X_k = cos((k+1/2) pi/M), in the second (true) barycentric form with
// the weights of first-kind Chebyshev points, w_k = (-1)^k sin((k+1/2) pi/M);
// a point on a node gives the Kronecker delta.
__device__ double lc_lagrange(int k, double X) {
  double num = 0.0, den = 0.0;
  for (int j = 0; j < LC_M; ++j) {
    const double d = X - cospi((j + 0.5) / LC_M);
    const double w = ((j & 1) ? -1.0 : 1.0) * sinpi((j + 0.5) / LC_M);
    if (d == 0.0) return j == k ? 1.0 : 0.0;
    const double t = w / d;
    den += t;
    if (j == k) num = t;
  }
  return num / den;
}
// Leaf matrices of the nodal variant, T(sigma)_{mk} = l_k(-1 + (2m+sigma)/s):
// Step 1 gives the leaf's expansion on its own Lagrange basis (the nodal w).
__global__ void k_plan_nodal_T(int s, double* __restrict__ T) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * s * LC_M) return;
  const int sigma = t / (s * LC_M), m = (t / LC_M) % s, k = t % LC_M;
  T[t] = lc_lagrange(k, -1.0 + double(2 * m + sigma) / double(s));
}
// Level maps of the nodal variant, P(l)_{kj} = l_k((X_j + 2l - 1)/2): a
// parent's Lagrange basis at the nodes of child l (the nodal counterpart of
// B(l), eq:Tmap; dense).  Table [2][M][M].
__global__ void k_plan_nodal_P(double* __restrict__ B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * LC_M * LC_M) return;
  const int l = t / (LC_M * LC_M), k = (t / LC_M) % LC_M, j = t % LC_M;
  B[t] = lc_lagrange(k, 0.5 * (cospi((j + 0.5) / LC_M) + double(2 * l - 1)));
}

// cosm[k][m] = cos(k (m + 1/2) pi / M): the DCT-II matrix of eq:aklmore.
// Row 1 holds the Chebyshev-Gauss points X_m.
__device__ __forceinline__ void plan_cos_entry(int t, double* __restrict__ cosm) {
  const int k = t / LC_M, m = t % LC_M;
  cosm[t] = cospi(double(k * (2 * m + 1)) / double(2 * LC_M));
}
// X_m = cosm[1][m], by the same expression.
__device__ __forceinline__ double lc_node(int m) { return cospi(double(1 * (2 * m + 1)) / double(2 * LC_M)); }
// T(sigma) and B(0) in one launch of two CTAs (the tables are tiny; separate
// launches cost more than their work).  Tdf and Bdf, if given, receive
// double-float copies.
__device__ __forceinline__ void plan_basis_block(int blk, int s, double* __restrict__ T, double* __restrict__ B,
                                                 lc_df* __restrict__ Tdf, lc_df* __restrict__ Bdf) {
  if (blk == 0) {
    if (threadIdx.x < 2 * s) {
      plan_T_row(threadIdx.x, s, T);
      if (Tdf)
        for (int k = 0; k < LC_M; ++k) {
          const size_t e = size_t(threadIdx.x) * LC_M + k;
          Tdf[e] = lc_df_from_double(T[e]);
        }
    }
  } else if (threadIdx.x < 32) {
    plan_B_warp(threadIdx.x, B);
    __syncwarp();
    if (Bdf)
      for (int t = threadIdx.x; t < LC_M * LC_M; t += 32) Bdf[t] = lc_df_from_double(B[t]);
  }
}
__global__ void k_plan_basis(int s, double* __restrict__ T, double* __restrict__ B) {
  plan_basis_block(blockIdx.x, s, T, B, nullptr, nullptr);
}

// Lambda((y - x)/2) at the M x M Chebyshev-Gauss points of a submatrix
// depends only on its level and on the offset j0 - i0, which is 4h for
// (p,q) = (0,0), (1,1) and 6h for (0,1) (eq:globalij): 2 M x M tables per
// level, shared by every block of the level (Sec. 4.3 reuses Lambda^- the
// same way).  Table [L][2][M][M].
// For C2L the table holds Lambda((y-x)/2) / (x - y + 1), the other factor of
// L(x, y) that depends only on y - x (eq:Lxymod).
// The launch also writes the DCT matrix cosm (its first M^2 threads), which
// the A-hat kernels read; the nodes here come from the same formula.
__global__ void k_plan_lminus(int L, int s, int dir, lc_geg G, double* __restrict__ cosm,
                              double* __restrict__ tab, lc_df* __restrict__ tab_df) {
  __shared__ double X[LC_M];  // the nodes, once per CTA
  if (threadIdx.x < LC_M) X[threadIdx.x] = lc_node(threadIdx.x);
  __syncthreads();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < LC_M * LC_M) plan_cos_entry(int(t), cosm);
  if (t >= int64_t(L) * 2 * LC_M * LC_M) return;
  const int gamma = int(t / (2 * LC_M * LC_M));
  const int c = int((t / (LC_M * LC_M)) % 2);
  const int m = int((t / LC_M) % LC_M), n = int(t % LC_M);
  const double h = double(int64_t(s) << (L - gamma - 1));
  const double off = (c == 0 ? 4.0 : 6.0) * h;  // j0 - i0
  // (y_n - x_m)/2 with x_m = i0 + h (X_m + 1), y_n = j0 + h (Y_n + 1)   (eq:Xfromx)
  const double ymx = off + h * (X[n] - X[m]);
  if (G.on) {  // Gegenbauer: lambda_a((y-x)/2) or u_a((y-x)/2)
    tab[t] = dir == LC_L2C ? lc_geg_lam(G, 0.5 * ymx) : lc_geg_u(G, 0.5 * ymx);
    return;
  }
  const double l = lc_Lambda(0.5 * ymx);
  const double v = dir == LC_L2C ? l : l / (1.0 - ymx);
  tab[t] = v;
  if (tab_df) tab_df[t] = lc_df_from_double(v);  // the double-float plan's copy
}

// One CTA (M*M threads) per submatrix: sample the kernel, then the 2-D DCT-II
// of eq:aklmore.  Lambda((x+y)/2) is symmetric in (m, n) because X and Y use
// the same nodes, so only m <= n is evaluated; the DCT matrix satisfies
// cos(k(M-1-m+1/2)pi/M) = (-1)^k cos(k(m+1/2)pi/M), so each 18-term sum is
// folded into 9 terms of sums or differences.
// GEG: Gegenbauer kernel samples (lc_geg); NODAL: keep the samples (eq:AijLag)
// instead of their DCT.  Template flags, so that the Legendre modal
// instantiation carries no code of the other variants.
template <bool GEG, bool NODAL>
__global__ void k_plan_ahat(int L, int s, int dir, int64_t nc, const double* __restrict__ cosm,
                            const double* __restrict__ lminus, double* __restrict__ Ahat, const lc_geg geg) {
  constexpr int H = LC_M / 2;
  __shared__ double S[LC_M][LC_M];
  __shared__ double F[2][H][LC_M];  // folded rows: sums (even k) and differences (odd k)
  __shared__ double Tm[LC_M][LC_M];
  __shared__ double G[2][LC_M][H];  // Tm folded along the column variable
  __shared__ double cs[LC_M][LC_M];
  const int tid = threadIdx.x;
  const int r0 = tid / LC_M, c0 = tid % LC_M;
  cs[r0][c0] = cosm[tid];
  // The symmetric factor is evaluated once per pair m <= n: 171 pairs on
  // threads 0..170 (6 warps, full) rather than on the threads whose (r0, c0)
  // happen to satisfy r0 <= c0 (every warp, half of each).
  constexpr int kPairs = LC_M * (LC_M + 1) / 2;
  int pm = 0, pn = 0;
  if (tid < kPairs) {
    int rest = tid;
    while (rest >= LC_M - pm) {
      rest -= LC_M - pm;
      ++pm;
    }
    pn = pm + rest;
  }
  for (int64_t a = blockIdx.x; a < nc; a += gridDim.x) {
    int gamma = 0;
    while (gamma + 1 < L && a >= lc_ahat_offset(gamma + 1)) ++gamma;
    const int64_t rem = a - lc_ahat_offset(gamma);
    const int64_t b = rem / 3;
    const int r = int(rem % 3);
    const int p = (r == 2) ? 1 : 0;
    const int q = (r == 0) ? 0 : 1;
    const double h = double(int64_t(s) << (L - gamma - 1));
    const double i0 = 2.0 * h * double(2 * b + p);
    const double j0 = 2.0 * h * double(2 * b + q + 2);
    const double* lm = lminus + (size_t(gamma) * 2 + (r == 1 ? 1 : 0)) * (LC_M * LC_M);
    __syncthreads();
    if (tid < kPairs) {  // the factor that depends on x_m + y_n: symmetric in (m, n)
      const double w = i0 + j0 + h * (cs[1][pm] + cs[1][pn] + 2.0);
      // L2C: Lambda((x+y)/2); C2L: 1 / ((x+y)(x+y+1) Lambda((x+y)/2))
      double lp;
      if constexpr (GEG)  // Gegenbauer: lambda_a((x+y)/2) or v_a((x+y)/2)
        lp = dir == LC_L2C ? lc_geg_lam(geg, 0.5 * w) : lc_geg_v(geg, 0.5 * w);
      else
        lp = dir == LC_L2C ? lc_Lambda_sample(0.5 * w) : lc_c2l_wfactor(w);
      S[pm][pn] = lp;
      S[pn][pm] = lp;
    }
    __syncthreads();
    {
      const double x = i0 + h * (cs[1][r0] + 1.0);
      const double y = j0 + h * (cs[1][c0] + 1.0);
      const double lmi = lm[tid];
      double val;
      if (dir == LC_L2C) {
        val = lmi * S[r0][c0];  // A(x, y) = Lambda((y-x)/2) Lambda((y+x)/2)
      } else {                  // L(x, y) of eq:Lxymod, no division
        val = 2.0 * (x + (GEG ? 0.5 * geg.two_alpha : 0.5)) * y * lmi * S[r0][c0];
      }
      if constexpr (NODAL) {  // eq:AijLag: the samples themselves are the block's representation
        Ahat[a * (LC_M * LC_M) + tid] = val;
        continue;
      }
      __syncthreads();
      S[r0][c0] = val;
    }
    __syncthreads();
    if (tid < 2 * H * LC_M) {  // fold the row variable
      const int e = tid / (H * LC_M), mm = (tid / LC_M) % H, n = tid % LC_M;
      const double u = S[mm][n], v = S[LC_M - 1 - mm][n];
      F[e][mm][n] = e ? u - v : u + v;
    }
    __syncthreads();
    {  // DCT along the row variable: Tm[k][n] = sum_m cos(k(m+1/2)pi/M) S[m][n]
      double acc = 0.0;
      const int e = r0 & 1;
      for (int mm = 0; mm < H; ++mm) acc = fma(cs[r0][mm], F[e][mm][c0], acc);
      Tm[r0][c0] = acc;
    }
    __syncthreads();
    {  // fold the column variable once per (row, nn) instead of once per output
      const int e = tid / (LC_M * H), r = (tid / H) % LC_M, nn = tid % H;
      const double u = Tm[r][nn], v = Tm[r][LC_M - 1 - nn];
      G[e][r][nn] = e ? u - v : u + v;
    }
    __syncthreads();
    {  // DCT along the column variable, then 4/(c_k c_l M^2)
      const int e = c0 & 1;
      double acc = 0.0;
      for (int nn = 0; nn < H; ++nn) acc = fma(G[e][r0][nn], cs[c0][nn], acc);
      const double w = 4.0 / (double(LC_M) * double(LC_M)) * (r0 == 0 ? 0.5 : 1.0) * (c0 == 0 ? 0.5 : 1.0);
      Ahat[a * (LC_M * LC_M) + tid] = acc * w;
    }
  }
}

// ------------------------------------------------- double-float A-hat --
// A-hat for the double-float tier, computed in double-float on the FP32 pipe
// (GB300's FP64 pipe runs at about 1/64 of its FP32 rate) and written straight
// into the compact layout of lc_internal.cuh: the samples and the folded 2-D
// DCT of k_plan_ahat, each operation a double-float one.  Legendre modal
// plans with s >= 10, where every sample has z = (x+y)/2 >= 2s >= 20 (the tau
// series needs no argument shift).  The entries agree with the FP64 plan's to
// a few units of 2^-48 of their matrix (tested).
__device__ __forceinline__ lc_df df_c(double x) { return lc_df_from_double(x); }
// 1/sqrt(y): FP32 estimate and two Newton steps r += r (1 - y r^2) / 2 in
// double-float (the relative error e goes to 1.5 e^2 per step: 2^-22 ->
// 2^-43 -> below the double-float rounding level; one step from an FP32-exact
// start would stop at 2e-14).
__device__ __forceinline__ lc_df df_rsqrt(const lc_df& y) {
  lc_df r(rsqrtf(y.hi), 0.0f);
  for (int it = 0; it < 2; ++it) {
    const lc_df e = lc_df(1.0f, 0.0f) - y * (r * r);
    r = r + lc_df(0.5f * r.hi, 0.5f * r.lo) * e;
  }
  return r;
}
// Lambda(z) (L2C) or 1/(w(w+1) Lambda(w/2)) with w = 2z (C2L), z >= 20: the
// series of lc_Lambda_sample / lc_c2l_wfactor in double-float.
__device__ __forceinline__ lc_df df_sample(int dir, const lc_df& z) {
  const lc_df y = z + lc_df(0.25f, 0.0f);
  const lc_df r = df_rsqrt(y);
  const lc_df r2 = r * r;
  const lc_df x = r2 * r2;  // x <= 1/400^2
  const float zf = z.hi, xf = x.hi;
  // Series 1 + c1 x + x^2 q2(x): the first-order term in double-float, the rest
  // (below 1e-13 of the sum) in FP32; the terms kept above z = 40, 134, 1844
  // as in lc_Lambda_sample.  L2C: tau, c1 = -1/64 (a power of two, exact);
  // C2L: Q, c1 = 5/64.
  float q2;
  if (dir == LC_L2C) {
    if (zf > 1844.0f) q2 = 0.0f;
    else if (zf > 134.0f) q2 = 21.0f / 8192.0f;
    else if (zf > 40.0f) q2 = fmaf(xf, -671.0f / 524288.0f, 21.0f / 8192.0f);
    else q2 = fmaf(xf, fmaf(xf, 180323.0f / 134217728.0f, -671.0f / 524288.0f), 21.0f / 8192.0f);
    const lc_df t = lc_df(1.0f, 0.0f) + lc_df(x.hi * (-1.0f / 64.0f), x.lo * (-1.0f / 64.0f)) +
                    lc_df(xf * xf * q2, 0.0f);
    return t * r;
  }
  if (zf > 1844.0f) q2 = 0.0f;
  else if (zf > 134.0f) q2 = 21.0f / 8192.0f;
  else if (zf > 40.0f) q2 = fmaf(xf, 715.0f / 524288.0f, 21.0f / 8192.0f);
  else q2 = fmaf(xf, fmaf(xf, -162877.0f / 134217728.0f, 715.0f / 524288.0f), 21.0f / 8192.0f);
  const lc_df t = lc_df(1.0f, 0.0f) + x * lc_df(5.0f / 64.0f, 0.0f) + lc_df(xf * xf * q2, 0.0f);
  return lc_df(0.25f, 0.0f) * r2 * r * t;
}

// 1/x for a positive double-float x: FP32 quotient and one Newton step
// r += r (1 - x r) in double-float (relative error 2^-24 -> 2^-48).
__device__ __forceinline__ lc_df df_recip(const lc_df& x) {
  const float r0 = 1.0f / x.hi;
  const lc_df r(r0, 0.0f);
  return r + r * (lc_df(1.0f, 0.0f) - x * r);
}
// The double-float tier's near-field tables, built in double-float: lambda
// (eq:Lambdaint: every 8th from the tau series, the 7 in between by the
// recursion, the first 24 from sqrt(pi)) and, for C2L, u and v from it with
// one reciprocal per entry (the FP64 kernels' formulas).
__device__ __forceinline__ lc_df df_lambda_ratio(int64_t i) {  // (2i - 1) / (2i)
  return lc_df(2 * i - 1) * df_recip(lc_df(2 * i));
}
// C2L: u_m and v_m from lambda_m (one reciprocal), into u[m], v[m].
__device__ __forceinline__ void df_c2l_entry(int64_t m, const lc_df& l, lc_df* __restrict__ u,
                                             lc_df* __restrict__ v) {
  if (m == 0) {
    u[0] = l;
    v[0] = lc_df(0.0f, 0.0f);
    return;
  }
  const lc_df one_m(1 - 2 * m);
  const lc_df d = lc_df(2 * m) * lc_df(2 * m + 1) * l;
  const lc_df q = -df_recip(-(one_m * d));  // one_m d < 0
  u[m] = l * d * q;
  v[m] = one_m * q;
}
// Thread t: lambda_i for i in [8t, 8t + 8); L2C stores them in lam, C2L
// stores u_i in lam and v_i in v.
__device__ __forceinline__ void plan_lambda_df(int64_t t, int64_t N, int dir, lc_df* __restrict__ lam,
                                               lc_df* __restrict__ v2) {
  const int64_t i0 = 8 * t;
  if (i0 >= N) return;
  lc_df v;
  if (i0 < 24) {
    v = df_c(1.7724538509055160273);  // Lambda(0) = sqrt(pi)
    for (int64_t i = 1; i <= i0; ++i) v = v * df_lambda_ratio(i);
  } else {
    v = df_sample(LC_L2C, lc_df(i0));
  }
  for (int64_t i = i0; i < i0 + 8 && i < N; ++i) {
    if (i > i0) v = v * df_lambda_ratio(i);
    if (dir == LC_L2C) lam[i] = v;
    else df_c2l_entry(i, v, lam, v2);
  }
}
// The double-float plan's small tables, as the first aux_ctas(N) CTAs (of M^2
// threads) of the A-hat launch: lambda (u, v) by the CTAs before the last,
// T(sigma) and B(0) with their double-float copies by the last one.
struct DfAux {
  int64_t N;
  int dir, s;
  lc_df* lam;  // L2C: lambda; C2L: u
  lc_df* v2;   // C2L: v
  double* T;
  double* B;
  lc_df* Tdf;
  lc_df* Bdf;
};
inline int64_t df_aux_ctas(int64_t N) { return ((N + 7) / 8 + LC_M * LC_M - 1) / (LC_M * LC_M) + 1; }
__device__ __forceinline__ void plan_df_aux(int64_t cta, int64_t ctas, const DfAux& x) {
  if (cta + 1 < ctas) {
    plan_lambda_df(cta * (LC_M * LC_M) + threadIdx.x, x.N, x.dir, x.lam, x.v2);
    return;
  }
  // T rows by warps 0-3 (2s <= 128), B(0) by warp 4
  if (threadIdx.x < 128) plan_basis_block(0, x.s, x.T, x.B, x.Tdf, x.Bdf);
  else if (threadIdx.x < 160) {
    // plan_basis_block's warp-level B expects lanes 0..31
    const int lane = threadIdx.x - 128;
    plan_B_warp(lane, x.B);
    __syncwarp();
    for (int t = lane; t < LC_M * LC_M; t += 32) x.Bdf[t] = lc_df_from_double(x.B[t]);
  }
}
// Without submatrices (L = 0) the same CTAs run alone.
__global__ void __launch_bounds__(LC_M * LC_M) k_plan_df_aux(DfAux x) { plan_df_aux(blockIdx.x, gridDim.x, x); }

__global__ void __launch_bounds__(LC_M * LC_M, 4) k_plan_ahat_df(int L, int s, int dir, int64_t nc,
                                                               const double* __restrict__ cosm,
                               const lc_df* __restrict__ lminus, float* __restrict__ Af,
                               DfAux aux, int64_t aux_ctas) {
  if (blockIdx.x < aux_ctas) {  // the small tables, beside the first submatrices
    plan_df_aux(blockIdx.x, aux_ctas, aux);
    return;
  }
  constexpr int H = LC_M / 2;
  __shared__ lc_df S[LC_M][LC_M];
  __shared__ lc_df F[2][H][LC_M];
  __shared__ lc_df Tm[LC_M][LC_M];
  __shared__ lc_df G[2][LC_M][H];
  __shared__ lc_df cs[LC_M][LC_M];
  __shared__ lc_df blk[3];  // h, i0, j0 of the current submatrix
  __shared__ int blk_lm;    // its Lambda^- table
  const int tid = threadIdx.x;
  const int r0 = tid / LC_M, c0 = tid % LC_M;
  cs[r0][c0] = df_c(cosm[tid]);
  int gamma = 0;  // thread 0: the level of submatrix a (a only grows)
  const int head = lc_dfa_head(dir), words = lc_dfa_words(dir);
  const int used = LC_M * LC_M + lc_dfa_rowstart(head + 1, head);
  constexpr int kPairs = LC_M * (LC_M + 1) / 2;
  int pm = 0, pn = 0;
  if (tid < kPairs) {
    int rest = tid;
    while (rest >= LC_M - pm) {
      rest -= LC_M - pm;
      ++pm;
    }
    pn = pm + rest;
  }
  // the scale 4/(c_k c_l M^2) of eq:aklmore
  const lc_df wkl = df_c(4.0 / (double(LC_M) * double(LC_M)) * (r0 == 0 ? 0.5 : 1.0) * (c0 == 0 ? 0.5 : 1.0));
  // this thread's places in the two folds and in the compact layout
  const int fe = tid / (H * LC_M), fmm = (tid / LC_M) % H, fn = tid % LC_M;       // row fold
  const int ge = tid / (LC_M * H), grr = (tid / H) % LC_M, gnn = tid % H;       // column fold
  const bool keep_lo = r0 + c0 <= head;
  const int lo_slot = LC_M * LC_M + lc_dfa_rowstart(r0, head) + c0;
  for (int64_t a = blockIdx.x - aux_ctas; a < nc; a += gridDim.x - aux_ctas) {
    __syncthreads();  // the previous submatrix is done with the shared tiles
    if (tid == 0) {   // the submatrix's position, once per CTA (64-bit work, conversions)
      while (gamma + 1 < L && a >= lc_ahat_offset(gamma + 1)) ++gamma;
      const int64_t rem = a - lc_ahat_offset(gamma);
      const int64_t b = rem / 3;
      const int r = int(rem % 3);
      const int p = (r == 2) ? 1 : 0;
      const int q = (r == 0) ? 0 : 1;
      const int64_t hi = int64_t(s) << (L - gamma - 1);
      blk[0] = lc_df(hi);
      blk[1] = lc_df(2 * hi * (2 * b + p));
      blk[2] = lc_df(2 * hi * (2 * b + q + 2));
      blk_lm = (gamma * 2 + (r == 1 ? 1 : 0)) * (LC_M * LC_M);
    }
    __syncthreads();
    const lc_df h = blk[0], i0 = blk[1], j0 = blk[2];
    const lc_df* lm = lminus + blk_lm;
    if (tid < kPairs) {  // symmetric in (m, n): w = x_m + y_n
      const lc_df w = i0 + j0 + h * (cs[1][pm] + cs[1][pn] + lc_df(2.0f, 0.0f));
      const lc_df z = lc_df(0.5f * w.hi, 0.5f * w.lo);
      const lc_df v = df_sample(dir, z);
      S[pm][pn] = v;
      S[pn][pm] = v;
    }
    __syncthreads();
    {
      const lc_df lmi = lm[tid];
      lc_df val;
      if (dir == LC_L2C) {
        val = lmi * S[r0][c0];
      } else {
        const lc_df x = i0 + h * (cs[1][r0] + lc_df(1.0f, 0.0f));
        const lc_df y = j0 + h * (cs[1][c0] + lc_df(1.0f, 0.0f));
        const lc_df x2 = x + x + lc_df(1.0f, 0.0f);  // 2 (x + 1/2)
        val = x2 * y * lmi * S[r0][c0];
      }
      __syncthreads();
      S[r0][c0] = val;
    }
    __syncthreads();
    if (tid < 2 * H * LC_M) {  // fold the row variable
      const lc_df u = S[fmm][fn], v = S[LC_M - 1 - fmm][fn];
      F[fe][fmm][fn] = u + (fe ? -v : v);
    }
    __syncthreads();
    {
      lc_df acc(0.0f, 0.0f);
      const int e = r0 & 1;
#pragma unroll
      for (int mm = 0; mm < H; ++mm) acc = fma(cs[r0][mm], F[e][mm][c0], acc);
      Tm[r0][c0] = acc;
    }
    __syncthreads();
    {
      const lc_df u = Tm[grr][gnn], v = Tm[grr][LC_M - 1 - gnn];
      G[ge][grr][gnn] = u + (ge ? -v : v);
    }
    __syncthreads();
    {
      const int e = c0 & 1;
      lc_df acc(0.0f, 0.0f);
#pragma unroll
      for (int nn = 0; nn < H; ++nn) acc = fma(G[e][r0][nn], cs[c0][nn], acc);
      acc = acc * wkl;
      const lc_df v = lc_df_two_sum(acc.hi, acc.lo);  // normalised: |lo| <= ulp(hi)/2
      float* d = Af + a * words;
      d[tid] = v.hi;
      if (keep_lo) d[lo_slot] = v.lo;
      if (tid < words - used) d[used + tid] = 0.0f;
    }
  }
}

// FP32 copy of A-hat, stored transposed per matrix: [m][l][k].
__global__ void k_d2f_T(int64_t nm, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t total = nm * LC_M * LC_M;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = i / (LC_M * LC_M);
    const int r = int(i % (LC_M * LC_M));
    b[m * (LC_M * LC_M) + (r % LC_M) * LC_M + r / LC_M] = float(a[i]);
  }
}

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = float(a[i]);
}

// -------------------------------------------------------------- geometry --
lc_status lc_compute_geometry(int64_t n, const lc_plan_options* opt, int fixed_default, lc_geom* g) {
  if (n < 1 || n > (int64_t(1) << 40)) return LC_ERR_INVALID_ARG;
  int s_hat = opt ? opt->s_hat : 32;
  int fixed_s = opt ? opt->fixed_s : 0;
  if (fixed_s == 0 && fixed_default) fixed_s = 32;
  if (s_hat < 4 || s_hat > LC_MAX_S) return LC_ERR_INVALID_ARG;
  if (fixed_s != 0 && (fixed_s < 4 || fixed_s > LC_MAX_S)) return LC_ERR_INVALID_ARG;
  memset(g, 0, sizeof(*g));
  g->n = n;
  const int64_t base = fixed_s ? fixed_s : s_hat;
  // smallest t with base 2^t >= n; L = t - 2   (eq:numlevels)
  int t = 0;
  while ((base << t) < n) ++t;
  const int L = t - 2;
  if (L <= 0) {  // the whole upper triangle is near field
    g->L = 0;
    g->s = int(base);
    g->N = n;
    g->nc = 0;
    g->nseg = 0;
    return LC_OK;
  }
  g->L = L;
  if (fixed_s) {
    g->s = fixed_s;
  } else {
    const int64_t d = int64_t(1) << (L + 2);
    g->s = int((n + d - 1) / d);  // in [s_hat/2, s_hat]
  }
  g->N = int64_t(g->s) << (L + 2);                          // eq:Ntot
  g->nc = 3 * ((g->N / (2 * g->s)) - L - 2);                // eq:total_blocks_and_mats
  g->nseg = 4 * ((int64_t(1) << L) - 1);
  return LC_OK;
}

// ------------------------------------------------------- workspace layout --
namespace {
struct carver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

size_t layout(lc_plan_s* p, char* base) {
  carver c{base, 0};
  const lc_geom& g = p->g;
  const size_t N = size_t(g.N);
  const size_t nw = size_t(p->batch) * size_t(g.nseg) * 2 * LC_M;
  p->lam = c.take<double>(N);
  p->lam2 = (p->dir == LC_C2L) ? c.take<double>(N) : p->lam;
  p->err = c.take<int>(64);
  p->T = c.take<double>(size_t(2) * g.s * LC_M);
  p->B = c.take<double>(2 * LC_M * LC_M);  // B(0) (modal) or P(0), P(1) (nodal)
  // + plan scratch: the DCT matrix and the per-level Lambda((y-x)/2) tables
  p->Ahat = c.take<double>(size_t(g.nc) * LC_M * LC_M + LC_M * LC_M + size_t(2 * (g.L > 0 ? g.L : 1)) * LC_M * LC_M);
  p->W = p->Cc = nullptr;
  p->lamf = p->lam2f = p->Tf = p->Bf = p->Ahatf = p->Wf = p->Ccf = nullptr;
  if (p->dtype == LC_F64) {
    p->W = c.take<double>(nw);
    p->Cc = c.take<double>(nw);
  } else if (p->dtype == LC_F32) {
    p->lamf = c.take<float>(N);
    p->lam2f = (p->dir == LC_C2L) ? c.take<float>(N) : p->lamf;
    p->Tf = c.take<float>(size_t(2) * g.s * LC_M);
    p->Bf = c.take<float>(2 * LC_M * LC_M);
    p->Ahatf = c.take<float>(size_t(g.nc) * LC_M * LC_M);
    p->Wf = c.take<float>(nw);
    p->Ccf = c.take<float>(nw);
  } else if (p->dtype == LC_F64_DF) {
    const size_t f2 = 2 * sizeof(float);
    p->df_lam = c.take<char>(N * f2);
    p->df_lam2 = (p->dir == LC_C2L) ? c.take<char>(N * f2) : p->df_lam;
    p->df_T = c.take<char>(size_t(2) * g.s * LC_M * f2);
    p->df_B = c.take<char>(LC_M * LC_M * f2);
    p->df_Ahat = c.take<char>(size_t(g.nc) * lc_dfa_words(p->dir) * sizeof(float));  // compact layout
    p->df_W = c.take<char>(nw * f2);
    p->df_Cc = c.take<char>(nw * f2);
    const size_t nb = size_t(p->batch);
    p->xexp = c.take<int>(nb);
    p->xexp_cnt = c.take<unsigned>(nb);
    p->xexp_part = c.take<int>(nb * size_t((g.n + LC_EXP_CHUNK - 1) / LC_EXP_CHUNK));
  } else if (p->dtype == LC_F64_SPLIT) {
    const size_t sb = lc_split_bytes(p);
    p->split = c.take<char>(sb);
  }
  p->val_tables = nullptr;
  p->val_scratch = nullptr;
  p->val_work = nullptr;
  if (p->opt.values) {
    p->val_tables = c.take<char>(lc_values_table_bytes(g.n));
    if (p->dir == LC_C2L) p->val_scratch = c.take<double>(size_t(p->batch) * size_t(g.n));
    const size_t wb = lc_values_work_bytes(g.n, p->batch);
    if (wb) p->val_work = c.take<char>(wb);
  }
  return c.off + 256;
}

// Slices per operand of the split tier when the options leave it to the
// library: 7 (about 56 bits per operand row) up to n = 1e5, where FP64-accurate
// output is held to a normwise relative error of 1e-13; 6 beyond, where the
// bound is 1e-12.
int auto_slices(int64_t n) { return n <= 100000 ? 7 : 6; }

// sin(pi a), exactly 0 at integers (the reflection formula below needs the zeros).
double sinpi_host(double a) {
  if (a == floor(a)) return 0.0;
  double r = a - 2.0 * floor(0.5 * a);  // [0, 2)
  if (r > 1.0) r -= 2.0;                // (-1, 1]
  if (r > 0.5) r = 1.0 - r;
  if (r < -0.5) r = -1.0 - r;
  return sin(M_PI * r);
}

// Coefficients of exp(sum_j e_j x^j), the series of Gamma(z+p)/Gamma(z+q)
// in x = 1/v^2 (lc_geg), with h = (p - q)/2 and
// e_j = -2 B_{2j+1}(1/2 + h) / (2j (2j+1)): the difference of the two Stirling
// series of log Gamma(v + 1/2 +- h), whose odd powers cancel.  The Bernoulli
// polynomials are expanded about 1/2: B_n(1/2 + h) = sum_k C(n,k) B_k(1/2) h^(n-k),
// B_k(1/2) = (2^(1-k) - 1) B_k (zero for odd k).
void geg_series(double h, double* pc) {
  static const double Bk[17] = {1.0, -0.5, 1.0 / 6, 0, -1.0 / 30, 0, 1.0 / 42, 0, -1.0 / 30, 0, 5.0 / 66, 0,
                                -691.0 / 2730, 0, 7.0 / 6, 0, -3617.0 / 510};
  double e[LC_GEG_TERMS + 1] = {0.0};
  for (int j = 1; j <= LC_GEG_TERMS; ++j) {
    const int n = 2 * j + 1;
    double b = 0.0, binom = 1.0;  // C(n, k)
    for (int k = 0; k <= n; ++k) {
      if (k > 0) binom = binom * double(n - k + 1) / double(k);
      if (k % 2 == 0 && k <= 16) b += binom * (ldexp(1.0, 1 - k) - 1.0) * Bk[k] * pow(h, double(n - k));
    }
    e[j] = -2.0 * b / (double(2 * j) * double(2 * j + 1));
  }
  pc[0] = 1.0;
  for (int n = 1; n <= LC_GEG_TERMS; ++n) {
    double acc = 0.0;
    for (int k = 1; k <= n; ++k) acc += double(k) * e[k] * pc[n - k];
    pc[n] = acc / double(n);
  }
}

// Validates lc_plan_options.alpha and fills p->geg (Legendre: on = 0).
lc_status geg_setup(lc_plan_s* p) {
  const double a = p->opt.alpha;
  memset(&p->geg, 0, sizeof(p->geg));
  p->geg.alpha = 0.5;
  p->geg.two_alpha = 1.0;
  if (a == 0.0 || a == 0.5) return LC_OK;
  if (!(a > -0.5 && a <= LC_GEGENBAUER_MAX_ALPHA)) return LC_ERR_INVALID_ARG;  // NaN fails too
  lc_geg& G = p->geg;
  G.on = 1;
  G.alpha = a;
  G.two_alpha = 2.0 * a;
  const double ga = tgamma(a);
  G.c_lam = sqrt(M_PI) / ga;
  // 1/Gamma(-a) = -a / Gamma(1-a) = -a Gamma(a) sin(pi a) / pi (reflection)
  G.c_u = 0.25 * ga * (-a * ga * sinpi_host(a) / M_PI);
  G.u0 = 0.25 * ga;
  G.v1 = 1.0 / (a * (a + 1.0) * ga);
  geg_series(0.5 * (a - 1.0), G.p_lam);
  geg_series(0.5 * (-a - 1.0), G.p_u);
  geg_series(0.5 * (-a - 1.0), G.p_v);
  return LC_OK;
}

bool valid_enum(lc_direction d, lc_dtype t) {
  return (d == LC_L2C || d == LC_C2L) &&
         (t == LC_F64 || t == LC_F64_SPLIT || t == LC_F32 || t == LC_F64_DF);
}

lc_status fill_plan(lc_plan_s* p, int64_t n, lc_direction dir, int64_t batch, lc_dtype dtype,
                    const lc_plan_options* opt) {
  if (!valid_enum(dir, dtype) || batch < 1 || batch > (int64_t(1) << 31)) return LC_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  lc_plan_options_default(&p->opt);
  if (opt) p->opt = *opt;
  if (p->opt.slices != 0 && (p->opt.slices < 3 || p->opt.slices > 7)) return LC_ERR_INVALID_ARG;
  lc_status st = lc_compute_geometry(n, &p->opt, 0, &p->g);
  if (st != LC_OK) return st;
  if (p->opt.slices == 0) p->opt.slices = auto_slices(n);
  if (p->opt.values != 0 && p->opt.values != 1) return LC_ERR_INVALID_ARG;
  if (p->opt.values && (!lc_values_supported(n) || dtype == LC_F32)) return LC_ERR_UNSUPPORTED;
  if (p->opt.nodal != 0 && p->opt.nodal != 1) return LC_ERR_INVALID_ARG;
  if (p->opt.nodal && dtype != LC_F64 && dtype != LC_F32) return LC_ERR_UNSUPPORTED;
  if (p->opt.fp64_plan != 0 && p->opt.fp64_plan != 1) return LC_ERR_INVALID_ARG;
  st = geg_setup(p);
  if (st != LC_OK) return st;
  p->dir = dir;
  p->dtype = dtype;
  p->batch = batch;
  p->count = batch;
  p->leaf_depth = 4;
  p->chunk_depth = 4;
  p->split_sched = 1;
  return LC_OK;
}

lc_status fill_ragged(lc_plan_s* p, const int64_t* n, int64_t count, lc_direction dir, lc_dtype dtype,
                      const lc_plan_options* opt) {
  if (!n || count < 1 || count > (int64_t(1) << 31)) return LC_ERR_INVALID_ARG;
  if (!valid_enum(dir, dtype)) return LC_ERR_INVALID_ARG;
  if (dtype != LC_F64_SPLIT) return LC_ERR_UNSUPPORTED;
  memset(p, 0, sizeof(*p));
  lc_plan_options_default(&p->opt);
  if (opt) p->opt = *opt;
  if (p->opt.fixed_s == 0) p->opt.fixed_s = 32;  // one s shared by every member
  if (p->opt.slices != 0 && (p->opt.slices < 3 || p->opt.slices > 7)) return LC_ERR_INVALID_ARG;
  if (p->opt.values) return LC_ERR_UNSUPPORTED;  // values at Chebyshev points: uniform plans only
  if (p->opt.nodal != 0 && p->opt.nodal != 1) return LC_ERR_INVALID_ARG;
  if (p->opt.nodal) return LC_ERR_UNSUPPORTED;  // the nodal variant: CUDA-core tiers
  if (geg_setup(p) != LC_OK) return LC_ERR_INVALID_ARG;
  int64_t nmax = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 1) return LC_ERR_INVALID_ARG;
    if (n[i] > nmax) nmax = n[i];
  }
  if (p->opt.slices == 0) p->opt.slices = auto_slices(nmax);
  lc_status st = lc_compute_geometry(nmax, &p->opt, 1, &p->g);
  if (st != LC_OK) return st;
  p->dir = dir;
  p->dtype = dtype;
  p->batch = count;
  p->count = count;
  p->ragged = 1;
  p->split_sched = 1;
  p->h_len = static_cast<int64_t*>(malloc(sizeof(int64_t) * size_t(count)));
  p->h_off = static_cast<int64_t*>(malloc(sizeof(int64_t) * size_t(count + 1)));
  if (!p->h_len || !p->h_off) return LC_ERR_HOST_ALLOC;
  p->h_off[0] = 0;
  for (int64_t i = 0; i < count; ++i) {
    p->h_len[i] = n[i];
    p->h_off[i + 1] = p->h_off[i] + n[i];
  }
  return LC_OK;
}

lc_status create_side(lc_plan_s* p) {
  p->side = p->fine = p->nearst = nullptr;
  p->ev_fork = p->ev_join = p->ev_start = p->ev_near = p->ev_done = nullptr;
  // Streams of one execution (see run() in lc_exec_kernels.cuh): the
  // latency-bound coarse-level chain at the highest priority, so that its few
  // CTAs are scheduled ahead of wide kernels; the far-field chain of the fine
  // levels next; the near-field band at the lowest, filling free SM slots.
  int lo_prio = 0, hi_prio = 0;
  LC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
  const int mid_prio = hi_prio + 1 <= lo_prio ? hi_prio + 1 : lo_prio;
  LC_CUDA_TRY(cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, hi_prio));
  LC_CUDA_TRY(cudaStreamCreateWithPriority(&p->fine, cudaStreamNonBlocking, mid_prio));
  LC_CUDA_TRY(cudaStreamCreateWithPriority(&p->nearst, cudaStreamNonBlocking, lo_prio));
  cudaEvent_t* evs[] = {&p->ev_fork, &p->ev_join, &p->ev_start, &p->ev_near, &p->ev_done};
  for (cudaEvent_t* e : evs) LC_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  return LC_OK;
}

void destroy_side(lc_plan_s* p) {
  cudaEvent_t* evs[] = {&p->ev_fork, &p->ev_join, &p->ev_start, &p->ev_near, &p->ev_done};
  for (cudaEvent_t* e : evs) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  cudaStream_t* sts[] = {&p->side, &p->fine, &p->nearst};
  for (cudaStream_t* q : sts) {
    if (*q) cudaStreamDestroy(*q);
    *q = nullptr;
  }
}

int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (int64_t(1) << 30)) b = int64_t(1) << 30;
  return int(b);
}

// The double-float tier builds its compact A-hat in double-float arithmetic
// (k_plan_ahat_df) unless the plan asks for the FP64 plan or needs what only
// the FP64 kernel has (Gegenbauer samples; leaf sizes below 10, whose finest
// samples need the argument shift).
bool df_plan(const lc_plan_s* p) {
  return p->dtype == LC_F64_DF && !p->opt.fp64_plan && !p->geg.on && !p->opt.nodal && p->g.s >= 10;
}

lc_status build_tables(lc_plan_s* p, cudaStream_t st) {
  const lc_geom& g = p->g;
  LC_CUDA_TRY(cudaMemsetAsync(p->err, 0, 64 * sizeof(int), st));
  if (df_plan(p)) {
    // The double-float tier's plan in two launches: Lambda^- (in double-float,
    // where the FP64 A-hat would be) with the DCT matrix, then the compact
    // A-hat built on the FP32 pipe, whose first CTAs build lambda (u, v),
    // T and B directly in double-float.
    p->df_tables_direct = 1;
    DfAux x;
    x.N = g.N;
    x.dir = int(p->dir);
    x.s = g.s;
    x.lam = static_cast<lc_df*>(p->df_lam);
    x.v2 = static_cast<lc_df*>(p->df_lam2);
    x.T = p->T;
    x.B = p->B;
    x.Tdf = static_cast<lc_df*>(p->df_T);
    x.Bdf = static_cast<lc_df*>(p->df_B);
    static_assert(2 * LC_MAX_S <= 128, "T rows by the first four warps of the last aux CTA");
    const int64_t aux = df_aux_ctas(g.N);
    if (g.L > 0) {
      double* cosm = p->Ahat + size_t(g.nc) * LC_M * LC_M;
      double* lminus = cosm + LC_M * LC_M;
      lc_df* lm_df = reinterpret_cast<lc_df*>(p->Ahat);
      k_plan_lminus<<<unsigned((int64_t(g.L) * 2 * LC_M * LC_M + 255) / 256), 256, 0, st>>>(
          g.L, g.s, int(p->dir), p->geg, cosm, lminus, lm_df);
      LC_LAUNCH_CHECK();
      p->df_ahat_direct = 1;
      const int64_t blocks = (g.nc < 1048576 ? g.nc : 1048576) + aux;
      k_plan_ahat_df<<<unsigned(blocks), LC_M * LC_M, 0, st>>>(g.L, g.s, int(p->dir), g.nc, cosm, lm_df,
                                                                static_cast<float*>(p->df_Ahat), x, aux);
    } else {
      k_plan_df_aux<<<unsigned(aux), LC_M * LC_M, 0, st>>>(x);
    }
    LC_LAUNCH_CHECK();
  } else {
    if (p->geg.on) {
      k_plan_geg_tables<<<grid_for((g.N + 7) / 8, 256), 256, 0, st>>>(g.N, int(p->dir), p->geg, p->lam, p->lam2);
      LC_LAUNCH_CHECK();
    } else {
      double* lam_target = (p->dir == LC_C2L) ? p->lam2 : p->lam;
      k_plan_lambda<<<grid_for((g.N + 7) / 8, 256), 256, 0, st>>>(g.N, lam_target);
      LC_LAUNCH_CHECK();
      if (p->dir == LC_C2L) {
        k_plan_c2l_tables<<<grid_for(g.N, 256), 256, 0, st>>>(g.N, p->lam, p->lam2);
        LC_LAUNCH_CHECK();
      }
    }
    if (p->opt.nodal) {
      k_plan_nodal_T<<<(2 * g.s * LC_M + 255) / 256, 256, 0, st>>>(g.s, p->T);
      LC_LAUNCH_CHECK();
      k_plan_nodal_P<<<(2 * LC_M * LC_M + 255) / 256, 256, 0, st>>>(p->B);
      LC_LAUNCH_CHECK();
    } else {
      static_assert(2 * LC_MAX_S <= 256, "one thread per row of T");
      k_plan_basis<<<2, 256, 0, st>>>(g.s, p->T, p->B);
      LC_LAUNCH_CHECK();
    }
    if (g.L > 0) {
      double* cosm = p->Ahat + size_t(g.nc) * LC_M * LC_M;
      double* lminus = cosm + LC_M * LC_M;
      k_plan_lminus<<<unsigned((int64_t(g.L) * 2 * LC_M * LC_M + 255) / 256), 256, 0, st>>>(
          g.L, g.s, int(p->dir), p->geg, cosm, lminus, nullptr);
      LC_LAUNCH_CHECK();
      const int64_t blocks = g.nc < 1048576 ? g.nc : 1048576;
      auto ahat = p->geg.on ? (p->opt.nodal ? k_plan_ahat<true, true> : k_plan_ahat<true, false>)
                            : (p->opt.nodal ? k_plan_ahat<false, true> : k_plan_ahat<false, false>);
      ahat<<<int(blocks), LC_M * LC_M, 0, st>>>(g.L, g.s, int(p->dir), g.nc, cosm, lminus, p->Ahat, p->geg);
      LC_LAUNCH_CHECK();
    }
  }
  if (p->dtype == LC_F32) {
    k_d2f<<<grid_for(g.N, 256), 256, 0, st>>>(g.N, p->lam, p->lamf);
    if (p->dir == LC_C2L) k_d2f<<<grid_for(g.N, 256), 256, 0, st>>>(g.N, p->lam2, p->lam2f);
    k_d2f<<<1, 256, 0, st>>>(int64_t(2) * g.s * LC_M, p->T, p->Tf);
    k_d2f<<<1, 256, 0, st>>>(2 * LC_M * LC_M, p->B, p->Bf);
    if (g.nc > 0)
      k_d2f_T<<<grid_for(g.nc * LC_M * LC_M, 256), 256, 0, st>>>(g.nc, p->Ahat, p->Ahatf);
    LC_LAUNCH_CHECK();
  } else if (p->dtype == LC_F64_DF) {
    LC_CUDA_TRY(cudaMemsetAsync(p->xexp_cnt, 0, size_t(p->batch) * sizeof(unsigned), st));
    lc_status s2 = lc_df_prepare(p, st);
    if (s2 != LC_OK) return s2;
  }
  if (p->opt.values) {
    lc_status s3 = lc_values_prepare(p, st);
    if (s3 != LC_OK) return s3;
  }
  return LC_OK;
}
}  // namespace

// ------------------------------------------------------------------ C ABI --
extern "C" {

lc_status lc_plan_options_default(lc_plan_options* opt) {
  if (!opt) return LC_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->s_hat = 32;
  opt->fixed_s = 0;
  opt->slices = 0;  // automatic (auto_slices)
  return LC_OK;
}

lc_status lc_plan_workspace_size_ex(int64_t n, lc_direction direction, int64_t batch, lc_dtype dtype,
                                    const lc_plan_options* opt, size_t* bytes) {
  if (!bytes) return LC_ERR_INVALID_ARG;
  lc_plan_s p;
  lc_status st = fill_plan(&p, n, direction, batch, dtype, opt);
  if (st != LC_OK) return st;
  *bytes = layout(&p, nullptr);
  return LC_OK;
}

lc_status lc_plan_workspace_size(int64_t n, lc_direction direction, int64_t batch, lc_dtype dtype,
                                 size_t* bytes) {
  return lc_plan_workspace_size_ex(n, direction, batch, dtype, nullptr, bytes);
}

lc_status lc_plan_create_ex(lc_plan* out, int64_t n, lc_direction direction, int64_t batch,
                            lc_dtype dtype, const lc_plan_options* opt, void* workspace, size_t bytes,
                            lc_stream stream) {
  if (!out || !workspace) return LC_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return LC_ERR_INVALID_ARG;
  *out = nullptr;
  lc_plan_s* p = static_cast<lc_plan_s*>(malloc(sizeof(lc_plan_s)));
  if (!p) return LC_ERR_HOST_ALLOC;
  lc_status st = fill_plan(p, n, direction, batch, dtype, opt);
  if (st != LC_OK) {
    free(p);
    return st;
  }
  const size_t need = layout(p, nullptr);
  if (bytes < need) {
    free(p);
    return LC_ERR_WORKSPACE_TOO_SMALL;
  }
  layout(p, static_cast<char*>(workspace));
  p->bytes_used = need;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  st = build_tables(p, s);  // enqueued first: the host creates the side streams while they run
  if (st == LC_OK) st = create_side(p);
  if (st == LC_OK && dtype == LC_F64_SPLIT) st = lc_split_prepare(p, static_cast<char*>(p->split), lc_split_bytes(p), s);
  if (st != LC_OK) {
    lc_split_release(p);
    destroy_side(p);
    free(p);
    return st;
  }
  lc_tune_apply_cached(p);
  *out = p;
  return LC_OK;
}

lc_status lc_plan_create(lc_plan* out, int64_t n, lc_direction direction, int64_t batch, lc_dtype dtype,
                         void* workspace, size_t bytes, lc_stream stream) {
  return lc_plan_create_ex(out, n, direction, batch, dtype, nullptr, workspace, bytes, stream);
}

lc_status lc_plan_set_timing(lc_plan plan, int32_t slots) {
  if (!plan || slots < 0 || slots > 100000) return LC_ERR_INVALID_ARG;
  if (plan->events) {
    for (int i = 0; i < plan->timing_slots * plan->timing_stride; ++i) cudaEventDestroy(plan->events[i]);
    free(plan->events);
    free(plan->kinds);
    free(plan->marks);
    plan->events = nullptr;
    plan->kinds = nullptr;
    plan->marks = nullptr;
  }
  plan->timing_slots = 0;
  if (slots == 0) return LC_OK;
  int32_t launches = 0;
  lc_plan_launches(plan, &launches);
  const int stride = launches + 2;
  plan->events = static_cast<cudaEvent_t*>(calloc(size_t(slots) * stride, sizeof(cudaEvent_t)));
  plan->kinds = static_cast<int32_t*>(calloc(size_t(slots) * stride, sizeof(int32_t)));
  plan->marks = static_cast<int*>(calloc(size_t(slots), sizeof(int)));
  if (!plan->events || !plan->kinds || !plan->marks) return LC_ERR_HOST_ALLOC;
  for (int i = 0; i < slots * stride; ++i) LC_CUDA_TRY(cudaEventCreate(&plan->events[i]));
  plan->timing_stride = stride;
  plan->timing_slots = slots;
  plan->exec_counter = 0;
  return LC_OK;
}

lc_status lc_plan_get_timing(lc_plan plan, int32_t slot, float* ms, int32_t* kinds, int32_t capacity,
                             int32_t* count) {
  if (!plan || !count || plan->timing_slots <= 0 || slot < 0 || slot >= plan->timing_slots) return LC_ERR_INVALID_ARG;
  const int m = plan->marks[slot];
  const int n = m > 0 ? m - 1 : 0;
  *count = n;
  if (n == 0) return LC_OK;
  cudaEvent_t* ev = plan->events + size_t(slot) * plan->timing_stride;
  LC_CUDA_TRY(cudaEventSynchronize(ev[n]));
  for (int i = 0; i < n && i < capacity; ++i) {
    if (ms) LC_CUDA_TRY(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
    if (kinds) kinds[i] = plan->kinds[size_t(slot) * plan->timing_stride + i];
  }
  return LC_OK;
}

lc_status lc_destroy(lc_plan plan) {
  if (!plan) return LC_ERR_INVALID_ARG;
  lc_plan_set_timing(plan, 0);
  lc_split_release(plan);
  destroy_side(plan);
  free(plan->h_len);
  free(plan->h_off);
  free(plan);
  return LC_OK;
}

const char* lc_status_string(lc_status status) {
  switch (status) {
    case LC_OK: return "LC_OK";
    case LC_ERR_INVALID_ARG: return "LC_ERR_INVALID_ARG: invalid size, enum, pointer or stride";
    case LC_ERR_WORKSPACE_TOO_SMALL: return "LC_ERR_WORKSPACE_TOO_SMALL: workspace below the required size";
    case LC_ERR_CUDA: return "LC_ERR_CUDA: a CUDA runtime call or kernel launch failed";
    case LC_ERR_DEVICE_TIMEOUT: return "LC_ERR_DEVICE_TIMEOUT: a bounded device wait gave up";
    case LC_ERR_UNSUPPORTED: return "LC_ERR_UNSUPPORTED: request not implemented";
    case LC_ERR_HOST_ALLOC: return "LC_ERR_HOST_ALLOC: host allocation failed";
  }
  return "unknown lc_status";
}

lc_status lc_plan_workspace_size_ragged(const int64_t* n, int64_t count, lc_direction direction, lc_dtype dtype,
                                        const lc_plan_options* opt, size_t* bytes) {
  if (!bytes) return LC_ERR_INVALID_ARG;
  lc_plan_s p;
  lc_status st = fill_ragged(&p, n, count, direction, dtype, opt);
  if (st == LC_OK) *bytes = layout(&p, nullptr);
  free(p.h_len);
  free(p.h_off);
  return st;
}

lc_status lc_plan_create_ragged(lc_plan* out, const int64_t* n, int64_t count, lc_direction direction,
                                lc_dtype dtype, const lc_plan_options* opt, void* workspace, size_t bytes,
                                lc_stream stream) {
  if (!out || !workspace) return LC_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return LC_ERR_INVALID_ARG;
  *out = nullptr;
  lc_plan_s* p = static_cast<lc_plan_s*>(malloc(sizeof(lc_plan_s)));
  if (!p) return LC_ERR_HOST_ALLOC;
  lc_status st = fill_ragged(p, n, count, direction, dtype, opt);
  if (st == LC_OK) {
    const size_t need = layout(p, nullptr);
    if (bytes < need) st = LC_ERR_WORKSPACE_TOO_SMALL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (st == LC_OK) {
    p->bytes_used = layout(p, static_cast<char*>(workspace));
    st = create_side(p);
  }
  if (st == LC_OK) st = build_tables(p, s);
  if (st == LC_OK) st = lc_split_prepare(p, static_cast<char*>(p->split), lc_split_bytes(p), s);
  if (st != LC_OK) {
    lc_split_release(p);
    destroy_side(p);
    free(p->h_len);
    free(p->h_off);
    free(p);
    return st;
  }
  *out = p;
  return LC_OK;
}

lc_status lc_plan_check(lc_plan plan, lc_stream stream) {
  if (!plan) return LC_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int h = 0;
  LC_CUDA_TRY(cudaMemcpyAsync(&h, plan->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  LC_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    LC_CUDA_TRY(cudaMemsetAsync(plan->err, 0, sizeof(int), s));
    LC_CUDA_TRY(cudaStreamSynchronize(s));
    return LC_ERR_DEVICE_TIMEOUT;
  }
  return LC_OK;
}

lc_status lc_plan_info(lc_plan plan, int64_t* n, int64_t* N, int32_t* L, int32_t* s, int32_t* M,
                       int64_t* n_c, int64_t* batch) {
  if (!plan) return LC_ERR_INVALID_ARG;
  if (n) *n = plan->g.n;
  if (N) *N = plan->g.N;
  if (L) *L = plan->g.L;
  if (s) *s = plan->g.s;
  if (M) *M = LC_M;
  if (n_c) *n_c = plan->g.nc;
  if (batch) *batch = plan->batch;
  return LC_OK;
}

lc_status lc_plan_table(lc_plan plan, int32_t which, double* dst, int64_t count, int64_t* copied,
                        lc_stream stream) {
  if (!plan || !dst || count < 0) return LC_ERR_INVALID_ARG;
  const double* src = nullptr;
  int64_t len = 0;
  switch (which) {
    case 0: src = (plan->dir == LC_C2L || plan->df_tables_direct) ? nullptr : plan->lam; len = plan->g.N; break;
    case 1: src = plan->T; len = int64_t(2) * plan->g.s * LC_M; break;
    case 2: src = plan->B; len = (plan->opt.nodal ? 2 : 1) * LC_M * LC_M; break;
    case 3:  // not built when the double-float tier makes its compact copy directly
      src = df_plan(plan) ? nullptr : plan->Ahat;
      len = plan->g.nc * LC_M * LC_M;
      break;
    case 4: src = plan->df_tables_direct ? nullptr : plan->lam; len = plan->g.N; break;   // C2L: u table
    case 5: src = plan->df_tables_direct ? nullptr : plan->lam2; len = plan->g.N; break;  // C2L: v table
    case 6:  // raw FP32 words of the compact double-float A-hat, two per double
      if (plan->dtype != LC_F64_DF) return LC_ERR_UNSUPPORTED;
      src = static_cast<const double*>(plan->df_Ahat);
      len = plan->g.nc * lc_dfa_words(plan->dir) / 2;
      break;
    default: return LC_ERR_INVALID_ARG;
  }
  if (!src) return LC_ERR_UNSUPPORTED;
  if (len > count) len = count;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (len > 0) LC_CUDA_TRY(cudaMemcpyAsync(dst, src, size_t(len) * sizeof(double), cudaMemcpyDeviceToHost, s));
  LC_CUDA_TRY(cudaStreamSynchronize(s));
  if (copied) *copied = len;
  return LC_OK;
}

lc_status lc_plan_launches(lc_plan plan, int32_t* launches) {
  if (!plan || !launches) return LC_ERR_INVALID_ARG;
  *launches = (plan->dtype == LC_F64_SPLIT) ? lc_exec_split_launches(plan) : lc_exec_cuda_cores_launches(plan);
  if (plan->opt.values) *launches += lc_values_launches(plan);  // the cosine transform
  return LC_OK;
}

static lc_status transform(lc_plan plan, const void* in, void* out, const lc_layout& lay, cudaStream_t s,
                           int adjoint) {
  switch (plan->dtype) {
    case LC_F64:
    case LC_F32: return lc_exec_cuda_cores(plan, in, out, lay, s, adjoint);
    case LC_F64_DF: return lc_exec_df(plan, in, out, lay, s, adjoint);
    case LC_F64_SPLIT: return lc_exec_split(plan, in, out, lay, s, adjoint);
  }
  return LC_ERR_INVALID_ARG;
}

static lc_status dispatch(lc_plan plan, const void* in, void* out, lc_layout lay, lc_stream stream, int adjoint) {
  if (!plan || !in || !out) return LC_ERR_INVALID_ARG;
  if (lay.ib < 0 || lay.ie < 0 || lay.ob < 0 || lay.oe < 0 || lay.iob < 0 || lay.oob < 0) return LC_ERR_INVALID_ARG;
  if (lay.inner < 1 || lay.inner > plan->batch) return LC_ERR_INVALID_ARG;
  if (lay.inner == plan->batch) lay.inner = 0;  // one batch stride
  if (plan->ragged) {
    if (lay.ib != 0 || lay.ob != 0 || lay.ie != 1 || lay.oe != 1 || lay.inner != 0) return LC_ERR_INVALID_ARG;
  } else {
    // no two outputs on one address: within a vector, within an inner group, across groups
    if (lay.oe == 0 && plan->g.n > 1) return LC_ERR_INVALID_ARG;
    if (lay.inner == 0 && lay.ob == 0 && plan->batch > 1) return LC_ERR_INVALID_ARG;
    if (lay.inner > 1 && lay.ob == 0) return LC_ERR_INVALID_ARG;
    if (lay.inner > 0 && lay.oob == 0) return LC_ERR_INVALID_ARG;
  }
  if (in == out) return LC_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (plan->opt.values) {
    // values at Chebyshev points: L2C, then the cosine transform of its
    // result in place; or the inverse cosine transform into the plan's
    // buffer, then C2L from there
    if (adjoint) return LC_ERR_UNSUPPORTED;
    if (plan->dir == LC_L2C) {
      lc_status e = transform(plan, in, out, lay, s, 0);
      if (e != LC_OK) return e;
      return lc_values_synth(plan, static_cast<double*>(out), lay, s);
    }
    lc_status e = lc_values_analysis(plan, static_cast<const double*>(in), lay, plan->val_scratch, s);
    if (e != LC_OK) return e;
    lc_layout packed = lay;
    packed.ib = plan->g.n;
    packed.ie = 1;
    packed.iob = 0;
    if (packed.inner > 0) packed.iob = packed.inner * plan->g.n;  // vector b at b n either way
    return transform(plan, plan->val_scratch, out, packed, s, 0);
  }
  return transform(plan, in, out, lay, s, adjoint);
}

lc_status lc_execute(lc_plan plan, const void* in, void* out, int64_t in_batch_stride, int64_t in_elem_stride,
                     int64_t out_batch_stride, int64_t out_elem_stride, lc_stream stream) {
  if (!plan) return LC_ERR_INVALID_ARG;
  const lc_layout lay{in_batch_stride, in_elem_stride, out_batch_stride, out_elem_stride, plan->batch, 0, 0};
  return dispatch(plan, in, out, lay, stream, 0);
}

lc_status lc_adjoint(lc_plan plan, const void* in, void* out, int64_t in_batch_stride, int64_t in_elem_stride,
                     int64_t out_batch_stride, int64_t out_elem_stride, lc_stream stream) {
  if (!plan) return LC_ERR_INVALID_ARG;
  const lc_layout lay{in_batch_stride, in_elem_stride, out_batch_stride, out_elem_stride, plan->batch, 0, 0};
  return dispatch(plan, in, out, lay, stream, 1);
}

lc_status lc_execute_ex(lc_plan plan, const void* in, void* out, int64_t in_batch_stride, int64_t in_elem_stride,
                        int64_t out_batch_stride, int64_t out_elem_stride, int64_t batch_inner,
                        int64_t in_outer_stride, int64_t out_outer_stride, lc_stream stream) {
  const lc_layout lay{in_batch_stride, in_elem_stride, out_batch_stride, out_elem_stride, batch_inner,
                      in_outer_stride, out_outer_stride};
  return dispatch(plan, in, out, lay, stream, 0);
}

lc_status lc_adjoint_ex(lc_plan plan, const void* in, void* out, int64_t in_batch_stride, int64_t in_elem_stride,
                        int64_t out_batch_stride, int64_t out_elem_stride, int64_t batch_inner,
                        int64_t in_outer_stride, int64_t out_outer_stride, lc_stream stream) {
  const lc_layout lay{in_batch_stride, in_elem_stride, out_batch_stride, out_elem_stride, batch_inner,
                      in_outer_stride, out_outer_stride};
  return dispatch(plan, in, out, lay, stream, 1);
}

}  // extern "C"
