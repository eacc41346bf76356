/*
 * lc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, direct O(n^2) CPU implementation of the Legendre<->Chebyshev
 * connection maps of Mortensen, "A faster multipole Legendre-Chebyshev
 * transform" (arXiv:2411.00033).  It is the oracle that the GPU library is
 * checked against.  It shares no code with the GPU library and may only be
 * used by the tests, by the smoke check and by the CPU-baseline leg of the
 * benchmark; nothing on the product path calls it.
 *
 * What it computes (the plain definitions, no blocking or approximation):
 *   L2C:          z = C^{-1} A f             (Sec. 1, eq:directmv)
 *   C2L:          z = (A^{-1} C) f           (Sec. 1, eq:directmv), with the
 *                 entries of A^{-1} C taken from the closed form L(x,y) of
 *                 Sec. 3.3 (eq:Lxymod) and entry (0,0) = 1.
 *   L2C adjoint:  g = A^T C^{-1} r
 *   C2L adjoint:  g = (A^{-1} C)^T r
 * where a_ij = Lambda((j-i)/2) Lambda((j+i)/2) for j >= i, j-i even
 * (eq:aij / eq:hik), Lambda(x) = Gamma(x+1/2)/Gamma(x+1) (eq:Lambda), and
 * C = diag(c_i pi/2), c_0 = 2, c_i = 1 (Sec. 1).
 *
 * Precision: every entry and every sum is carried in double-double
 * (error-free TwoSum / TwoProd with fma) and rounded once to double at the
 * end, so each output is within about one ulp of the exact value.  The
 * lambda table is built by the integer recursion Lambda(0) = sqrt(pi),
 * Lambda(k) = Lambda(k-1) (k - 1/2)/k (eq:Lambdaint) in double-double; this
 * is deliberately a different route from the tau series that the GPU plan
 * uses (eq:tau).
 *
 * Values at Chebyshev points (lco_dct): the Chebyshev series with
 * coefficients c evaluated at the n Chebyshev-Gauss points
 * x_m = cos((m + 1/2) pi / n), v_m = sum_k c_k T_k(x_m) =
 * sum_k c_k cos(pi k (2m + 1) / (2n)) (kind 0), and its inverse by discrete
 * orthogonality, c_k = (2 / n) / (1 + [k = 0]) sum_m v_m cos(pi k (2m+1)/(2n))
 * (kind 1), exact for degree < n.  Direct O(n^2) sums in double-double; each
 * cosine's argument is reduced exactly in integers first (k (2m+1) mod 4n),
 * so every cosine is within about one ulp.  With lco_apply these give the
 * Legendre synthesis on Chebyshev points (L2C, then kind 0; Sec. 1 names the
 * Chebyshev-Legendre Galerkin use) and its inverse (kind 1, then C2L).
 *
 * Gegenbauer bases (lco_apply_geg, lco_entry_geg).  The Conclusions note that
 * the method carries over to transforms between Gegenbauer bases.  The maps
 * here connect the Gegenbauer polynomials C_j^(a), a > -1/2, a != 0, with the
 * Chebyshev polynomials; a = 1/2 gives the Legendre maps above.  Their plain
 * definitions, written out without any Gamma function:
 *   Gegenbauer -> Chebyshev.  The generating function
 *   (1 - 2xt + t^2)^(-a) = (1 - e^{it} t)^(-a) (1 - e^{-it} t)^(-a) at x = cos t,
 *   expanded as a product of two binomial series, gives
 *   C_j^(a)(cos t) = sum_k g_k g_{j-k} cos((j - 2k) t), g_k = (a)_k / k!,
 *   so entry (i, j), j - i = 2l >= 0, is (2/c_i) g_l g_m with m = (i + j)/2.
 *   Chebyshev -> Gegenbauer.  The connection C^(mu) -> C^(a) (DLMF 18.18.16)
 *   in the limit T_j = (j/2) lim_{mu->0} C_j^(mu)/mu gives, for j >= 1,
 *   entry (i, j) = (2i + 2a) j K u_l w_m with K = 1/(4a(a+1)),
 *   u_l = (-a)_l / l!, w_m = (m-1)! / (a+2)_{m-1}; entry (0,0) = 1.
 * The three sequences come from their ratio recursions in double-double.
 *
 * Rows are independent; with OpenMP available they are spread over threads.
 */
#define _GNU_SOURCE 1
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  dd r = {s, e};
  return r;
}
static inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  dd r = {s, b - (s - a)};
  return r;
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  dd r = {p, fma(a, b, -p)};
  return r;
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_div(dd a, dd b) {
  /* long division: q1 = a/b, r = a - q1 b, q2 = r/b, ... */
  double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_mul_d(b, -q1));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_mul_d(b, -q2));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, (dd){q3, 0.0});
}
static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }
static inline double dd_to(dd a) { return a.hi + a.lo; }

/* sqrt(pi) = Gamma(1/2) = Lambda(0) (eq:Lambdaint) and pi, as double-doubles:
 * hi = RN(x), lo = RN(x - hi), from a 50-digit evaluation. */
static const dd SQRT_PI_DD = {1.772453850905516, -7.666586499825799e-17};
static const dd PI_DD = {3.141592653589793, 1.2246467991473532e-16};

/* Lambda(k) for k < n as double-double (eq:Lambdaint recursion). */
static void lambda_table(int64_t n, dd* lam) {
  if (n <= 0) return;
  lam[0] = SQRT_PI_DD;
  for (int64_t k = 1; k < n; ++k) {
    /* (k - 1/2)/k = (2k - 1)/(2k): both exact doubles for k < 2^51. */
    dd num = dd_mul_d(lam[k - 1], (double)(2 * k - 1));
    lam[k] = dd_div(num, dd_from((double)(2 * k)));
  }
}

/* Entry (i, j) of C^{-1} A in double-double, 0 <= i, j < n (no bounds check
 * beyond j >= i and j - i even). */
static dd l2c_entry(const dd* lam, int64_t i, int64_t j) {
  if (j < i || ((j - i) & 1)) return dd_from(0.0);
  int64_t k = (j - i) / 2;
  dd a = dd_mul(lam[k], lam[i + k]);            /* a_ij, eq:hik */
  /* C^{-1}: 1/pi for row 0, 2/pi otherwise */
  dd cinv = dd_div(dd_from(i == 0 ? 1.0 : 2.0), PI_DD);
  return dd_mul(a, cinv);
}

/* Entry (i, j) of A^{-1} C from L(x, y) (eq:Lxymod):
 *   L(x,y) = 2(x+1/2) y / ((x+y)(x+y+1)(x-y+1)) * Lambda((y-x)/2)/Lambda((x+y)/2)
 * with x = i, y = j = i + 2k, and the (0,0) entry equal to 1. */
static dd c2l_entry(const dd* lam, int64_t i, int64_t j) {
  if (j < i || ((j - i) & 1)) return dd_from(0.0);
  if (i == 0 && j == 0) return dd_from(1.0);
  int64_t k = (j - i) / 2;
  dd num = dd_mul(dd_from((double)(2 * i + 1)), dd_from((double)j));   /* 2(x+1/2) y */
  dd den = dd_mul(dd_from((double)(i + j)), dd_from((double)(i + j + 1)));
  den = dd_mul(den, dd_from((double)(i - j + 1)));                      /* (x+y)(x+y+1)(x-y+1) */
  dd ratio = dd_div(lam[k], lam[i + k]);                                 /* Lambda((y-x)/2)/Lambda((x+y)/2) */
  return dd_mul(dd_div(num, den), ratio);
}

static dd entry(int direction, const dd* lam, int64_t i, int64_t j) {
  return direction == 0 ? l2c_entry(lam, i, j) : c2l_entry(lam, i, j);
}

/* Gegenbauer parameter a: the double-double sequences of the header,
 * t0[k] = g_k = (a)_k/k! (direction 0), or t0[l] = u_l = (-a)_l/l! and
 * t1[m] = w_m = (m-1)!/(a+2)_{m-1}, t1[0] = 0 (direction 1), for indices < n. */
static void geg_tables(int direction, double a, int64_t n, dd* t0, dd* t1) {
  if (n <= 0) return;
  t0[0] = dd_from(1.0);
  for (int64_t k = 1; k < n; ++k) {
    /* g_k = g_{k-1} (k - 1 + a)/k, u_k = u_{k-1} (k - 1 - a)/k: the sums are
     * exact as double-doubles */
    dd f = two_sum((double)(k - 1), direction == 0 ? a : -a);
    t0[k] = dd_div(dd_mul(t0[k - 1], f), dd_from((double)k));
  }
  if (direction == 0) return;
  t1[0] = dd_from(0.0);
  if (n > 1) t1[1] = dd_from(1.0);
  for (int64_t m = 2; m < n; ++m)
    t1[m] = dd_div(dd_mul_d(t1[m - 1], (double)(m - 1)), two_sum((double)m, a));
}

static dd geg_entry(int direction, double a, const dd* t0, const dd* t1, int64_t i, int64_t j) {
  if (j < i || ((j - i) & 1)) return dd_from(0.0);
  const int64_t l = (j - i) / 2, m = (i + j) / 2;
  if (direction == 0) {
    dd e = dd_mul(t0[l], t0[m]);
    return i == 0 ? e : dd_mul_d(e, 2.0);
  }
  if (i == 0 && j == 0) return dd_from(1.0);
  /* K = 1 / (4 a (a + 1)) */
  dd den = dd_mul(dd_from(4.0 * a), two_sum(a, 1.0));
  dd e = dd_div(dd_mul(t0[l], t1[m]), den);
  e = dd_mul(e, two_sum((double)(2 * i), 2.0 * a));
  return dd_mul_d(e, (double)j);
}

/* ---------------------------------------------------------------- API -- */

/* Lambda(k), k < n, rounded to double (hi) plus the double-double tail. */
int lco_lambda(int64_t n, double* hi, double* lo) {
  if (n < 0 || !hi) return 1;
  dd* lam = (dd*)malloc(sizeof(dd) * (size_t)(n > 0 ? n : 1));
  if (!lam) return 2;
  lambda_table(n, lam);
  for (int64_t k = 0; k < n; ++k) {
    dd v = quick_two_sum(lam[k].hi, lam[k].lo);
    hi[k] = v.hi;
    if (lo) lo[k] = v.lo;
  }
  free(lam);
  return 0;
}

/* One matrix entry of the map (direction 0 = L2C matrix C^{-1}A,
 * 1 = C2L matrix A^{-1}C), rounded to double. */
int lco_entry(int direction, int64_t n, int64_t i, int64_t j, double* out) {
  if (n <= 0 || i < 0 || j < 0 || i >= n || j >= n || !out) return 1;
  dd* lam = (dd*)malloc(sizeof(dd) * (size_t)n);
  if (!lam) return 2;
  lambda_table(n, lam);
  *out = dd_to(entry(direction, lam, i, j));
  free(lam);
  return 0;
}

/* Apply the map (or its transpose when adjoint != 0) to x[0:n].
 * rows == NULL: compute all n outputs into out[0:n].
 * rows != NULL: compute outputs rows[0:nrows] into out[0:nrows].
 * Returns 0 on success. */
int lco_apply(int direction, int adjoint, int64_t n, const double* x,
              int64_t nrows, const int64_t* rows, double* out) {
  if (n <= 0 || !x || !out || (direction != 0 && direction != 1)) return 1;
  int64_t count = rows ? nrows : n;
  for (int64_t r = 0; rows && r < count; ++r)
    if (rows[r] < 0 || rows[r] >= n) return 1;
  dd* lam = (dd*)malloc(sizeof(dd) * (size_t)n);
  if (!lam) return 2;
  lambda_table(n, lam);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < count; ++r) {
    int64_t i = rows ? rows[r] : r;
    dd acc = dd_from(0.0);
    if (!adjoint) {
      /* z_i = sum_{j >= i, j - i even} M_ij x_j */
      for (int64_t j = i; j < n; j += 2)
        acc = dd_add(acc, dd_mul_d(entry(direction, lam, i, j), x[j]));
    } else {
      /* g_j = sum_{i <= j, j - i even} M_ij r_i, with j the output index */
      int64_t j = i;
      for (int64_t ii = (j & 1); ii <= j; ii += 2)
        acc = dd_add(acc, dd_mul_d(entry(direction, lam, ii, j), x[ii]));
    }
    out[r] = dd_to(acc);
  }
  free(lam);
  return 0;
}

/* The Gegenbauer maps of the header (direction 0: Gegenbauer -> Chebyshev,
 * 1: Chebyshev -> Gegenbauer), or their transposes, for parameter a with
 * -1/2 < a, a != 0; arguments as lco_apply. */
int lco_apply_geg(int direction, int adjoint, double a, int64_t n, const double* x,
                  int64_t nrows, const int64_t* rows, double* out) {
  if (n <= 0 || !x || !out || (direction != 0 && direction != 1)) return 1;
  if (!(a > -0.5) || a == 0.0 || !isfinite(a)) return 1;
  int64_t count = rows ? nrows : n;
  for (int64_t r = 0; rows && r < count; ++r)
    if (rows[r] < 0 || rows[r] >= n) return 1;
  dd* t0 = (dd*)malloc(sizeof(dd) * (size_t)n);
  dd* t1 = (dd*)malloc(sizeof(dd) * (size_t)n);
  if (!t0 || !t1) {
    free(t0);
    free(t1);
    return 2;
  }
  geg_tables(direction, a, n, t0, t1);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < count; ++r) {
    int64_t i = rows ? rows[r] : r;
    dd acc = dd_from(0.0);
    if (!adjoint) {
      for (int64_t j = i; j < n; j += 2)
        acc = dd_add(acc, dd_mul_d(geg_entry(direction, a, t0, t1, i, j), x[j]));
    } else {
      int64_t j = i;
      for (int64_t ii = (j & 1); ii <= j; ii += 2)
        acc = dd_add(acc, dd_mul_d(geg_entry(direction, a, t0, t1, ii, j), x[ii]));
    }
    out[r] = dd_to(acc);
  }
  free(t0);
  free(t1);
  return 0;
}

/* The sequences of geg_tables rounded to double: t0 = g (direction 0) or u
 * (direction 1), t1 = w (direction 1; may be NULL for direction 0). */
int lco_geg_tables(int direction, double a, int64_t n, double* t0, double* t1) {
  if (n <= 0 || !t0 || (direction != 0 && direction != 1) || (direction == 1 && !t1)) return 1;
  if (!(a > -0.5) || a == 0.0 || !isfinite(a)) return 1;
  dd* d0 = (dd*)malloc(sizeof(dd) * (size_t)n);
  dd* d1 = (dd*)malloc(sizeof(dd) * (size_t)n);
  if (!d0 || !d1) {
    free(d0);
    free(d1);
    return 2;
  }
  geg_tables(direction, a, n, d0, d1);
  for (int64_t k = 0; k < n; ++k) {
    t0[k] = dd_to(d0[k]);
    if (direction == 1) t1[k] = dd_to(d1[k]);
  }
  free(d0);
  free(d1);
  return 0;
}

/* One entry of a Gegenbauer map, rounded to double. */
int lco_entry_geg(int direction, double a, int64_t n, int64_t i, int64_t j, double* out) {
  if (n <= 0 || i < 0 || j < 0 || i >= n || j >= n || !out) return 1;
  if (direction != 0 && direction != 1) return 1;
  if (!(a > -0.5) || a == 0.0 || !isfinite(a)) return 1;
  dd* t0 = (dd*)malloc(sizeof(dd) * (size_t)n);
  dd* t1 = (dd*)malloc(sizeof(dd) * (size_t)n);
  if (!t0 || !t1) {
    free(t0);
    free(t1);
    return 2;
  }
  geg_tables(direction, a, n, t0, t1);
  *out = dd_to(geg_entry(direction, a, t0, t1, i, j));
  free(t0);
  free(t1);
  return 0;
}

/* Number of threads the OpenMP runtime would use (1 without OpenMP). */
/* cos(pi r / d) for integers 0 <= r < 2d, d >= 1: reduced to an angle in
 * [0, pi/4] by the symmetries of cos, then one libm call. */
static double cospi_ratio(int64_t r, int64_t d) {
  double sign = 1.0;
  if (r > d) r = 2 * d - r;            /* cos(2 pi - t) = cos t */
  if (2 * r > d) {                     /* cos(pi - t) = -cos t */
    r = d - r;
    sign = -1.0;
  }
  if (4 * r <= d) return sign * cos(M_PI * (double)r / (double)d);
  return sign * sin(M_PI * (double)(d - 2 * r) / (2.0 * (double)d)); /* cos t = sin(pi/2 - t) */
}

/* kind 0: y_m = sum_k x_k cos(pi k (2m+1) / (2n)); kind 1: y_k =
 * (2/n)/(1 + [k = 0]) sum_m x_m cos(pi k (2m+1) / (2n)).  rows == NULL: all
 * n outputs; otherwise outputs rows[0:nrows] into y[0:nrows]. */
int lco_dct_rows(int kind, int64_t n, const double* x, int64_t nrows, const int64_t* rows, double* y) {
  if (n < 1 || !x || !y || (kind != 0 && kind != 1)) return 1;
  const int64_t count = rows ? nrows : n;
  for (int64_t r = 0; rows && r < count; ++r)
    if (rows[r] < 0 || rows[r] >= n) return 1;
  const int64_t d = 2 * n; /* angle pi q / d with q = k (2m+1) mod 2d */
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < count; ++r) {
    const int64_t o = rows ? rows[r] : r;
    dd acc = dd_from(0.0);
    for (int64_t t = 0; t < n; ++t) {
      const int64_t k = kind == 0 ? t : o, m = kind == 0 ? o : t;
      const int64_t q = (k % (2 * d)) * ((2 * m + 1) % (2 * d)) % (2 * d);
      acc = dd_add(acc, two_prod(x[t], cospi_ratio(q, d)));
    }
    if (kind == 1) acc = dd_mul_d(acc, (o == 0 ? 1.0 : 2.0) / (double)n);
    y[r] = dd_to(acc);
  }
  return 0;
}

int lco_dct(int kind, int64_t n, const double* x, double* y) { return lco_dct_rows(kind, n, x, 0, NULL, y); }

int lco_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
