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
// Launch structure: the levels are cut into chunks and each CTA owns the
// subtree of one node of a chunk's top level, so consecutive levels never
// need a grid-wide barrier inside a chunk:
//   up chunks (bottom to top): the first one restricts the input over
//     2^5 leaf segments and climbs 5 levels; each later one climbs up to 4
//     more levels from the previous chunk's top level;
//   down chunks (top to bottom): each adds, level by level, the parent's
//     contribution of Step 4 to the coupling result of Step 3; the last chunk
//     ends at the leaves and also does the spread, the near-field band with
//     its operands staged in shared memory, and the scaling.
// After the first up chunk, the coarse levels' up chunks, their coupling and
// their down chunks run on a high-priority side stream, concurrently with the
// coupling of the fine levels on the caller's stream; the last down chunk
// waits for both.  For L = 13 (n = 1e6): 8 launches instead of 2L+1 = 27,
// with the coarse chain hidden behind the fine coupling.
//
// The transposed pass (lc_adjoint) runs the same kernels with the roles of
// the trees exchanged: restriction over row segments and the row tree
// upwards, A-hat transposed in the coupling, the column tree downwards,
// spread over column segments and the transposed band.
#pragma once
#include "lc_internal.cuh"
#include "lc_tma.cuh"

namespace lc_exec {

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

// Dot-product accumulation.  Generic: fused multiply-add in R.  The
// double-float tier specialises these to keep an unnormalised error word and
// normalise once at the end (see lc_df.cu).
template <typename R>
__device__ __forceinline__ R acc2(const R& acc, const R& a, const R& b) { return fma(a, b, acc); }
template <typename R>
__device__ __forceinline__ R acc3(const R& acc, const R& a, const R& b, const R& c) { return fma(a * b, c, acc); }
template <typename R>
__device__ __forceinline__ R finish(const R& acc) { return acc; }
// Whether splitting a short sum into two independent chains pays off: it
// does for the hardware types (latency of dependent FMAs), not for the
// double-float type, whose extra normalisations cost more than they hide.
template <typename R>
struct split_chains { static constexpr bool value = true; };
// A-hat(m)[k][l]: the FP64 table keeps row-major [k][l]; the FP32 and
// double-float copies are stored transposed, [l][k], so that threads that
// own consecutive k read consecutive addresses.
template <typename R>
__device__ __forceinline__ const R& ahat_at(const R* Ah, int64_t m, int k, int l) {
  return Ah[m * (LC_M * LC_M) + l * LC_M + k];
}
template <>
__device__ __forceinline__ const double& ahat_at<double>(const double* Ah, int64_t m, int k, int l) {
  return Ah[m * (LC_M * LC_M) + k * LC_M + l];
}

constexpr int kThreads = 256;
// Chunk geometry (per plan, chosen by lc_plan_autotune; defaults 4 and 4):
// leaf depth = levels climbed by the first up chunk / descended by the last
// down chunk, chunk depth = levels per coarse chunk.
constexpr int kSeg = 2 * LC_M;  // values per segment: [sigma][k]

// Node x at level gamma of the column tree (segments g >= 2) or of the row
// tree (segments v < 2 b_gamma).
__device__ __forceinline__ bool node_valid(bool col, int gamma, int64_t x) {
  const int64_t n = int64_t(4) << gamma;
  return col ? (x >= 2 && x < n) : (x >= 0 && x < n - 2);
}

// Offsets (in R elements) of level d inside a subtree buffer.
__device__ __forceinline__ int sub_off(int d) { return ((1 << d) - 1) * kSeg; }

// ---------------------------------------------------------------- up chunk
// Root x0 = blockIdx.x at level rho; bottom level rho + depth.  leaf != 0:
// the bottom level is the leaf level, computed from the input (Step 1).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_up_chunk(Args<R> a, int rho, int depth, int leaf, int adj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* nodes = reinterpret_cast<R*>(smem_raw);                 // (2^(depth+1) - 1) segments
  R* zt = nodes + sub_off(depth + 1);                         // 2 x 2^(depth-1) segments
  R* Ts = zt + 2 * (1 << (depth > 0 ? depth - 1 : 0)) * kSeg;  // [2][s][M]
  R* fs = Ts + 2 * a.s * LC_M;                                // [2^depth][2s]
  __shared__ R Bt[LC_M * LC_M];  // B(0) transposed: Bt[j][k] = b_kj
  const bool col = !adj;
  const int s = a.s;
  const int64_t x0 = blockIdx.x;
  const int gb = rho + depth;
  const int nb = 1 << depth;
  for (int i = threadIdx.x; i < LC_M * LC_M; i += blockDim.x) Bt[(i % LC_M) * LC_M + i / LC_M] = a.t.B[i];
  if (leaf)
    for (int i = threadIdx.x; i < 2 * s * LC_M; i += blockDim.x) Ts[i] = a.t.T[i];
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    R* Wb = a.t.W + b * a.nseg * kSeg;
    __syncthreads();
    if (leaf) {
      const int64_t p0 = (x0 << depth) * 2 * s;
      const typename lc_io<R>::type* f = a.in + b * a.ib;
      const bool scale = adj && a.dir == LC_L2C;  // transposed L2C starts with C^{-1}
      for (int i = threadIdx.x; i < nb * 2 * s; i += blockDim.x) {
        const int64_t j = p0 + i;
        R v = R(0);
        if (j < a.n) {
          v = lc_ld<R>(f + j * a.ie);
          if (scale) v *= cinv<R>(j);
        }
        fs[i] = v;
      }
      __syncthreads();
      R* lev = nodes + sub_off(depth);
      for (int t = threadIdx.x; t < nb * kSeg; t += blockDim.x) {
        const int j = t / kSeg, sigma = (t % kSeg) / LC_M, k = t % LC_M;
        const int64_t x = (x0 << depth) + j;
        R acc = R(0);
        if (node_valid(col, gb, x)) {
          const R* fseg = fs + j * 2 * s + sigma;
          const R* tcol = Ts + sigma * s * LC_M + k;
          for (int m = 0; m < s; ++m) acc = acc2(acc, fseg[2 * m], tcol[m * LC_M]);
          acc = finish(acc);
          Wb[(lc_seg_offset(gb) + x) * kSeg + sigma * LC_M + k] = acc;
        }
        lev[t] = acc;
      }
    } else {
      R* lev = nodes + sub_off(depth);
      for (int t = threadIdx.x; t < nb * kSeg; t += blockDim.x) {
        const int64_t x = (x0 << depth) + t / kSeg;
        lev[t] = node_valid(col, gb, x) ? Wb[(lc_seg_offset(gb) + x) * kSeg + t % kSeg] : R(0);
      }
    }
    for (int d = depth - 1; d >= 0; --d) {
      __syncthreads();
      const int gamma = rho + d;
      const int nd = 1 << d;
      const R* ch = nodes + sub_off(d + 1);
      // z0 = w(2x) + w(2x+1), z1 = w(2x) - w(2x+1)   (Algorithm a.1)
      for (int t = threadIdx.x; t < nd * kSeg; t += blockDim.x) {
        const int j = t / kSeg, e = t % kSeg;
        const R l = ch[(2 * j) * kSeg + e], r = ch[(2 * j + 1) * kSeg + e];
        zt[t] = l + r;
        zt[nd * kSeg + t] = l - r;
      }
      __syncthreads();
      R* lev = nodes + sub_off(d);
      for (int t = threadIdx.x; t < nd * kSeg; t += blockDim.x) {
        const int j = t / kSeg, sigma = (t % kSeg) / LC_M, k = t % LC_M;
        const int64_t x = (x0 << d) + j;
        R acc = R(0);
        if (node_valid(col, gamma, x)) {
          // Algorithm a.1: b_kj times z0 on even k-j, z1 on odd k-j (two chains)
          const R* z0 = zt + j * kSeg + sigma * LC_M;
          const R* z1 = z0 + nd * kSeg;
          for (int jj = 0; jj <= k; ++jj) acc = acc2(acc, Bt[jj * LC_M + k], ((k - jj) & 1) ? z1[jj] : z0[jj]);
          acc = finish(acc);
          Wb[(lc_seg_offset(gamma) + x) * kSeg + sigma * LC_M + k] = acc;
        }
        lev[t] = acc;
      }
    }
  }
}

// ------------------------------------------------------------- coupling
// Step 3 for every level in one launch.  Each CTA takes kCBlocks consecutive
// blocks b of one level; their 3 kCBlocks A-hat matrices are contiguous in
// the plan, so they are staged into shared memory with coalesced loads
// before the products.  Block b couples
//   forward:    rows 2b, 2b+1 with columns 2b+2, 2b+3:
//     c(2b) = A(b,0) w(2b+2) + A(b,1) w(2b+3),  c(2b+1) = A(b,2) w(2b+3);
//   transposed: columns 2b+2, 2b+3 with rows 2b, 2b+1:
//     c(2b+2) = A(b,0)^T w(2b),  c(2b+3) = A(b,1)^T w(2b) + A(b,2)^T w(2b+1).
constexpr int kCBlocks = 7;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_couple_blocks(Args<R> a, int adj, int g_lo, int g_hi) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  R* As = reinterpret_cast<R*>(smem_raw);          // [3 kCBlocks][M][M]
  R* Ws = As + 3 * kCBlocks * LC_M * LC_M;          // [2 kCBlocks][2][M]
  // locate (level, first block) of this CTA among levels [g_lo, g_hi)
  int gamma = g_lo;
  int64_t first = blockIdx.x, per;
  for (;;) {
    per = ((int64_t(2) << gamma) - 1 + kCBlocks - 1) / kCBlocks;
    if (first < per || gamma + 1 >= g_hi) break;
    first -= per;
    ++gamma;
  }
  const int64_t nblk = (int64_t(2) << gamma) - 1;  // b_gamma
  const int64_t b0 = first * kCBlocks;
  const int nb = int(nblk - b0 < kCBlocks ? nblk - b0 : kCBlocks);
  if (nb <= 0) return;
  const int64_t m0 = lc_ahat_offset(gamma) + 3 * b0;
  const uint32_t bytesA = uint32_t(3 * nb * LC_M * LC_M * sizeof(R));
  const uint32_t bytesW = uint32_t(2 * nb * kSeg * sizeof(R));
  const uint32_t mb = uint32_t(__cvta_generic_to_shared(&mbar));
  if (threadIdx.x == 0) {
    lc_mbar_init(mb);
  }
  uint32_t phase = 0;
  for (int64_t bt = blockIdx.y; bt < a.batch; bt += gridDim.y) {
    const R* Wl = a.t.W + (bt * a.nseg + lc_seg_offset(gamma)) * kSeg;
    R* Cl = a.t.Cc + (bt * a.nseg + lc_seg_offset(gamma)) * kSeg;
    // source segments: forward columns 2b0+2 .., transposed rows 2b0 ..
    const int64_t s0 = adj ? 2 * b0 : 2 * b0 + 2;
    const bool loadA = (bt == blockIdx.y);
    __syncthreads();
    if (threadIdx.x == 0) {
      lc_fence_proxy_async();
      const uint32_t bytes = bytesW + (loadA ? bytesA : 0u);
      lc_mbar_expect(mb, bytes);
      if (loadA && !(a.t.debug & 1)) lc_bulk_g2s(As, a.t.Ahat + m0 * (LC_M * LC_M), bytesA, mb);
      lc_bulk_g2s(Ws, Wl + s0 * kSeg, bytesW, mb);
    }
    bool ok = lc_mbar_wait_bounded(mb, phase);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(a.t.err, 1);
        lc_mbar_wait_bounded(mb, phase);  // let a late copy land before the CTA exits
      }
      return;
    }
    phase ^= 1u;
    for (int t = threadIdx.x; t < nb * kSeg; t += blockDim.x) {
      const int jb = t / kSeg;                  // block within the group
      const int sigma = (t % kSeg) / LC_M, k = t % LC_M;
      const R* A0 = As + (3 * jb) * (LC_M * LC_M);
      const R* w0 = Ws + (2 * jb) * kSeg + sigma * LC_M;
      const R* w1 = w0 + kSeg;
      R c0 = R(0), c0b = R(0), c1 = R(0);
      if (!adj) {
        // c(2b) = A(b,0) w(2b+2) + A(b,1) w(2b+3);  c(2b+1) = A(b,2) w(2b+3)
        for (int l = 0; l < LC_M; ++l) {
          const R wa = w0[l], wb = w1[l];
          c0 = acc2(c0, ahat_at(A0, 0, k, l), wa);
          c0b = acc2(c0b, ahat_at(A0, 1, k, l), wb);
          c1 = acc2(c1, ahat_at(A0, 2, k, l), wb);
        }
        R* out = Cl + (2 * (b0 + jb)) * kSeg + sigma * LC_M + k;
        out[0] = finish(c0) + finish(c0b);
        out[kSeg] = finish(c1);
      } else {
        // c(2b+2) = A(b,0)^T w(2b);  c(2b+3) = A(b,1)^T w(2b) + A(b,2)^T w(2b+1)
        for (int l = 0; l < LC_M; ++l) {
          const R wa = w0[l], wb = w1[l];
          c0 = acc2(c0, ahat_at(A0, 0, l, k), wa);
          c1 = acc2(c1, ahat_at(A0, 1, l, k), wa);
          c0b = acc2(c0b, ahat_at(A0, 2, l, k), wb);
        }
        R* out = Cl + (2 * (b0 + jb) + 2) * kSeg + sigma * LC_M + k;
        out[0] = finish(c0);
        out[kSeg] = finish(c1) + finish(c0b);
      }
    }
  }
}

template <typename R>
inline int64_t couple_ctas(int g_lo, int g_hi) {
  int64_t n = 0;
  for (int g = g_lo; g < g_hi; ++g) n += ((int64_t(2) << g) - 1 + kCBlocks - 1) / kCBlocks;
  return n;
}

// Shared-memory sizes (bytes) of the chunk kernels.
template <typename R>
inline size_t up_smem(int depth, int s, int leaf) {
  size_t v = size_t((2 << depth) - 1) * kSeg + 2 * size_t(1 << (depth > 0 ? depth - 1 : 0)) * kSeg;
  if (leaf) v += size_t(2) * s * LC_M + size_t(1 << depth) * 2 * s;
  return v * sizeof(R) + 16;
}
template <typename R>
inline size_t down_smem(int depth, int s, int fin, int64_t nrows_direct) {
  size_t v = size_t((2 << depth) - 1) * kSeg;
  if (fin) {
    const size_t rows = nrows_direct > 0 ? size_t(nrows_direct) : (size_t(1) << depth) * 2 * s;
    v += size_t(2) * s * LC_M;             // T
    v += rows + 4 * size_t(s) + 8;         // operand tile
    v += 2 * size_t(s) + 8;                // lambda_k
    v += rows + 2 * size_t(s) + 8;         // lambda_(i+k)
    if (nrows_direct > 0) v += 2 * rows;   // direct-only plans: full triangle tables
  }
  return v * sizeof(R) + 16;
}

// -------------------------------------------------------------- down chunk
// Root x0 = blockIdx.x at level rho; levels rho .. rho + depth, each node:
//   c(gamma, x) = couple(gamma, x) + [parent valid] B(x mod 2)^T c(gamma-1, x/2).
// fin != 0: the bottom level is the leaf level; finish with Steps 5-7 for the
// rows (forward) or columns (transposed) of the subtree.  L == 0: direct-only
// plan, one CTA computes the whole triangle.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_down_chunk(Args<R> a, int rho, int depth, int fin, int adj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R Bs[LC_M * LC_M];
  const bool col = adj;  // forward: row tree; transposed: column tree
  const int s = a.s, L = a.L;
  const int64_t two_s = 2 * int64_t(s);
  const int64_t x0 = blockIdx.x;
  R* nodes = reinterpret_cast<R*>(smem_raw);
  R* Ts = nodes + sub_off(depth + 1);
  for (int i = threadIdx.x; i < LC_M * LC_M; i += blockDim.x) Bs[i] = a.t.B[i];
  if (fin)
    for (int i = threadIdx.x; i < 2 * s * LC_M; i += blockDim.x) Ts[i] = a.t.T[i];
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    R* Cb = a.t.Cc + b * a.nseg * kSeg;
    if (L > 0) {
      for (int d = 0; d <= depth; ++d) {
        __syncthreads();
        const int gamma = rho + d;
        const int nd = 1 << d;
        R* lev = nodes + sub_off(d);
        for (int t = threadIdx.x; t < nd * kSeg; t += blockDim.x) {
          const int j = t / kSeg, sigma = (t % kSeg) / LC_M, k = t % LC_M;
          const int64_t x = (x0 << d) + j;
          R c = R(0);
          if (node_valid(col, gamma, x)) {
            c = Cb[(lc_seg_offset(gamma) + x) * kSeg + sigma * LC_M + k];  // Step 3 result (k_couple_blocks)
            if (gamma > 0 && node_valid(col, gamma - 1, x >> 1)) {
              const R* pv = (d == 0) ? Cb + (lc_seg_offset(gamma - 1) + (x >> 1)) * kSeg + sigma * LC_M
                                     : nodes + sub_off(d - 1) + (j >> 1) * kSeg + sigma * LC_M;
              // B(1) = B(0) with odd diagonals negated
              if constexpr (split_chains<R>::value) {
                R ce = R(0), co = R(0);
                for (int jj = k; jj < LC_M; jj += 2) ce = acc2(ce, Bs[jj * LC_M + k], pv[jj]);
                for (int jj = k + 1; jj < LC_M; jj += 2) co = acc2(co, Bs[jj * LC_M + k], pv[jj]);
                c = c + ((x & 1) ? finish(ce) - finish(co) : finish(ce) + finish(co));
              } else {
                const bool odd = (x & 1) != 0;
                for (int jj = k; jj < LC_M; ++jj) {
                  const R bjk = Bs[jj * LC_M + k];
                  c = acc2(c, (odd && ((jj - k) & 1)) ? negate(bjk) : bjk, pv[jj]);
                }
                c = finish(c);
              }
            }
          }
          lev[t] = c;
        }
      }
      if (!fin) {
        __syncthreads();
        const int gamma = rho + depth;
        const R* lev = nodes + sub_off(depth);
        for (int t = threadIdx.x; t < (1 << depth) * kSeg; t += blockDim.x) {
          const int64_t x = (x0 << depth) + t / kSeg;
          if (node_valid(col, gamma, x)) Cb[(lc_seg_offset(gamma) + x) * kSeg + t % kSeg] = lev[t];
        }
        continue;
      }
    }
    // ---------------- Steps 5-7 for this subtree's rows (forward) or columns (transposed)
    const R* leafc = nodes + sub_off(depth);
    const int64_t lo = (L > 0) ? (x0 << depth) * two_s : 0;
    const int64_t hi_raw = (L > 0) ? ((x0 + 1) << depth) * two_s : a.n;
    const int64_t hi = hi_raw < a.n ? hi_raw : a.n;
    if (lo >= hi) continue;
    const typename lc_io<R>::type* f = a.in + b * a.ib;
    R* opnd = Ts + 2 * s * LC_M;  // operand tile (input values, pre-scaled)
    int64_t olo, ohi;             // operand index range
    if (!adj) {
      olo = lo;
      ohi = (L > 0) ? hi + 2 * two_s : a.n;
    } else {
      olo = (L > 0) ? (lo - two_s > 0 ? lo - two_s : 0) : 0;
      ohi = hi;
    }
    if (ohi > a.n) ohi = a.n;
    const int64_t olen = ohi - olo;
    R* lamk = opnd + olen + 8;       // lambda_k (L2C) / u_k (C2L), k < kmax
    const int64_t kmax = (L > 0) ? two_s : (a.n + 1) / 2;
    R* lamm = lamk + kmax + 8;       // lambda_m / v_m for m in [mlo, mhi)
    const int64_t mlo = adj ? (olo + lo) / 2 : lo;
    const int64_t mhi = adj ? hi : (hi + ohi) / 2 + 1;
    const int64_t mcap = mhi < a.N ? mhi : a.N;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < olen; i += blockDim.x) {
      const int64_t q = olo + i;
      R v = lc_ld<R>(f + q * a.ie);
      if (!adj) {
        if (a.dir == LC_C2L) v = R(q) * v;                // L(i, j) = (2i+1) j u v: scale column j
      } else {
        v = (a.dir == LC_L2C) ? cinv<R>(q) * v : R(2 * q + 1) * v;  // C^{-1} r or (2i+1) r
      }
      opnd[i] = v;
    }
    for (int64_t k = threadIdx.x; k < kmax; k += blockDim.x) lamk[k] = (k < a.N) ? a.t.lam[k] : R(0);
    for (int64_t m = mlo + threadIdx.x; m < mhi; m += blockDim.x) lamm[m - mlo] = (m < mcap) ? a.t.lam2[m] : R(0);
    __syncthreads();
    const bool l2c = (a.dir == LC_L2C);
    // Work unit: within one 2s-row strip and parity, rows m and s-1-m, whose
    // band lengths add up to about 3s, so the threads of a warp stay balanced.
    const int half = (s + 1) / 2;
    const int64_t nstrips = (hi - lo + two_s - 1) / two_s;
    const int64_t units = nstrips * 2 * half;
    for (int64_t u = threadIdx.x; u < units; u += blockDim.x) {
      const int64_t strip = u / (2 * half);
      const int rem = int(u - strip * 2 * half);
      const int sigma = rem / half, mm = rem % half;
      for (int rep = 0; rep < 2; ++rep) {
        const int m = rep ? s - 1 - mm : mm;
        if (rep && m == mm) break;
        const int64_t i = lo + strip * two_s + 2 * m + sigma;
        if (i >= hi) continue;
        const int64_t v = i / two_s;
        R far = R(0);
        if (L > 0 && node_valid(col, L - 1, v)) {
          const R* c = leafc + (v - (x0 << depth)) * kSeg + sigma * LC_M;
          const R* Trow = Ts + (sigma * s + m) * LC_M;
          for (int k = 0; k < LC_M; ++k) far = acc2(far, c[k], Trow[k]);
          far = finish(far);
        }
        R near = R(0);
        if (!adj) {
          // row i: sum over j = i + 2k in the band  (eq:hik, eq:Lxymod)
          const int64_t end = (L > 0) ? (two_s * (v + 2) < a.n ? two_s * (v + 2) : a.n) : a.n;
          const int cnt = int((end - i + 1) >> 1);
          const R* fo = opnd + (i - olo);
          const R* lm = lamm + (i - mlo);
          for (int kk = 0; kk < cnt; ++kk) near = acc3(near, lamk[kk], lm[kk], fo[2 * kk]);
          near = finish(near);
          R res;
          if (l2c) {
            res = cinv<R>(i) * (far + near);
          } else {
            // (2i+1) u_k v_(i+k) (j f_j) summed; entry (0,0) = 1 adds f_0 (eq:Lxymod)
            res = far + R(2 * i + 1) * near;
            if (i == 0) res += lc_ld<R>(f);
          }
          lc_st<R>(a.out + b * a.ob + i * a.oe, res);
        } else {
          // column j = i: sum over rows r <= j in the band
          int64_t st = (L > 0) ? (two_s * (v - 1) > 0 ? two_s * (v - 1) : 0) : 0;
          if ((st & 1) != (i & 1)) ++st;
          const int cnt = int((i - st) / 2 + 1);
          const R* ro = opnd + (i - olo);          // ro[-2k] = row i - 2k
          const R* lm = lamm + (i - mlo);           // lm[-k]  = (r + i)/2 = i - k
          for (int k = 0; k < cnt; ++k) near = acc3(near, lamk[k], lm[-k], ro[-2 * k]);
          near = finish(near);
          if (!l2c) {
            near = R(i) * near;
            if (i == 0) near += lc_ld<R>(f);
          }
          lc_st<R>(a.out + b * a.ob + i * a.oe, far + near);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ driver
template <typename R>
inline void chunk_roots(int L, int leaf_depth, int chunk_depth, int* roots, int* count) {
  // roots[0] = top level of the first up chunk, then up to chunk_depth levels per chunk
  int n = 0;
  int r = L - 1 - leaf_depth;
  if (r < 0) r = 0;
  roots[n++] = r;
  while (r > 0) {
    r = r - chunk_depth > 0 ? r - chunk_depth : 0;
    roots[n++] = r;
  }
  *count = n;
}

template <typename R>
inline int launches_for(int L, int leaf_depth, int chunk_depth) {
  if (L <= 0) return 1;
  int roots[64], nr;
  chunk_roots<R>(L, leaf_depth, chunk_depth, roots, &nr);
  return 2 * nr + (roots[0] > 0 ? 2 : 1);
}

template <typename R>
lc_status set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) LC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return LC_OK;
}

template <typename R>
lc_status run(lc_plan_s* p, Args<R> a, cudaStream_t st, int adjoint) {
  const int L = a.L, s = a.s;
  const unsigned gy = unsigned(a.batch < 65535 ? a.batch : 65535);
  lc_timer_begin(p);
  if (L <= 0) {
    const size_t sm = down_smem<R>(0, s, 1, a.n);
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_down_chunk<R>), sm);
    if (e != LC_OK) return e;
    lc_timer_mark(p, st, LC_K_FINAL);
    k_down_chunk<R><<<dim3(1, gy), kThreads, sm, st>>>(a, 0, 0, 1, adjoint);
    LC_LAUNCH_CHECK();
    lc_timer_end(p, st);
    return LC_OK;
  }
  int roots[64], nr;
  chunk_roots<R>(L, p->leaf_depth, p->chunk_depth, roots, &nr);
  const size_t smc = (size_t(3) * kCBlocks * LC_M * LC_M + size_t(2) * kCBlocks * kSeg) * sizeof(R) + 16;
  {
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_couple_blocks<R>), smc);
    if (e != LC_OK) return e;
  }
  // Once the first up chunk is done, w is final on the levels [roots[0], L).
  // The coarse levels (up chunks, their coupling, their down chunks) form a
  // latency-bound chain of small grids; it runs on the plan's high-priority
  // side stream while the wide coupling of the fine levels runs on the
  // caller's stream, and the last down chunk waits for both.  (Everything
  // stays on the caller's stream when per-kernel timing is on.)
  const bool overlap = p->timing_slots <= 0 && roots[0] > 0 && p->side != nullptr;
  cudaStream_t sk = overlap ? p->side : st;  // stream of the coarse chain
  {  // first up chunk: leaf restriction and the fine levels
    const int rho = roots[0];
    const int depth = L - 1 - rho;
    const size_t sm = up_smem<R>(depth, s, 1);
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_up_chunk<R>), sm);
    if (e != LC_OK) return e;
    lc_timer_mark(p, st, LC_K_LEAF);
    k_up_chunk<R><<<dim3(unsigned(int64_t(4) << rho), gy), kThreads, sm, st>>>(a, rho, depth, 1, adjoint);
    LC_LAUNCH_CHECK();
  }
  if (overlap) {
    LC_CUDA_TRY(cudaEventRecord(p->ev_fork, st));
    LC_CUDA_TRY(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  }
  if (roots[0] > 0) {
    for (int c = 1; c < nr; ++c) {  // coarse up chunks
      const int rho = roots[c];
      const int depth = roots[c - 1] - rho;
      const size_t sm = up_smem<R>(depth, s, 0);
      lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_up_chunk<R>), sm);
      if (e != LC_OK) return e;
      lc_timer_mark(p, st, LC_K_UP);
      k_up_chunk<R><<<dim3(unsigned(int64_t(4) << rho), gy), kThreads, sm, sk>>>(a, rho, depth, 0, adjoint);
      LC_LAUNCH_CHECK();
    }
    lc_timer_mark(p, st, LC_K_COUPLE);  // coupling of the coarse levels
    k_couple_blocks<R><<<dim3(unsigned(couple_ctas<R>(0, roots[0])), gy), kThreads, smc, sk>>>(a, adjoint, 0, roots[0]);
    LC_LAUNCH_CHECK();
    for (int c = nr - 1; c >= 1; --c) {  // coarse down chunks: levels [roots[c], roots[c-1] - 1]
      const int rho = roots[c];
      const int depth = roots[c - 1] - 1 - rho;
      const size_t sm = down_smem<R>(depth, s, 0, 0);
      lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_down_chunk<R>), sm);
      if (e != LC_OK) return e;
      lc_timer_mark(p, st, LC_K_DOWN);
      k_down_chunk<R><<<dim3(unsigned(int64_t(4) << rho), gy), kThreads, sm, sk>>>(a, rho, depth, 0, adjoint);
      LC_LAUNCH_CHECK();
    }
    if (overlap) LC_CUDA_TRY(cudaEventRecord(p->ev_join, p->side));
  }
  // coupling of the fine levels [roots[0], L) on the caller's stream
  lc_timer_mark(p, st, LC_K_COUPLE);
  k_couple_blocks<R><<<dim3(unsigned(couple_ctas<R>(roots[0], L)), gy), kThreads, smc, st>>>(a, adjoint, roots[0], L);
  LC_LAUNCH_CHECK();
  if (overlap) LC_CUDA_TRY(cudaStreamWaitEvent(st, p->ev_join, 0));
  {  // last down chunk: fine levels, then Steps 5-7
    const int rho = roots[0];
    const int depth = L - 1 - rho;
    const size_t sm = down_smem<R>(depth, s, 1, 0);
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_down_chunk<R>), sm);
    if (e != LC_OK) return e;
    lc_timer_mark(p, st, LC_K_FINAL);
    k_down_chunk<R><<<dim3(unsigned(int64_t(4) << rho), gy), kThreads, sm, st>>>(a, rho, depth, 1, adjoint);
    LC_LAUNCH_CHECK();
  }
  lc_timer_end(p, st);
  return LC_OK;
}

}  // namespace lc_exec
