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
//     2^leaf_depth leaf segments and climbs leaf_depth levels (default 4);
//     each later one climbs up to chunk_depth more levels;
//   down chunks (top to bottom): each adds, level by level, the parent's
//     contribution of Step 4 to the coupling result of Step 3; the last chunk
//     ends at the leaves, does the spread and adds it to the band's part;
//   the band (k_near, Steps 6-7) needs only the input and lambda and runs
//     beside the whole far-field chain for one vector (batches: inside the
//     last down chunk).
// One vector: the first up chunk, the coupling of the fine levels and the
// last down chunk run on a plan stream; the coarse levels' up chunks, their
// coupling and their down chunks on a higher-priority one once the first up
// chunk is done; k_near on a lower-priority one from the start.  The last
// down chunk waits for all three.  For L = 13 (n = 1e6): 9 launches instead
// of 2L+2 = 28.
//
// The transposed pass (lc_adjoint) runs the same kernels with the roles of
// the trees exchanged: restriction over row segments and the row tree
// upwards, A-hat transposed in the coupling, the column tree downwards,
// spread over column segments and the transposed band.
#pragma once
#include "lc_internal.cuh"
#include "lc_tma.cuh"

namespace lc_exec {

template <typename R>
struct lc_io { typedef R type; };

template <typename R>
struct Args {
  const typename lc_io<R>::type* in;
  typename lc_io<R>::type* out;
  int64_t ib, ie, ob, oe;
  int64_t inner, iob, oob;  // two-level batches (lc_layout)
  int64_t n, N;
  int L, s;
  int64_t nseg;
  int64_t batch;
  int dir;
  lc_tables<R> t;
  // Per-vector power-of-two exponents (double-float tier; NULL elsewhere):
  // vector b is computed as x_b 2^-xe[b] and its output scaled back by
  // 2^xe[b], both exact, so that FP32's exponent range never clips FP64
  // data.  xe_part / xe_cnt: partial maxima and arrival counters of the
  // pre-pass that finds them (k_vec_exponent).
  int* xe;
  int* xe_part;
  unsigned* xe_cnt;
  // C2L row factor 2i + two_alpha (1 for Legendre; 2a for Gegenbauer a).
  double two_alpha;
  // Nodal variant (eq:AijLag): t.B holds the dense level maps P(0), P(1)
  // ([2][M][M]) instead of the triangular B(0).
  int nodal;
  // 1: let the next kernel of the stream start early (programmatic
  // dependent launch; set for the small grids of the coarse chain).
  int trigger;
};


template <typename R>
__device__ __forceinline__ R cinv(int64_t i) {
  return i == 0 ? R(0.31830988618379067154) : R(0.63661977236758134308);  // 1/pi, 2/pi
}

template <typename R>
__device__ __forceinline__ R lc_from_double(double x) { return R(x); }
// C2L row factor 2i + 2a of the entries (2i + 2a) j u_k v_(i+k): at a = 1/2
// (eq:Lxymod) the integer 2i + 1.
template <typename R>
__device__ __forceinline__ R c2l_row(const Args<R>& a, int64_t i) {
  if (a.two_alpha == 1.0) return R(2 * i + 1);
  return lc_from_double<R>(double(2 * i) + a.two_alpha);
}

// Input element x as R, times 2^-e (e: the vector's exponent, 0 unless the
// tier scales; see Args::xe).
template <typename R, typename IO>
__device__ __forceinline__ R lc_ld_in(const IO* p, int) { return R(*p); }
// Output values in the output precision IO from results v in R that carry
// the factor 2^-e (the caller has applied C^{-1} or the C2L row factor in R):
// v (out1), far + near (out2), acc + v (out_acc).  These are the sums of
// Step 7 of Algorithm 4 -- the near- and far-field parts of an output
// coefficient -- and they run in IO arithmetic: FP64 for every FP64-output
// tier.
template <typename R, typename IO>
__device__ __forceinline__ IO lc_out1(const R& v, int) { return IO(v); }
template <typename R, typename IO>
__device__ __forceinline__ IO lc_out2(const R& far, const R& near, int) { return IO(far) + IO(near); }
template <typename R, typename IO>
__device__ __forceinline__ IO lc_out_acc(IO acc, const R& v, int) { return acc + IO(v); }
// A tile's own exponent (double-float tier): kernels whose results go
// straight to the FP64 output may scale their input tile by the exponent of
// its own largest entry instead of the vector's, which needs no pre-pass.
template <typename R, typename IO>
struct local_scale { static constexpr bool value = false; };
__device__ __forceinline__ int vec_exp(const int* xe, int64_t b) { return xe ? xe[b] : 0; }
// Unbiased binary exponent of |x| (|x| in [2^e, 2^(e+1)), subnormals
// normalised), or kNoTileExp for zero, infinity and NaN.
constexpr int kNoTileExp = -(1 << 20);
__device__ __forceinline__ int tile_exp_of(double x) {
  const uint64_t u = __double_as_longlong(x);
  const int E = int((u >> 52) & 0x7ff);
  const uint64_t m = u & ((uint64_t(1) << 52) - 1);
  if (E == 2047) return kNoTileExp;
  if (E == 0) return m ? 1 - (__clzll(m) - 11) - 1023 : kNoTileExp;
  return E - 1023;
}
__device__ __forceinline__ int tile_exp_of(float x) { return tile_exp_of(double(x)); }
template <typename R>
__device__ __forceinline__ R negate(const R& v) { return -v; }
// Step 4 with one pass per parent for both children (halves the multiplies,
// halves the parallelism): worth it where the arithmetic pipe binds (FP64).
template <typename R>
struct eo_pairs { static constexpr bool value = false; };
template <>
struct eo_pairs<double> { static constexpr bool value = true; };
// A-hat in the compact double-float layout of lc_internal.cuh (leading words
// of all entries, trailing words of the k + l <= head triangle only).
template <typename R>
struct compact_ahat { static constexpr bool value = false; };

// Dot-product accumulation.  Generic: fused multiply-add in R.  The
// double-float tier specialises these to keep an unnormalised error word,
// which finish() folds back into the leading word (see lc_df.cu).  Sums of
// more than a few terms call finish() every few terms as well: the error
// word's own FP32 rounding grows with its size, and an error word left to
// collect 60 terms (a long band row) costs about 2e-13 relative.
template <typename R>
__device__ __forceinline__ R acc2(const R& acc, const R& a, const R& b) { return fma(a, b, acc); }
template <typename R>
__device__ __forceinline__ R acc3(const R& acc, const R& a, const R& b, const R& c) { return fma(a * b, c, acc); }
template <typename R>
__device__ __forceinline__ R finish(const R& acc) { return acc; }
// sum_{k < cnt} of the terms that step(acc, k) accumulates, renormalised
// every 4 terms.
template <typename R, typename F>
__device__ __forceinline__ R band_sum(int cnt, F&& step) {
  R acc = R(0);
  int k = 0;
#pragma unroll 1
  for (; k + 4 <= cnt; k += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = step(acc, k + q);
    acc = finish(acc);
  }
  for (; k < cnt; ++k) acc = step(acc, k);
  return finish(acc);
}
// A-hat(m)[k][l]: the FP64 table keeps row-major [k][l]; the FP32 copy is
// stored transposed, [l][k], so that threads that own consecutive k read
// consecutive addresses.  (The double-float copy is compact, read by the
// coupling kernel directly.)
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
constexpr int kPadS = 2;        // spare elements per 2s block of the band-sum tiles (even s)

// Node x at level gamma of the column tree (segments g >= 2) or of the row
// tree (segments v < 2 b_gamma).
__device__ __forceinline__ bool node_valid(bool col, int gamma, int64_t x) {
  const int64_t n = int64_t(4) << gamma;
  return col ? (x >= 2 && x < n) : (x >= 0 && x < n - 2);
}

// Elements of the up chunk's dynamic tiles: subtree nodes, the work array of
// Algorithm a.1, and for the leaf chunk T and the input strip; a nodal plan
// appends the transposed second level map P(1)^T.
__host__ __device__ inline size_t up_words(int depth, int s, int leaf) {
  size_t v = size_t((2 << depth) - 1) * kSeg + 2 * size_t(1 << (depth > 0 ? depth - 1 : 0)) * kSeg;
  if (leaf) v += size_t(2) * s * LC_M + size_t(1 << depth) * 2 * s;
  return v;
}

// Offsets (in R elements) of level d inside a subtree buffer.
__device__ __forceinline__ int sub_off(int d) { return ((1 << d) - 1) * kSeg; }

// Tile staging: n elements, element i read by ld(i) and written by st(i, v).
// Each thread issues up to U reads before its first write, so a tile costs
// one memory round trip per U elements a thread copies rather than one per
// element.  U > 1 pays in latency-bound launches of few CTAs (one vector);
// in launches that fill the GPU many times over (batches) the registers it
// holds cost more than it saves.
template <int U = 1, typename Ld, typename St>
__device__ __forceinline__ void stage(int n, Ld ld, St st) {
  for (int b0 = threadIdx.x; b0 < n; b0 += U * int(blockDim.x)) {
    decltype(ld(0)) v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = b0 + u * int(blockDim.x);
      if (i < n) v[u] = ld(i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = b0 + u * int(blockDim.x);
      if (i < n) st(i, v[u]);
    }
  }
}

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
  __shared__ R Bt[LC_M * LC_M];  // B(0) transposed: Bt[j][k] = b_kj (nodal: P(0) transposed)
  R* Bt1 = nodes + up_words(depth, a.s, leaf);  // nodal: P(1) transposed
  const bool col = !adj;
  const int s = a.s;
  const int64_t x0 = blockIdx.x;
  const int gb = rho + depth;
  const int nb = 1 << depth;
  const int nB = a.nodal ? 2 : 1;
  if (a.trigger) lc_grid_trigger();
  for (int i = threadIdx.x; i < nB * LC_M * LC_M; i += blockDim.x) {
    const int r = i % (LC_M * LC_M);
    (i < LC_M * LC_M ? Bt : Bt1)[(r % LC_M) * LC_M + r / LC_M] = a.t.B[i];
  }
  if (leaf)
    for (int i = threadIdx.x; i < 2 * s * LC_M; i += blockDim.x) Ts[i] = a.t.T[i];
  lc_grid_wait();  // (the plan tables above are constant)
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    R* Wb = a.t.W + b * a.nseg * kSeg;
    __syncthreads();
    if (leaf) {
      const int64_t p0 = (x0 << depth) * 2 * s;
      const typename lc_io<R>::type* f = a.in + lc_boff(b, a.ib, a.inner, a.iob);
      const bool scale = adj && a.dir == LC_L2C;  // transposed L2C starts with C^{-1}
      const int e = vec_exp(a.xe, b);
      for (int i = threadIdx.x; i < nb * 2 * s; i += blockDim.x) {
        const int64_t j = p0 + i;
        R v = R(0);
        if (j < a.n) {
          v = lc_ld_in<R>(f + j * a.ie, e);
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
#pragma unroll 4
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
      for (int t = threadIdx.x; t < (a.nodal ? 0 : nd * kSeg); t += blockDim.x) {
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
          if (a.nodal) {  // dense P(0) w(2x) + P(1) w(2x+1)
            const R* wl = ch + (2 * j) * kSeg + sigma * LC_M;
            const R* wr = wl + kSeg;
#pragma unroll 6
            for (int jj = 0; jj < LC_M; ++jj) {
              acc = acc2(acc, Bt[jj * LC_M + k], wl[jj]);
              acc = acc2(acc, Bt1[jj * LC_M + k], wr[jj]);
            }
          } else if constexpr (eo_pairs<R>::value) {  // FP64 pipe: only the nonzero b_kj (j <= k)
            for (int jj = 0; jj <= k; ++jj) acc = acc2(acc, Bt[jj * LC_M + k], ((k - jj) & 1) ? z1[jj] : z0[jj]);
          } else {
            // b_kj = 0 exactly for j > k, so all M terms, unrolled: the lanes of a
            // warp (different k) run the same instructions, with no loop or select
            const R* ze = (k & 1) ? z1 : z0;  // even j
            const R* zo = (k & 1) ? z0 : z1;  // odd j
#pragma unroll
            for (int jj = 0; jj < LC_M; ++jj) acc = acc2(acc, Bt[jj * LC_M + k], (jj & 1) ? zo[jj] : ze[jj]);
          }
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

// Step 3 products of one CTA's group of nb blocks from the compact
// double-float A-hat (layout in lc_internal.cuh) staged at Af.  Thread item
// (q, jb, sigma): q is the row k of A-hat (forward) or its column l
// (transposed), consecutive threads take consecutive (block jb, parity
// sigma) with the same q, so that a warp shares the split point: the terms
// with k + l <= head in double-float, the rest as FP32 products of the
// leading words, gathered in an FP32 sum that joins the error word.
template <typename R>
__device__ __forceinline__ void couple_compact(const Args<R>& a, int adj, int nb, int64_t b0, const float* Af,
                                               const R* Ws, R* Cl) {
  const int head = lc_dfa_head(a.dir);
  const int mw = lc_dfa_words(a.dir);
  const int pairs = 2 * nb;
  for (int t = threadIdx.x; t < nb * kSeg; t += blockDim.x) {
    const int q = t / pairs;
    const int jb = (t % pairs) >> 1, sigma = t & 1;
    const float* A0 = Af + 3 * jb * mw;   // A(b,0); A(b,1), A(b,2) follow at mw, 2 mw
    const float* L0 = A0 + LC_M * LC_M;   // trailing words
    const R* w0 = Ws + (2 * jb) * kSeg + sigma * LC_M;
    const R* w1 = w0 + kSeg;
    const int nd = head + 1 - q > 0 ? head + 1 - q : 0;  // double-float terms of row/column q
    R c0 = R(0), c0b = R(0), c1 = R(0);
    float e0 = 0.0f, e0b = 0.0f, e1 = 0.0f;
    if (!adj) {
      // c(2b) = A(b,0) w(2b+2) + A(b,1) w(2b+3);  c(2b+1) = A(b,2) w(2b+3)
      const float* h = A0 + q * LC_M;
      const float* lo = L0 + lc_dfa_rowstart(q, head);
      int l = 0;
      for (; l < nd; ++l) {
        const R wa = w0[l], wb = w1[l];
        c0 = acc2(c0, R(h[l], lo[l]), wa);
        c0b = acc2(c0b, R(h[mw + l], lo[mw + l]), wb);
        c1 = acc2(c1, R(h[2 * mw + l], lo[2 * mw + l]), wb);
      }
      for (; l < LC_M; ++l) {
        const float wa = w0[l].hi, wb = w1[l].hi;
        e0 = fmaf(h[l], wa, e0);
        e0b = fmaf(h[mw + l], wb, e0b);
        e1 = fmaf(h[2 * mw + l], wb, e1);
      }
      R* out = Cl + (2 * (b0 + jb)) * kSeg + sigma * LC_M + q;
      out[0] = finish(R(c0.hi, c0.lo + e0)) + finish(R(c0b.hi, c0b.lo + e0b));
      out[kSeg] = finish(R(c1.hi, c1.lo + e1));
    } else {
      // c(2b+2) = A(b,0)^T w(2b);  c(2b+3) = A(b,1)^T w(2b) + A(b,2)^T w(2b+1)
      const float* h = A0 + q;
      int k = 0, rs = q;  // rs: trailing-word index of entry (k, q)
      for (; k < nd; ++k) {
        const R wa = w0[k], wb = w1[k];
        c0 = acc2(c0, R(h[k * LC_M], L0[rs]), wa);
        c1 = acc2(c1, R(h[mw + k * LC_M], L0[mw + rs]), wa);
        c0b = acc2(c0b, R(h[2 * mw + k * LC_M], L0[2 * mw + rs]), wb);
        rs += head + 1 - k;
      }
      for (; k < LC_M; ++k) {
        const float wa = w0[k].hi, wb = w1[k].hi;
        e0 = fmaf(h[k * LC_M], wa, e0);
        e1 = fmaf(h[mw + k * LC_M], wa, e1);
        e0b = fmaf(h[2 * mw + k * LC_M], wb, e0b);
      }
      R* out = Cl + (2 * (b0 + jb) + 2) * kSeg + sigma * LC_M + q;
      out[0] = finish(R(c0.hi, c0.lo + e0));
      out[kSeg] = finish(R(c1.hi, c1.lo + e1)) + finish(R(c0b.hi, c0b.lo + e0b));
    }
  }
}

// Bytes of one A-hat matrix as the coupling kernel stages it.
template <typename R>
__host__ __device__ inline size_t ahat_matrix_bytes(int dir) {
  return compact_ahat<R>::value ? size_t(lc_dfa_words(dir)) * sizeof(float) : size_t(LC_M) * LC_M * sizeof(R);
}
template <typename R>
inline size_t couple_smem(int dir) {
  return 3 * kCBlocks * ahat_matrix_bytes<R>(dir) + size_t(2) * kCBlocks * kSeg * sizeof(R) + 16;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_couple_blocks(Args<R> a, int adj, int g_lo, int g_hi) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  const size_t mat = ahat_matrix_bytes<R>(a.dir);
  R* As = reinterpret_cast<R*>(smem_raw);                                // [3 kCBlocks] matrices
  R* Ws = reinterpret_cast<R*>(smem_raw + 3 * kCBlocks * mat);           // [2 kCBlocks][2][M]
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
  if (a.trigger) lc_grid_trigger();
  if (nb <= 0) return;
  lc_grid_wait();
  const int64_t m0 = lc_ahat_offset(gamma) + 3 * b0;
  const uint32_t bytesA = uint32_t(3 * nb * mat);
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
      if (loadA && !(a.t.debug & 1))
        lc_bulk_g2s(As, reinterpret_cast<const unsigned char*>(a.t.Ahat) + m0 * mat, bytesA, mb);
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
    if constexpr (compact_ahat<R>::value) {
      couple_compact(a, adj, nb, b0, reinterpret_cast<const float*>(As), Ws, Cl);
    } else {
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
}

template <typename R>
inline int64_t couple_ctas(int g_lo, int g_hi) {
  int64_t n = 0;
  for (int g = g_lo; g < g_hi; ++g) n += ((int64_t(2) << g) - 1 + kCBlocks - 1) / kCBlocks;
  return n;
}

// Shared-memory sizes (bytes) of the chunk kernels.
template <typename R>
inline size_t up_smem(int depth, int s, int leaf, int nodal) {
  return (up_words(depth, s, leaf) + (nodal ? size_t(LC_M) * LC_M : 0)) * sizeof(R) + 16;
}
template <typename R>
inline size_t down_smem(int depth, int s, int fin) {
  size_t v = size_t((2 << depth) - 1) * kSeg;
  if (fin) v += size_t(2) * s * LC_M;  // T
  return v * sizeof(R) + 16;
}
constexpr int kNearStrips = 16;  // strips of 2s rows per CTA of k_near
// rows: rows of the tile (a multiple of 2s), or, direct != 0, n of a
// direct-only plan (the whole triangle).
template <typename R>
inline size_t near_smem(int s, int64_t nrows, int direct) {
  const int64_t nrows_direct = direct ? nrows : 0;
  const size_t rows = size_t(nrows);
  const size_t pad = (direct || (s & 1)) ? 0 : kPadS;
  const size_t blocks = rows / (2 * size_t(s)) + 4;
  size_t v = rows + 4 * size_t(s) + 8 + pad * blocks;               // operand tile
  v += 2 * size_t(s) + 8;                                            // lambda_k
  v += (pad ? 2 : 1) * (rows + 2 * size_t(s) + 16 + pad * blocks);  // lambda_(i+k), per parity if padded
  if (nrows_direct > 0) v += 2 * rows;                               // direct-only plans: whole triangle
  return v * sizeof(R) + 16;
}

// ------------------------------------------------- near-field band sums
// Shared tiles of the band sums for even s: kPadS spare elements after every
// block of 2s; pad_index maps an offset x >= 0 from the block origin.
__device__ __forceinline__ int pad_index(int64_t x, int64_t two_s, int pad) {
  return int(x + (pad ? pad * (x / two_s) : 0));
}
// Forward rows i and i + 2 of one parity: row i + 2r takes, at step k, the
// entry factors lamk[k] and lm[2r + k] (lambda_k, lambda_(i+2r+k), or u, v
// for C2L) and the operand fo[2(r + k)].  Row i has cnt >= 1 terms, row i + 2
// one fewer.  fwd_steps runs steps [k, kend) two at a time (renormalising
// the sums after every second pair of steps) with the operand
// and lambda tiles fp, lp; the values of row i + 2 at step k are those of row
// i at steps k + 1 and k + 2, kept in registers (f0, l0, l1) from step to step.
template <typename R>
__device__ __forceinline__ void fwd_steps(const R* __restrict__ lamk, const R* __restrict__ fp,
                                          const R* __restrict__ lp, int& k, int kend, R& a0, R& a1, R& f0,
                                          R& l0, R& l1) {
  int kk = k;
  R A0 = a0, A1 = a1, F0 = f0, L0 = l0, L1 = l1;
  const R* pk = lamk + kk;
  const R* pf = fp + 2 * kk;
  const R* pl = lp + kk;
  int it = 0;
#pragma unroll 4
  for (; kk + 2 <= kend; kk += 2, pk += 2, pf += 4, pl += 2, ++it) {
    const R k0 = pk[0], k1 = pk[1];
    const R F1 = pf[2], F2 = pf[4];
    const R L2 = pl[2], L3 = pl[3];
    A0 = acc3(A0, k0, L0, F0);
    A1 = acc3(A1, k0, L2, F1);
    A0 = acc3(A0, k1, L1, F1);
    A1 = acc3(A1, k1, L3, F2);
    if (it & 1) {
      A0 = finish(A0);
      A1 = finish(A1);
    }
    F0 = F2;
    L0 = L2;
    L1 = L3;
  }
  if (kk < kend) {
    const R k0 = lamk[kk];
    const R F1 = fp[2 * kk + 2];
    const R L2 = lp[kk + 2];
    A0 = acc3(A0, k0, L0, F0);
    A1 = acc3(A1, k0, L2, F1);
    F0 = F1;
    L0 = L1;
    L1 = L2;
    ++kk;
  }
  k = kk;
  a0 = A0;
  a1 = A1;
  f0 = F0;
  l0 = L0;
  l1 = L1;
}
// With padded tiles (pad != 0) the operand reads cross into the next block
// from step kF on and the lambda reads from step kL on (kF <= kL).
template <typename R>
__device__ __forceinline__ void near_fwd2(const R* __restrict__ lamk, const R* __restrict__ lm,
                                          const R* __restrict__ fo, int cnt, int kF, int kL, int pad, R& n0,
                                          R& n1) {
  R a0 = R(0), a1 = R(0);
  R f0 = fo[0], l0 = lm[0], l1 = lm[1];
  const int last = cnt - 1;
  int k = 0;
  if (pad == 0) {
    fwd_steps(lamk, fo, lm, k, last, a0, a1, f0, l0, l1);
  } else {
    fwd_steps(lamk, fo, lm, k, kF < last ? kF : last, a0, a1, f0, l0, l1);
    fwd_steps(lamk, fo + pad, lm, k, kL < last ? kL : last, a0, a1, f0, l0, l1);
    fwd_steps(lamk, fo + pad, lm + pad, k, last, a0, a1, f0, l0, l1);
  }
  a0 = acc3(a0, lamk[k], l0, f0);  // last term of row i
  n0 = finish(a0);
  n1 = finish(a1);
}
// Transposed: columns i and i + 2 of one parity; column i sums rows i - 2k for
// k < cnt, column i + 2 rows i + 2 - 2k for k <= cnt (same first row).  has1
// is false when column i + 2 lies outside the staged operand range.
template <typename R>
__device__ __forceinline__ void adj_steps(const R* __restrict__ lamk, const R* __restrict__ rp,
                                          const R* __restrict__ lp, int& k, int kend, R& a0, R& a1, R& g1,
                                          R& l1, R& l2) {
  int kk = k;
  R A0 = a0, A1 = a1, G1 = g1, L1 = l1, L2 = l2;
  const R* pk = lamk + kk;
  const R* pg = rp - 2 * kk;
  const R* pl = lp - kk;
  int it = 0;
#pragma unroll 4
  for (; kk + 2 <= kend; kk += 2, pk += 2, pg -= 4, pl -= 2, ++it) {
    const R k0 = pk[0], k1 = pk[1];
    const R G0 = pg[0], Gm = pg[-2];
    const R L0 = pl[0], Lm = pl[-1];
    A0 = acc3(A0, k0, L0, G0);
    A1 = acc3(A1, k0, L2, G1);
    A0 = acc3(A0, k1, Lm, Gm);
    A1 = acc3(A1, k1, L1, G0);
    if (it & 1) {
      A0 = finish(A0);
      A1 = finish(A1);
    }
    G1 = Gm;
    L2 = L0;
    L1 = Lm;
  }
  if (kk < kend) {
    const R k0 = lamk[kk];
    const R G0 = rp[-2 * kk];
    const R L0 = lp[-kk];
    A0 = acc3(A0, k0, L0, G0);
    A1 = acc3(A1, k0, L2, G1);
    G1 = G0;
    L2 = L1;
    L1 = L0;
    ++kk;
  }
  k = kk;
  a0 = A0;
  a1 = A1;
  g1 = G1;
  l1 = L1;
  l2 = L2;
}
// Padded tiles: operand reads drop into the previous block from step kF on,
// lambda reads from step kL on.
template <typename R>
__device__ __forceinline__ void near_adj2(const R* __restrict__ lamk, const R* __restrict__ lm,
                                          const R* __restrict__ ro, int cnt, bool has1, int kF, int kL, int pad,
                                          R& n0, R& n1) {
  R a0 = R(0), a1 = R(0);
  R g1 = has1 ? ro[2] : R(0), l1 = lm[1], l2 = lm[2];
  int k = 0;
  if (pad == 0) {
    adj_steps(lamk, ro, lm, k, cnt, a0, a1, g1, l1, l2);
  } else {
    adj_steps(lamk, ro, lm, k, kF < cnt ? kF : cnt, a0, a1, g1, l1, l2);
    adj_steps(lamk, ro - pad, lm, k, kL < cnt ? kL : cnt, a0, a1, g1, l1, l2);
    adj_steps(lamk, ro - pad, lm - pad, k, cnt, a0, a1, g1, l1, l2);
  }
  a1 = acc3(a1, lamk[k], l2, g1);  // first row of the band, column i + 2 only
  n0 = finish(a0);
  n1 = finish(a1);
}

// ----------------------------------------------------------- near field
// Steps 6 and 7 for the band (eq:hik, eq:Lxymod): CTA x takes the rows
// (forward) or columns (transposed) of kNearStrips strips of 2s and writes
// the near-field part of the output, scaled as the output is (C^{-1} for
// L2C; the (2i+1) and j factors of the C2L entries).  The far-field part is
// added by the last down chunk.  The band needs only the input and lambda,
// so this kernel runs beside the far-field chain.  L == 0 (direct-only plan):
// one CTA, the whole triangle, which is then the complete result.
// The band for the rows (forward) or columns (transposed) [lo, hi) of batch
// member b, its tiles at `tile` in shared memory (near_smem bytes).  add == 0:
// the output receives the band's part; add != 0: it already holds the
// far-field part of these rows, written by this CTA before a barrier, and the
// band's part is added.
template <typename R>
__device__ __forceinline__ void near_tile(const Args<R>& a, int64_t b, int64_t lo, int64_t hi, int adj,
                                          unsigned char* tile) {
  typedef typename lc_io<R>::type IO;
  const int s = a.s, L = a.L;
  const int64_t two_s = 2 * int64_t(s);
  const bool l2c = (a.dir == LC_L2C);
  const IO* f = a.in + lc_boff(b, a.ib, a.inner, a.iob);
  IO* const ob = a.out + lc_boff(b, a.ob, a.inner, a.oob);
  __shared__ int tile_exp;
  R* opnd = reinterpret_cast<R*>(tile);  // operand tile (input values, pre-scaled)
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
  // Even s: the operand and lambda_m tiles keep kPadS spare elements after
  // every 2s-element block (blocks aligned to strips), so that threads
  // reading 2s apart hit distinct banks; lambda_m is then kept twice, its
  // blocks aligned to the rows of each parity.
  const int pad = (L > 0 && !(s & 1)) ? kPadS : 0;
  const int64_t pbase = adj ? lo - two_s : lo;  // operand block origin
  const int64_t lbase = lo - two_s;             // lambda_m block origin (+ sigma)
  const int ooff = pad_index(olo - pbase, two_s, pad);
  const int64_t olen_p = olen + (pad ? pad * (olen / two_s + 2) : 0);
  R* lamk = opnd + olen_p + 8;     // lambda_k (L2C) / u_k (C2L), k < kmax + 2
  const int64_t kmax = (L > 0) ? two_s : (a.n + 1) / 2;
  R* lamm = lamk + kmax + 8;       // lambda_m / v_m for m in [mlo, mhi + 2)
  const int64_t mlo = adj ? (olo + lo) / 2 : lo;
  const int64_t mhi = adj ? hi : (hi + ohi) / 2 + 1;
  const int64_t mcap = mhi < a.N ? mhi : a.N;
  const int64_t mlen = mhi + 2 - mlo;
  R* lamm1 = lamm + mlen + (pad ? pad * (mlen / two_s + 2) : 0) + 8;  // parity-1 copy (pad != 0)
  const int moff0 = pad_index(mlo - lbase, two_s, pad);
  const int moff1 = pad ? pad_index(mlo - lbase - 1, two_s, pad) : 0;
  // the operand tile, scaled by 2^-e: e is the vector's exponent, or, where
  // the tier allows, this tile's own (the band's outputs need no other)
  auto scale_put = [&](int64_t q, R v) {
    if (!adj) {
      if (a.dir == LC_C2L) v = R(q) * v;  // L(i, j) = (2i+2a) j u v: scale column j
    } else {
      v = (a.dir == LC_L2C) ? cinv<R>(q) * v : c2l_row(a, q) * v;  // C^{-1} r or (2i+2a) r
    }
    opnd[pad_index(q - pbase, two_s, pad) - ooff] = v;
  };
  int e;
  if constexpr (local_scale<R, IO>::value) {
    // raw FP64 values first (same 8 bytes per slot), the tile's largest
    // exponent, then the scaled conversion in place
    static_assert(sizeof(R) == sizeof(IO), "in-place conversion needs equal sizes");
    if (threadIdx.x == 0) tile_exp = kNoTileExp;
    __syncthreads();
    int m = kNoTileExp;
    stage<4>(
        int(olen), [&](int i) { return f[(olo + i) * a.ie]; },
        [&](int i, IO x) {
          m = max(m, tile_exp_of(x));
          reinterpret_cast<IO*>(opnd)[pad_index(olo + i - pbase, two_s, pad) - ooff] = x;
        });
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m > kNoTileExp) atomicMax(&tile_exp, m);
    __syncthreads();
    e = tile_exp == kNoTileExp ? 0 : tile_exp;
    for (int i = threadIdx.x; i < int(olen); i += blockDim.x) {  // the slots this thread staged
      const int64_t q = olo + i;
      const int slot = pad_index(q - pbase, two_s, pad) - ooff;
      scale_put(q, lc_ld_in<R>(reinterpret_cast<const IO*>(opnd) + slot, e));
    }
  } else {
    e = vec_exp(a.xe, b);
    stage<4>(int(olen), [&](int i) { return f[(olo + i) * a.ie]; },
             [&](int i, IO x) { scale_put(olo + i, lc_ld_in<R>(&x, e)); });
  }
  // output i receives v (scaled back by 2^e, in IO arithmetic); C2L row
  // (column) 0 also takes the entry L(0,0) = 1 times f_0 (eq:Lxymod)
  auto put = [&](int64_t i, const R& v) {
    IO r = lc_out1<R, IO>(v, e);
    if (!l2c && i == 0) r += f[0];
    ob[i * a.oe] = r;
  };
  stage<4>(int(kmax + 2), [&](int k) { return k < a.N ? a.t.lam[k] : R(0); }, [&](int k, R v) { lamk[k] = v; });
  stage<4>(
      int(mlen), [&](int j) { return mlo + j < mcap ? a.t.lam2[mlo + j] : R(0); },
      [&](int j, R v) {
        const int64_t m = mlo + j;
        lamm[pad_index(m - lbase, two_s, pad) - moff0] = v;
        if (pad) lamm1[pad_index(m - lbase - 1, two_s, pad) - moff1] = v;
      });
  __syncthreads();
  if (L == 0) {
    // Direct-only plan: every row (column) by itself, the whole triangle.
    for (int64_t i = threadIdx.x; i < hi; i += blockDim.x) {
      R near = R(0);
      if (!adj) {
        const int cnt = int((a.n - i + 1) >> 1);
        const R* fo = opnd + (i - olo);
        const R* lm = lamm + (i - mlo);
        near = band_sum<R>(cnt, [&](const R& c, int kk) { return acc3(c, lamk[kk], lm[kk], fo[2 * kk]); });
        put(i, l2c ? cinv<R>(i) * near : c2l_row(a, i) * near);
      } else {
        const int cnt = int(i / 2 + 1);
        const R* ro = opnd + (i - olo);
        const R* lm = lamm + (i - mlo);
        near = band_sum<R>(cnt, [&](const R& c, int k) { return acc3(c, lamk[k], lm[-k], ro[-2 * k]); });
        put(i, l2c ? near : R(i) * near);
      }
    }
    return;
  }
  // Work item: rows (forward) or columns (transposed) m0 = 2g and m0 + 1 of
  // parity sigma in one 2s-row strip, i.e. i and i + 2, summed together by
  // near_fwd2 / near_adj2; then the mirrored pair g' = ng - 1 - g, so that
  // every item has about 3s band terms per row (when that still leaves an item
  // for every thread; otherwise one pair of rows per item).  Consecutive threads take
  // consecutive (strip, parity) with the same g: their band lengths agree,
  // and their shared-memory reads, 2s apart, fall into distinct banks when
  // s is odd.
  const int ng = (s + 1) >> 1, npair = (ng + 1) >> 1;
  const int nstrips = int((hi - lo + two_s - 1) / two_s);
  const bool mirror = nstrips * 2 * npair >= int(blockDim.x);
  const int items = nstrips * 2 * (mirror ? npair : ng);
  for (int u = threadIdx.x; u < items; u += blockDim.x) {
    const int sigma = u & 1;
    const int t = (u >> 1) % nstrips;
    const int pr = (u >> 1) / nstrips;
    for (int rep = 0; rep < 2; ++rep) {
      const int g = rep ? ng - 1 - pr : pr;
      if (rep && (g == pr || !mirror)) break;
      const int m0 = 2 * g;
      const int64_t i = lo + t * two_s + 2 * m0 + sigma;
      if (i >= hi) continue;
      const bool has1 = (m0 + 1 < s) && (i + 2 < hi);  // second row/column i + 2 in this strip
      const int64_t v = i / two_s;
      const R* op = opnd + (pad_index(i - pbase, two_s, pad) - ooff);
      const R* lm = sigma && pad ? lamm1 + (pad_index(i - lbase - 1, two_s, pad) - moff1)
                                 : lamm + (pad_index(i - lbase, two_s, pad) - moff0);
      R n0, n1;
      if (!adj) {
        const int64_t e2 = two_s * (v + 2);
        const int64_t end = e2 < a.n ? e2 : a.n;
        near_fwd2(lamk, lm, op, int((end - i + 1) >> 1), s - m0 - 1, 2 * s - 2 * m0 - 2, pad, n0, n1);
        if (l2c) {
          put(i, cinv<R>(i) * n0);
          if (has1) put(i + 2, cinv<R>(i + 2) * n1);
        } else {
          // (2i+2a) u_k v_(i+k) (j f_j) summed
          put(i, c2l_row(a, i) * n0);
          if (has1) put(i + 2, c2l_row(a, i + 2) * n1);
        }
      } else {
        int64_t st = two_s * (v - 1) > 0 ? two_s * (v - 1) : 0;
        if ((st & 1) != (i & 1)) ++st;
        near_adj2(lamk, lm, op, int((i - st) / 2 + 1), has1, m0 + 1, 2 * m0 + 1, pad, n0, n1);
        put(i, l2c ? n0 : R(i) * n0);
        if (has1) put(i + 2, l2c ? n1 : R(i + 2) * n1);
      }
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 4) k_near(Args<R> a, int adj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t two_s = 2 * int64_t(a.s);
  // groups of kNearStrips strips, grid-strided (the grid may be smaller than
  // the number of groups, to leave SM room for the far-field chain)
  const int64_t groups = (a.L > 0) ? (a.n + kNearStrips * two_s - 1) / (kNearStrips * two_s) : 1;
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    for (int64_t gi = blockIdx.x; gi < groups; gi += gridDim.x) {
      const int64_t lo = (a.L > 0) ? gi * kNearStrips * two_s : 0;
      const int64_t hi_raw = (a.L > 0) ? lo + kNearStrips * two_s : a.n;
      const int64_t hi = hi_raw < a.n ? hi_raw : a.n;
      if (lo >= hi) continue;
      __syncthreads();  // shared tiles of the previous group are free
      near_tile(a, b, lo, hi, adj, smem_raw);
    }
  }
}

// -------------------------------------------------------------- down chunk
// Root x0 = blockIdx.x at level rho; levels rho .. rho + depth, each node:
//   c(gamma, x) = couple(gamma, x) + [parent valid] B(x mod 2)^T c(gamma-1, x/2).
// fin != 0: the bottom level is the leaf level; finish with Step 5 for the
// rows (forward) or columns (transposed) of the subtree and add the
// near-field part that k_near has written to the output (Steps 6-7), or,
// with fuse (batched plans), compute that part here as well.
template <typename R, bool fuse>
__global__ void __launch_bounds__(kThreads, fuse ? 5 : 6) k_down_chunk(Args<R> a, int rho, int depth, int fin, int adj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ R Bs[LC_M * LC_M];
  const bool col = adj;  // forward: row tree; transposed: column tree
  const int s = a.s, L = a.L;
  const int64_t two_s = 2 * int64_t(s);
  const int64_t x0 = blockIdx.x;
  R* nodes = reinterpret_cast<R*>(smem_raw);
  R* Ts = nodes + sub_off(depth + 1);
  __shared__ R par[kSeg];  // c of the root's parent
  // B(1): B(0) with odd diagonals negated; nodal: the second level map P(1)
  __shared__ R Bs1[LC_M * LC_M];
  constexpr int U = fuse ? 1 : 4;
  if (a.trigger) lc_grid_trigger();
  stage<U>(LC_M * LC_M, [&](int i) { return a.t.B[i]; }, [&](int i, R v) {
    Bs[i] = v;
    if (!a.nodal) Bs1[i] = ((i / LC_M - i % LC_M) & 1) ? negate(v) : v;
  });
  if (a.nodal) stage<U>(LC_M * LC_M, [&](int i) { return a.t.B[LC_M * LC_M + i]; }, [&](int i, R v) { Bs1[i] = v; });
  if (fin) stage<U>(2 * s * LC_M, [&](int i) { return a.t.T[i]; }, [&](int i, R v) { Ts[i] = v; });
  lc_grid_wait();  // (the plan tables above are constant)
  for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
    R* Cb = a.t.Cc + b * a.nseg * kSeg;
    {
      __syncthreads();  // shared tiles of the previous batch member are free
      // Step 3 results of every node of the subtree (zero where the node is not
      // valid) and of the root's parent, all read before any is used (one
      // round trip instead of one per level).  Batched plans, whose launches
      // fill the GPU many times over, read them level by level instead
      // (except for the FP64 E/O form, which works on the staged copy).
      const int ntot = sub_off(depth + 1);
      if (!fuse || eo_pairs<R>::value) stage<U>(
          ntot + kSeg,
          [&](int q) {
            if (q >= ntot) {
              const int64_t xp = x0 >> 1;
              return rho > 0 && node_valid(col, rho - 1, xp) ? Cb[(lc_seg_offset(rho - 1) + xp) * kSeg + (q - ntot)]
                                                             : R(0);
            }
            const int d = 31 - __clz((q / kSeg) + 1);  // level of entry q
            const int64_t x = (x0 << d) + (q - sub_off(d)) / kSeg;
            return node_valid(col, rho + d, x) ? Cb[(lc_seg_offset(rho + d) + x) * kSeg + (q - sub_off(d)) % kSeg]
                                               : R(0);
          },
          [&](int q, R v) {
            if (q >= ntot) par[q - ntot] = v;
            else nodes[q] = v;
          });
      // Step 4 level by level.  B(1) is B(0) with its odd diagonals negated.
      // FP64 (bound by its pipe): one pass over a parent's c gives E (even
      // diagonals of B(0)^T c) and O (odd diagonals); child 2x receives E + O,
      // child 2x + 1 receives E - O -- half the multiplies.  Other types
      // (latency-bound): one thread per child entry, twice the parallelism.
      if (eo_pairs<R>::value && !a.nodal) {
        for (int d = 0; d <= depth; ++d) {
          __syncthreads();
          const int gamma = rho + d;
          if (gamma == 0) continue;
          const int np = d == 0 ? 1 : 1 << (d - 1);  // parents inside the subtree (d == 0: the root's)
          R* lev = nodes + sub_off(d);
          for (int t = threadIdx.x; t < np * kSeg; t += blockDim.x) {
            const int jp = t / kSeg, sigma = (t % kSeg) / LC_M, k = t % LC_M;
            const int64_t xp = d == 0 ? (x0 >> 1) : (x0 << (d - 1)) + jp;
            if (!node_valid(col, gamma - 1, xp)) continue;
            const R* pv = (d == 0 ? par : nodes + sub_off(d - 1) + jp * kSeg) + sigma * LC_M;
            R e = R(0), o = R(0);
            for (int jj = k; jj < LC_M; jj += 2) e = acc2(e, Bs[jj * LC_M + k], pv[jj]);
            for (int jj = k + 1; jj < LC_M; jj += 2) o = acc2(o, Bs[jj * LC_M + k], pv[jj]);
            e = finish(e);
            o = finish(o);
            for (int q = 0; q < 2; ++q) {
              const int64_t x = 2 * xp + q;
              if (d == 0 && x != x0) continue;
              if (!node_valid(col, gamma, x)) continue;
              R* cc = lev + (d == 0 ? 0 : 2 * jp + q) * kSeg + sigma * LC_M + k;
              *cc = *cc + (q ? e - o : e + o);
            }
          }
        }
      } else {
        for (int d = 0; d <= depth; ++d) {
          __syncthreads();
          const int gamma = rho + d;
          const int nd = 1 << d;
          R* lev = nodes + sub_off(d);
          for (int t = threadIdx.x; t < nd * kSeg; t += blockDim.x) {
            const int j = t / kSeg, sigma = (t % kSeg) / LC_M, k = t % LC_M;
            const int64_t x = (x0 << d) + j;
            R c = fuse ? (node_valid(col, gamma, x) ? Cb[(lc_seg_offset(gamma) + x) * kSeg + sigma * LC_M + k] : R(0))
                       : lev[t];  // Step 3 result (k_couple_blocks)
            if (gamma > 0 && node_valid(col, gamma, x) && node_valid(col, gamma - 1, x >> 1)) {
              const R* pv = (d == 0) ? (fuse ? Cb + (lc_seg_offset(gamma - 1) + (x >> 1)) * kSeg : par) + sigma * LC_M
                                     : nodes + sub_off(d - 1) + (j >> 1) * kSeg + sigma * LC_M;
              // B(x mod 2) (nodal: P(x mod 2)); for B, b_jk = 0 exactly for j < k:
              // all M terms, unrolled
              const R* Bp = (x & 1) ? Bs1 : Bs;
#pragma unroll
              for (int jj = 0; jj < LC_M; ++jj) c = acc2(c, Bp[jj * LC_M + k], pv[jj]);
              c = finish(c);
            }
            lev[t] = c;
          }
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
    // ---------------- Step 5 for this subtree's rows (forward) or columns (transposed)
    __syncthreads();  // the leaf level of the subtree is complete
    const R* leafc = nodes + sub_off(depth);
    const int64_t lo = (x0 << depth) * two_s;
    const int64_t hi_raw = ((x0 + 1) << depth) * two_s;
    const int64_t hi = hi_raw < a.n ? hi_raw : a.n;
    if (lo >= hi) continue;
    const bool l2c = (a.dir == LC_L2C);
    if constexpr (!fuse) {
      const bool scale = !adj && l2c;  // forward L2C: C^{-1} (far + near)
      // Item: rows m0 = 2g and m0 + 1 of parity sigma in one strip (they share
      // the leaf coefficients c), consecutive threads on consecutive strips.
      const int ng = (s + 1) >> 1;
      const int nstrips = int((hi - lo + two_s - 1) / two_s);
      const int items = nstrips * 2 * ng;
      for (int u = threadIdx.x; u < items; u += blockDim.x) {
        const int sigma = u & 1;
        const int t = (u >> 1) % nstrips;
        const int m0 = 2 * ((u >> 1) / nstrips);
        const int64_t i = lo + t * two_s + 2 * m0 + sigma;
        if (i >= hi) continue;
        const bool has1 = (m0 + 1 < s) && (i + 2 < hi);
        R far0 = R(0), far1 = R(0);
        if (node_valid(col, L - 1, (x0 << depth) + t)) {
          const R* c = leafc + t * kSeg + sigma * LC_M;
          const R* T0 = Ts + (sigma * s + m0) * LC_M;
          const R* T1 = (m0 + 1 < s) ? T0 + LC_M : T0;
#pragma unroll
          for (int k = 0; k < LC_M; ++k) {
            const R ck = c[k];
            far0 = acc2(far0, ck, T0[k]);
            far1 = acc2(far1, ck, T1[k]);
          }
          far0 = finish(far0);
          far1 = finish(far1);
        }
        if (scale) {
          far0 = cinv<R>(i) * far0;
          far1 = cinv<R>(i + 2) * far1;
        }
        // Step 7: the band's part (already in the output) + far, summed in the
        // output precision
        typedef typename lc_io<R>::type IO;
        const int e = vec_exp(a.xe, b);
        IO* o = a.out + lc_boff(b, a.ob, a.inner, a.oob) + i * a.oe;
        *o = lc_out_acc<R, IO>(*o, far0, e);
        if (has1) o[2 * a.oe] = lc_out_acc<R, IO>(o[2 * a.oe], far1, e);
      }
    } else {
      // Batched plans: Steps 5-7 here, one row (column) per step of a thread,
      // which keeps register use low enough for many CTAs per SM.
      typedef typename lc_io<R>::type IO;
      const IO* f = a.in + lc_boff(b, a.ib, a.inner, a.iob);
      const int e = vec_exp(a.xe, b);
      R* opnd = Ts + 2 * s * LC_M;  // operand tile (input values, pre-scaled)
      int64_t olo, ohi;             // operand index range
      if (!adj) {
        olo = lo;
        ohi = hi + 2 * two_s;
      } else {
        olo = lo - two_s > 0 ? lo - two_s : 0;
        ohi = hi;
      }
      if (ohi > a.n) ohi = a.n;
      const int64_t olen = ohi - olo;
      R* lamk = opnd + olen + 8;  // lambda_k (L2C) / u_k (C2L), k < 2s
      R* lamm = lamk + two_s + 8;  // lambda_m / v_m for m in [mlo, mhi)
      const int64_t mlo = adj ? (olo + lo) / 2 : lo;
      const int64_t mhi = adj ? hi : (hi + ohi) / 2 + 1;
      const int64_t mcap = mhi < a.N ? mhi : a.N;
      stage(
          int(olen), [&](int i) { return f[(olo + i) * a.ie]; },
          [&](int i, IO x) {
            const int64_t q = olo + i;
            R v = lc_ld_in<R>(&x, e);
            if (!adj) {
              if (!l2c) v = R(q) * v;  // L(i, j) = (2i+1) j u v: scale column j
            } else {
              v = l2c ? cinv<R>(q) * v : c2l_row(a, q) * v;  // C^{-1} r or (2i+2a) r
            }
            opnd[i] = v;
          });
      stage(int(two_s), [&](int k) { return k < a.N ? a.t.lam[k] : R(0); }, [&](int k, R v) { lamk[k] = v; });
      stage(
          int(mhi - mlo), [&](int j) { return mlo + j < mcap ? a.t.lam2[mlo + j] : R(0); },
          [&](int j, R v) { lamm[j] = v; });
      __syncthreads();
      // Work unit: within one strip and parity, rows m and s-1-m, whose band
      // lengths add up to about 3s, so the threads of a warp stay balanced.
      const int half = (s + 1) / 2;
      const int units = int((hi - lo + two_s - 1) / two_s) * 2 * half;
      for (int u = threadIdx.x; u < units; u += blockDim.x) {
        const int strip = u / (2 * half);
        const int rem = u - strip * 2 * half;
        const int sigma = rem / half, mm = rem % half;
        for (int rep = 0; rep < 2; ++rep) {
          const int m = rep ? s - 1 - mm : mm;
          if (rep && m == mm) break;
          const int64_t i = lo + strip * two_s + 2 * m + sigma;
          if (i >= hi) continue;
          const int64_t v = (x0 << depth) + strip;
          R far = R(0);
          if (node_valid(col, L - 1, v)) {
            const R* c = leafc + strip * kSeg + sigma * LC_M;
            const R* Trow = Ts + (sigma * s + m) * LC_M;
#pragma unroll
            for (int k = 0; k < LC_M; ++k) far = acc2(far, c[k], Trow[k]);
            far = finish(far);
          }
          R near = R(0);
          IO res;
          // Step 7 in the output precision: near + far (times C^{-1} for
          // forward L2C); C2L row/column 0 adds L(0,0) f_0 = f_0 (eq:Lxymod)
          if (!adj) {
            // row i: sum over j = i + 2k in the band  (eq:hik, eq:Lxymod)
            const int64_t end = two_s * (v + 2) < a.n ? two_s * (v + 2) : a.n;
            const int cnt = int((end - i + 1) >> 1);
            const R* fo = opnd + (i - olo);
            const R* lm = lamm + (i - mlo);
            near = band_sum<R>(cnt, [&](const R& c, int kk) { return acc3(c, lamk[kk], lm[kk], fo[2 * kk]); });
            if (l2c) {
              const R c = cinv<R>(i);
              res = lc_out2<R, IO>(c * far, c * near, e);
            } else {
              // (2i+2a) u_k v_(i+k) (j f_j) summed
              res = lc_out2<R, IO>(far, c2l_row(a, i) * near, e);
              if (i == 0) res += f[0];
            }
          } else {
            // column j = i: sum over rows r <= j in the band
            int64_t st = two_s * (v - 1) > 0 ? two_s * (v - 1) : 0;
            if ((st & 1) != (i & 1)) ++st;
            const int cnt = int((i - st) / 2 + 1);
            const R* ro = opnd + (i - olo);  // ro[-2k] = row i - 2k
            const R* lm = lamm + (i - mlo);  // lm[-k]  = (r + i)/2 = i - k
            near = band_sum<R>(cnt, [&](const R& c, int k) { return acc3(c, lamk[k], lm[-k], ro[-2 * k]); });
            res = lc_out2<R, IO>(far, l2c ? near : R(i) * near, e);
            if (!l2c && i == 0) res += f[0];
          }
          a.out[lc_boff(b, a.ob, a.inner, a.oob) + i * a.oe] = res;
        }
      }
    }
  }
}

// ------------------------------------------------- per-vector exponents
// Pre-pass of the double-float tier: xe[b] = the binary exponent of vector
// b's largest finite entry (|x| in [2^xe, 2^(xe+1))), 0 for a vector without
// nonzero finite entries.  The kernels then work on x 2^-xe.
constexpr int kExpChunk = LC_EXP_CHUNK;  // elements per CTA
constexpr int kNoExp = -(1 << 20);      // "no nonzero finite entry"
// Biased exponent of |x| as if normalised (below 1 for subnormals), or
// kNoExp for zero, infinity and NaN.
__device__ __forceinline__ int exp_field(double x) {
  const uint64_t u = __double_as_longlong(x);
  const int E = int((u >> 52) & 0x7ff);
  const uint64_t m = u & ((uint64_t(1) << 52) - 1);
  if (E == 2047) return kNoExp;
  if (E == 0) return m ? 1 - (__clzll(m) - 11) : kNoExp;
  return E;
}
__device__ __forceinline__ int block_max_256(int v, int* red) {
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int r = (threadIdx.x & 31) < 8 ? red[threadIdx.x & 31] : kNoExp;
  r = __reduce_max_sync(0xffffffffu, r);
  __syncthreads();
  return r;
}
// CTA (x, y) reduces elements [x kExpChunk, (x+1) kExpChunk) of vectors
// y, y + gridDim.y, ...; with several chunks per vector the last CTA to
// arrive (counter cnt[b], reset by that CTA) combines the partial maxima.
template <typename IO>
__global__ void __launch_bounds__(256) k_vec_exponent(const IO* __restrict__ in, int64_t n, int64_t batch, int64_t ib,
                                                      int64_t ie, int64_t inner, int64_t iob, int chunks,
                                                      int* __restrict__ xe, int* part, unsigned* cnt) {
  __shared__ int red[8];
  __shared__ int last;
  lc_grid_trigger();  // the leaf restriction may be scheduled meanwhile (it waits for this grid)
  lc_grid_wait();
  const int64_t j0 = int64_t(blockIdx.x) * kExpChunk;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const IO* f = in + lc_boff(b, ib, inner, iob);
    int m = kNoExp;
    if (ie == 1 && j0 + kExpChunk <= n && (reinterpret_cast<uintptr_t>(f + j0) & 15) == 0 && sizeof(IO) == 8) {
      // whole chunk, contiguous and 16-byte aligned: all loads issued first, 16 bytes each
      const double2* p = reinterpret_cast<const double2*>(f + j0);
      double2 v[kExpChunk / 512];
#pragma unroll
      for (int u = 0; u < kExpChunk / 512; ++u) v[u] = __ldg(p + u * 256 + threadIdx.x);
#pragma unroll
      for (int u = 0; u < kExpChunk / 512; ++u) m = max(m, max(exp_field(v[u].x), exp_field(v[u].y)));
    } else {
#pragma unroll
      for (int u = 0; u < kExpChunk / 256; ++u) {
        const int64_t j = j0 + u * 256 + threadIdx.x;
        if (j < n) m = max(m, exp_field(double(f[j * ie])));
      }
    }
    m = block_max_256(m, red);
    if (threadIdx.x == 0) {
      last = 0;
      if (chunks == 1) {
        xe[b] = m == kNoExp ? 0 : m - 1023;
      } else {
        part[b * chunks + blockIdx.x] = m;
        __threadfence();
        last = atomicAdd(&cnt[b], 1u) == unsigned(chunks - 1);
      }
    }
    __syncthreads();
    if (last) {  // every other CTA of vector b fenced its partial before arriving
      __threadfence();
      int v = kNoExp;
      for (int c = threadIdx.x; c < chunks; c += 256) v = max(v, *reinterpret_cast<volatile int*>(part + b * chunks + c));
      v = block_max_256(v, red);
      if (threadIdx.x == 0) {
        xe[b] = v == kNoExp ? 0 : v - 1023;
        cnt[b] = 0u;
      }
    }
    __syncthreads();
  }
}
// Many short strided fibres (element stride != 1): one thread per vector,
// so that a warp reads 32 neighbouring vectors' entries j together.
template <typename IO>
__global__ void __launch_bounds__(256) k_vec_exponent_rows(const IO* __restrict__ in, int64_t n, int64_t batch,
                                                           int64_t ib, int64_t ie, int64_t inner, int64_t iob,
                                                           int* __restrict__ xe) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const IO* f = in + lc_boff(b, ib, inner, iob);
  int m = kNoExp;
#pragma unroll 8
  for (int64_t j = 0; j < n; ++j) m = max(m, exp_field(double(f[j * ie])));
  xe[b] = m == kNoExp ? 0 : m - 1023;
}
inline int64_t vec_exponent_chunks(int64_t n) { return (n + kExpChunk - 1) / kExpChunk; }

template <typename R>
lc_status launch_vec_exponent(const Args<R>& a, cudaStream_t st) {
  typedef typename lc_io<R>::type IO;
  if (a.ie != 1 && a.n <= kExpChunk && a.batch >= 1024) {
    k_vec_exponent_rows<IO><<<unsigned((a.batch + 255) / 256), 256, 0, st>>>(a.in, a.n, a.batch, a.ib, a.ie, a.inner,
                                                                             a.iob, a.xe);
  } else {
    const int64_t chunks = vec_exponent_chunks(a.n);
    const dim3 grid(unsigned(chunks), unsigned(a.batch < 65535 ? a.batch : 65535));
    k_vec_exponent<IO><<<grid, 256, 0, st>>>(a.in, a.n, a.batch, a.ib, a.ie, a.inner, a.iob, int(chunks), a.xe,
                                             a.xe_part, a.xe_cnt);
  }
  LC_LAUNCH_CHECK();
  return LC_OK;
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
inline int launches_for(int L, int leaf_depth, int chunk_depth, int64_t batch) {
  if (L <= 0) return 1;
  int roots[64], nr;
  chunk_roots<R>(L, leaf_depth, chunk_depth, roots, &nr);
  return 2 * nr + (roots[0] > 0 ? 2 : 1) + (batch > 1 ? 0 : 1);  // + the band (k_near) for one vector
}

template <typename R>
lc_status set_smem(const void* fn, size_t bytes) {
  // The default limit of 48 KB covers static and dynamic shared memory together;
  // the kernels' static arrays stay below 4 KB.
  if (bytes > 44 * 1024) LC_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  return LC_OK;
}

template <typename R>
lc_status run(lc_plan_s* p, Args<R> a, cudaStream_t st, int adjoint) {
  const int L = a.L, s = a.s;
  const unsigned gy = unsigned(a.batch < 65535 ? a.batch : 65535);
  lc_timer_begin(p);
  if (L <= 0) {  // the band kernel alone (it scales its tile by its own exponent)
    const size_t sm = near_smem<R>(s, a.n, 1);
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_near<R>), sm);
    if (e != LC_OK) return e;
    lc_timer_mark(p, st, LC_K_NEAR);
    k_near<R><<<dim3(1, gy), kThreads, sm, st>>>(a, adjoint);
    LC_LAUNCH_CHECK();
    lc_timer_end(p, st);
    return LC_OK;
  }
  int roots[64], nr;
  chunk_roots<R>(L, p->leaf_depth, p->chunk_depth, roots, &nr);
  const size_t smc = couple_smem<R>(a.dir);
  {
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_couple_blocks<R>), smc);
    if (e != LC_OK) return e;
  }
  // Three independent pieces of work: the band (k_near, which needs only the
  // input), the far-field chain (leaf restriction -> coupling of the fine
  // levels -> last down chunk) and, once the first up chunk has made w final
  // on the levels [roots[0], L), the coarse levels (up chunks, their coupling,
  // their down chunks: a latency-bound chain of small grids).  For one vector
  // they run on the plan's streams -- coarse chain at the highest priority,
  // far-field chain next, band at the lowest -- so that the band's CTAs take
  // the SM slots the latency- and memory-bound far-field kernels leave free;
  // the last down chunk waits for the other two, the caller's stream for it.
  // A batch keeps the far-field chain (with the band fused into its last
  // kernel) on the caller's stream and only the coarse chain beside it.
  // Per-kernel timing keeps everything on the caller's stream, in order.
  // A batch fills the GPU from every kernel, so its band rides in the last
  // down chunk instead (one pass over the output, no separate launch).
  const bool fused = a.batch > 1;
  const bool streams = p->timing_slots <= 0 && p->fine && p->nearst && p->side;
  const bool overlap = streams && !fused;                 // band beside the far-field chain
  const bool coarse_side = streams && roots[0] > 0;       // coarse chain beside the fine coupling
  cudaStream_t sf = overlap ? p->fine : st;    // far-field chain
  cudaStream_t sn = overlap ? p->nearst : st;  // band
  cudaStream_t sk = coarse_side ? p->side : st;  // coarse chain
  // Consecutive kernels of one stream with programmatic dependent launch
  // (never in per-kernel timing mode, whose events sit between kernels).
  auto launch = [&](bool pdl, cudaStream_t stm, dim3 grid, size_t sm, auto kern, auto... args) -> lc_status {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = stm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (pdl && streams) ? 1 : 0;
    LC_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args...));
    return LC_OK;
  };
  Args<R> ac = a;  // the coarse chain's kernels let their successors start early
  ac.trigger = 1;
  if (overlap) {
    LC_CUDA_TRY(cudaEventRecord(p->ev_start, st));
    LC_CUDA_TRY(cudaStreamWaitEvent(sf, p->ev_start, 0));
    LC_CUDA_TRY(cudaStreamWaitEvent(sn, p->ev_start, 0));
  }
  if (a.xe) {  // per-vector exponents, read by the far-field chain (not by the band)
    lc_timer_mark(p, st, LC_K_PREP);
    lc_status e = launch_vec_exponent(a, sf);
    if (e != LC_OK) return e;
  }
  auto launch_band = [&]() -> lc_status {  // rows (columns) of kNearStrips strips per CTA
    const size_t sm = near_smem<R>(s, int64_t(kNearStrips) * 2 * s, 0);
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_near<R>), sm);
    if (e != LC_OK) return e;
    const int64_t strips = (a.n + 2 * s - 1) / (2 * s);
    int64_t ctas = (strips + kNearStrips - 1) / kNearStrips;
    if (p->band_ctas > 0 && p->band_ctas < ctas) ctas = p->band_ctas;
    lc_timer_mark(p, st, LC_K_NEAR);
    k_near<R><<<dim3(unsigned(ctas), gy), kThreads, sm, sn>>>(a, adjoint);
    LC_LAUNCH_CHECK();
    if (overlap) LC_CUDA_TRY(cudaEventRecord(p->ev_near, sn));
    return LC_OK;
  };
  const bool band_late = overlap && p->band_after_leaf;
  {  // first up chunk: leaf restriction and the fine levels
    const int rho = roots[0];
    const int depth = L - 1 - rho;
    const size_t sm = up_smem<R>(depth, s, 1, a.nodal);
    lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_up_chunk<R>), sm);
    if (e != LC_OK) return e;
    lc_timer_mark(p, st, LC_K_LEAF);
    e = launch(a.xe != nullptr, sf, dim3(unsigned(int64_t(4) << rho), gy), sm, k_up_chunk<R>, a, rho, depth, 1,
               adjoint);  // after the exponent pre-pass on the same stream
    if (e != LC_OK) return e;
  }
  if (!fused) {
    if (band_late) {  // the band starts once the first up chunk is done
      LC_CUDA_TRY(cudaEventRecord(p->ev_fork, sf));
      LC_CUDA_TRY(cudaStreamWaitEvent(sn, p->ev_fork, 0));
    }
    lc_status e = launch_band();
    if (e != LC_OK) return e;
  }
  if (roots[0] > 0) {
    if (coarse_side) {
      LC_CUDA_TRY(cudaEventRecord(p->ev_fork, sf));
      LC_CUDA_TRY(cudaStreamWaitEvent(sk, p->ev_fork, 0));
    }
    for (int c = 1; c < nr; ++c) {  // coarse up chunks
      const int rho = roots[c];
      const int depth = roots[c - 1] - rho;
      const size_t sm = up_smem<R>(depth, s, 0, a.nodal);
      lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_up_chunk<R>), sm);
      if (e != LC_OK) return e;
      lc_timer_mark(p, st, LC_K_UP);
      e = launch(c > 1, sk, dim3(unsigned(int64_t(4) << rho), gy), sm, k_up_chunk<R>, ac, rho, depth, 0, adjoint);
      if (e != LC_OK) return e;
    }
    lc_timer_mark(p, st, LC_K_COUPLE);  // coupling of the coarse levels
    lc_status e = launch(nr > 1, sk, dim3(unsigned(couple_ctas<R>(0, roots[0])), gy), smc, k_couple_blocks<R>, ac,
                         adjoint, 0, roots[0]);
    if (e != LC_OK) return e;
    for (int c = nr - 1; c >= 1; --c) {  // coarse down chunks: levels [roots[c], roots[c-1] - 1]
      const int rho = roots[c];
      const int depth = roots[c - 1] - 1 - rho;
      const size_t sm = down_smem<R>(depth, s, 0);
      lc_status e = set_smem<R>(reinterpret_cast<const void*>(k_down_chunk<R, false>), sm);
      if (e != LC_OK) return e;
      lc_timer_mark(p, st, LC_K_DOWN);
      e = launch(true, sk, dim3(unsigned(int64_t(4) << rho), gy), sm, k_down_chunk<R, false>, ac, rho, depth, 0,
                 adjoint);
      if (e != LC_OK) return e;
    }
    if (coarse_side) LC_CUDA_TRY(cudaEventRecord(p->ev_join, sk));
  }
  // coupling of the fine levels [roots[0], L)
  lc_timer_mark(p, st, LC_K_COUPLE);
  k_couple_blocks<R><<<dim3(unsigned(couple_ctas<R>(roots[0], L)), gy), kThreads, smc, sf>>>(a, adjoint, roots[0], L);
  LC_LAUNCH_CHECK();
  if (coarse_side) LC_CUDA_TRY(cudaStreamWaitEvent(sf, p->ev_join, 0));
  if (overlap) LC_CUDA_TRY(cudaStreamWaitEvent(sf, p->ev_near, 0));
  {  // last down chunk: fine levels, then Step 5 plus the band's part
    const int rho = roots[0];
    const int depth = L - 1 - rho;
    size_t sm = down_smem<R>(depth, s, 1);
    if (fused) {  // operand, lambda_k and lambda_m tiles of the band
      const size_t rows = (size_t(1) << depth) * 2 * s;
      sm += ((rows + 4 * size_t(s) + 8) + (2 * size_t(s) + 8) + (rows + 2 * size_t(s) + 8)) * sizeof(R);
    }
    const void* fn = fused ? reinterpret_cast<const void*>(k_down_chunk<R, true>)
                           : reinterpret_cast<const void*>(k_down_chunk<R, false>);
    lc_status e = set_smem<R>(fn, sm);
    if (e != LC_OK) return e;
    lc_timer_mark(p, st, LC_K_FINAL);
    const dim3 grid(unsigned(int64_t(4) << rho), gy);
    if (fused) k_down_chunk<R, true><<<grid, kThreads, sm, sf>>>(a, rho, depth, 1, adjoint);
    else k_down_chunk<R, false><<<grid, kThreads, sm, sf>>>(a, rho, depth, 1, adjoint);
    LC_LAUNCH_CHECK();
  }
  if (overlap) {
    LC_CUDA_TRY(cudaEventRecord(p->ev_done, sf));
    LC_CUDA_TRY(cudaStreamWaitEvent(st, p->ev_done, 0));
  }
  lc_timer_end(p, st);
  return LC_OK;
}

}  // namespace lc_exec
