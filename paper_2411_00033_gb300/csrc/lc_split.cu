// lc_split.cu -- split-precision tensor-core tier (LC_F64_SPLIT) for batches.
//
// When many vectors share one plan, every step of Algorithm 4 becomes a
// matrix product whose left operand holds one row per vector:
//   leaf    W(g)      = F(g) T(sigma)                  (Step 1, eq:wMM)
//   up      W(G)      = [W(2G) W(2G+1)] [B(0) B(1)]^T   (Step 2, eq:wtk)
//   couple  C(v)      = [W(v+2) W(v+3)] [A-hat A-hat]^T (Step 3)
//   down    C(v)     += C(v/2) B(v mod 2)              (Step 4)
//   final   Z(strip)  = C(v) T(sigma)^T + F(strip) E^T (Steps 5-6), then C^{-1} (Step 7)
// (E = the near-field block of the strip.)  Each product runs on the
// tensor cores (tcgen05.mma kind::f16, M = 128 members, N = 32, K = 16,
// bf16 operands from shared memory, FP32 accumulators in TMEM) as an exact
// multi-word product: every operand row/column is scaled by a power of two
// and cut into S signed 8-bit slices (|q| <= 128, exact in bf16), so each
// slice product is an exact integer below 2^14 and every FP32 partial sum
// over K <= 64 terms and <= S slice pairs stays below 2^24 -- exact.  The
// slice pairs (s, t) with s + t <= S + 1 are accumulated per diagonal
// u = s + t and recombined by a Horner sum in base 2^8 in double-float
// (pairs of FP32).  Shared matrices are sliced once at plan time (FP64).
//
// Per-vector intermediates are stored as "block floating" double-float rows:
// 18 (hi, lo) pairs scaled into [-1/2, 1/2] plus one power-of-two exponent
// per row, so the next product slices them without another scan.  Step 7
// (near + far, times C^{-1} for L2C) runs in FP64 on each output.
//
// Transposed pass (lc_adjoint): the same products in reverse roles --
//   leaf    W'(0, v)  = R(v) T(sigma)                  (row strip v: spread^T)
//   up      W'(d+1,V) = [W'(d, 2V) W'(d, 2V+1)] [B(0) B(1)]^T   (Step 4^T)
//   couple  C'(d, g)  = [W'(d, g-2) W'(d, g-3)] [A-hat(b,2) A-hat(b,1)] (g odd),
//                       W'(d, g-2) A-hat(b,0) (g even)  (Step 3^T)
//   down    C'(d, g) += C'(d+1, g/2) B(g mod 2)         (Step 2^T)
//   final   F'(strip) = C'(0, t) T(sigma)^T + R(strips t-1, t) E'^T (Step 1^T, band^T)
// with R = C^{-1} r for L2C (applied while the input is sliced).  A row
// segment v is owned by the same members as column segment v + 2, so every
// row array keeps its slot numbering.
//
// Batches: members are sorted by length (descending).  At every level the
// members owning a segment form a prefix of that order, so each task takes
// one (segment, parity, 128-member tile).  A uniform batch is the special
// case of equal lengths; a ragged batch shares one coefficient table built
// for its longest member with a fixed s (A-hat depends only on the position
// of a submatrix in A, eq:globalij).
//
// Schedules: one kernel launch per level (a CTA per task), or Steps 1-4 in
// one persistent launch whose CTAs draw the tasks in a list-scheduled order
// and wait only for the row blocks each task reads (k_s_persist), followed
// by the final launch.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <utility>
#include <vector>

#include "lc_internal.cuh"
#include "lc_tma.cuh"
#include "lc_umma.cuh"

namespace {

constexpr int kRows = 128;      // members per CTA tile: the MMA's M (one TMEM lane per member)
constexpr int kThreads = 256;   // 8 warps; warp w reads TMEM lanes 32 (w % 4) .. + 31
constexpr int kNP = 32;         // outputs per product (18, or s <= 32) padded to the MMA's N
constexpr int kCols = kNP / 2;  // accumulator columns per thread (two threads per member row)
constexpr int kTmemCols = 256;  // S <= 7 diagonals x kNP columns, rounded up to a power of two
constexpr int kXCols = 32;      // per-vector operand columns staged at a time
// dynamic shared memory of the leaf and final stages beyond their operands:
// per-row input/output bases and lengths ([3][kRows] int64)
constexpr size_t kRowBytes = size_t(3) * kRows * 8;

enum YKind {
  Y_LEAF = 0, Y_SPREAD = 1, Y_UP = 2, Y_DOWN = 3, Y_COUPLE = 4, Y_NEAR = 5,
  Y_COUPLE_T = 6,  // transposed pass: A-hat blocks per column segment
  Y_NEAR_T = 7,    // transposed pass: band entries per column strip
  Y_KINDS = 8
};

struct YTable {
  int items, K, KP;     // KP: K rounded up to 16 (at least 32)
  size_t off_q, off_e;  // byte offsets in the split region: bf16 [items][S][kNP x KP canonical], int32 [items][kNP]
};

struct Work {
  int32_t d, seg, tile;
};

// One task of the persistent schedule: a work item (kind, level d, segment
// or strip, member tile) and its dependencies.  rd[i] names the row block
// the task reads (a counter slot; 2 rd[i] + sigma is the counter of parity
// sigma) and need[i] how many writes of that block must be complete first;
// wr is the slot of the block it writes (-1: none).
struct PTask {
  int32_t kind, d, seg, tile;
  int32_t rd[2], need[2];
  int32_t wr;
};

struct SplitHost {
  int S, s, Lmax;
  int64_t count, Nmax, nstrips;
  std::vector<int64_t> len_sorted, orig, off_sorted;  // sorted order
  std::vector<int32_t> Lm;
  std::vector<int64_t> Lcount;                        // [Lmax + 2]
  std::vector<int64_t> cntN;                          // [nstrips]
  std::vector<int64_t> rowbase;                       // concatenated over d
  int64_t rows;
  YTable y[Y_KINDS];
  // work lists: launches in execution order (forward; a* = transposed pass)
  std::vector<Work> work, awork;
  std::vector<int64_t> launch_off, alaunch_off;  // [launches + 1]
  std::vector<int> launch_kind, alaunch_kind;    // LC_K_*
  std::vector<int> launch_level;                 // d for up/down
  // persistent schedule (one launch): task lists with their dependencies
  std::vector<PTask> ptask, aptask;
  bool persist;  // both lists were built and checked
  // device byte offsets
  size_t off_len, off_orig, off_off, off_Lcount, off_cntN, off_rowbase, off_work, off_awork;
  size_t off_ptask, off_aptask, off_sched;  // off_sched: ticket counter, abort word, block counters
  size_t off_W, off_We, off_C, off_Ce;
  size_t total;
};

// cnt(d, g): members owning segment g at relative level d (levels counted
// from the leaves), given Lcount[l] = #members with L_m >= l.
inline int64_t seg_threshold(int d, int64_t g) {
  int lg = 0;
  while ((int64_t(2) << lg) <= g) ++lg;  // floor(log2 g) for g >= 1
  if (g < 1) lg = 0;
  return d + (lg > 1 ? lg : 1);
}

int member_levels(int64_t n, int s) {
  if (n <= 4 * int64_t(s)) return 0;
  int t = 0;
  while ((int64_t(s) << t) < n) ++t;
  return t - 2;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The persistent schedule of one pass (Steps 1-4).  The data flow comes
// from the level launches, whose order is the reference: every work item
// with the row blocks (array W or C, level, segment, member tile) it reads
// and writes, as the stage bodies do; a read needs every write of the block
// by items before it in that order.  A block's counter slot is the index of
// its first writer.  The ticket order is a list schedule of that graph on
// `workers` CTAs with unit task times: round by round, the ready items with
// the longest chain of dependants ahead of them first -- the coarse levels
// of Steps 2 and 4 form the long chain, the wide levels fill the CTAs around
// it.  Returns false -- the plan then keeps the level-by-level launches --
// if a read finds no earlier writer, or if a block could be rewritten
// before a reader that needs its earlier value has read it (only a
// read-modify-write by the writer itself is allowed).
bool build_ptasks(bool adj, int Lmax, const std::vector<Work>& work, const std::vector<int64_t>& loff,
                  const std::vector<int>& lkind, int workers, std::vector<PTask>& out) {
  out.clear();
  if (Lmax <= 0) return true;  // no levels: only the final stage
  // row blocks in flat arrays: (array W or C, level d, segment g, member tile)
  int32_t ntiles = 1;
  for (const Work& w : work) ntiles = std::max(ntiles, w.tile + 1);
  const int64_t nsegtot = (int64_t(4) << Lmax) - 4;  // sum over d < Lmax of 2^(Lmax+1-d)
  const int64_t nblk = 2 * nsegtot * ntiles;
  if (nblk >= (int64_t(1) << 31)) return false;
  auto block = [&](int arr, int d, int64_t g, int32_t tile) -> int64_t {
    if (d < 0 || d >= Lmax || g < 0 || g >= (int64_t(2) << (Lmax - d))) return -1;
    const int64_t seg = (int64_t(4) << Lmax) - (int64_t(4) << (Lmax - d)) + g;
    return (int64_t(arr) * nsegtot + seg) * ntiles + tile;
  };
  std::vector<int32_t> slot(size_t(nblk), -1), nw(size_t(nblk), 0), last(size_t(nblk), -1);
  std::vector<PTask> items;
  std::vector<std::array<int32_t, 2>> pred;
  std::vector<int64_t> wblk_of;                               // block each item writes
  std::vector<std::array<int64_t, 3>> reads_all;              // (item, block, need)
  items.reserve(work.size());
  pred.reserve(work.size());
  wblk_of.reserve(work.size());
  reads_all.reserve(2 * work.size());
  for (size_t l = 0; l < lkind.size(); ++l) {
    const int kind = lkind[l];
    if (kind == LC_K_FINAL) continue;  // the final stage is a launch of its own
    for (int64_t w = loff[l]; w < loff[l + 1]; ++w) {
      const Work& it = work[w];
      const int32_t me = int32_t(items.size());
      PTask t{kind, it.d, it.seg, it.tile, {-1, -1}, {0, 0}, -1};
      std::array<int32_t, 2> pr{-1, -1};
      const int64_t v = it.seg;
      int64_t rb[2] = {-2, -2};  // -2: no read
      int64_t wb = -1;
      switch (kind) {
        case LC_K_LEAF: wb = block(0, 0, v, it.tile); break;
        case LC_K_UP:
          rb[0] = block(0, it.d - 1, 2 * v, it.tile);
          rb[1] = block(0, it.d - 1, 2 * v + 1, it.tile);
          wb = block(0, it.d, v, it.tile);
          break;
        case LC_K_COUPLE:
          if (adj) {
            rb[0] = block(0, it.d, v - 2, it.tile);
            if (v & 1) rb[1] = block(0, it.d, v - 3, it.tile);
          } else {
            rb[0] = block(0, it.d, v + 2, it.tile);
            if ((v & 1) == 0) rb[1] = block(0, it.d, v + 3, it.tile);
          }
          wb = block(1, it.d, v, it.tile);
          break;
        case LC_K_DOWN:
          rb[0] = block(1, it.d + 1, v >> 1, it.tile);
          rb[1] = block(1, it.d, v, it.tile);
          wb = block(1, it.d, v, it.tile);
          break;
        default:
          return false;
      }
      int32_t own_need = -1;  // the need of this item's read of the block it writes
      for (int i = 0; i < 2; ++i) {
        if (rb[i] == -2) continue;
        if (rb[i] < 0 || nw[size_t(rb[i])] == 0) return false;  // no earlier writer
        const size_t b = size_t(rb[i]);
        t.rd[i] = slot[b];
        t.need[i] = nw[b];
        pr[i] = last[b];
        reads_all.push_back({me, rb[i], nw[b]});
        if (rb[i] == wb) own_need = nw[b];
      }
      if (wb < 0) return false;
      const size_t b = size_t(wb);
      if (nw[b] == 0) slot[b] = me;
      else if (own_need != nw[b]) return false;  // a rewrite must read the write before it
      ++nw[b];
      last[b] = me;
      t.wr = slot[b];
      items.push_back(t);
      pred.push_back(pr);
      wblk_of.push_back(wb);
    }
  }
  // a read that needs fewer writes than its block gets must be the next
  // writer's own read-modify-write
  for (const auto& r : reads_all)
    if (r[2] < nw[size_t(r[1])] && wblk_of[size_t(r[0])] != r[1]) return false;
  const int32_t n = int32_t(items.size());
  if (size_t(n) >= (size_t(1) << 29)) return false;
  // dependants (CSR), and the longest chain from each item (level order is topological)
  std::vector<int32_t> indeg(size_t(n), 0), rank(size_t(n), 1), sfirst(size_t(n) + 1, 0);
  auto for_preds = [&](int32_t i, auto&& f) {
    const int32_t q0 = pred[size_t(i)][0], q1 = pred[size_t(i)][1];
    if (q0 >= 0) f(q0);
    if (q1 >= 0 && q1 != q0) f(q1);
  };
  for (int32_t i = 0; i < n; ++i) for_preds(i, [&](int32_t q) { ++sfirst[size_t(q) + 1]; });
  for (int32_t i = 0; i < n; ++i) sfirst[size_t(i) + 1] += sfirst[size_t(i)];
  const size_t nsucc = size_t(sfirst[size_t(n)]);
  std::vector<int32_t> succ(nsucc);
  std::vector<int32_t> fill(sfirst.begin(), sfirst.end() - 1);
  for (int32_t i = 0; i < n; ++i)
    for_preds(i, [&](int32_t q) {
      succ[size_t(fill[size_t(q)]++)] = i;
      ++indeg[size_t(i)];
    });
  for (int32_t i = n - 1; i >= 0; --i)
    for (int32_t k = sfirst[size_t(i)]; k < sfirst[size_t(i) + 1]; ++k)
      rank[size_t(i)] = std::max(rank[size_t(i)], rank[size_t(succ[size_t(k)])] + 1);
  // the list schedule: two tickets (parities) per item; ready items in
  // buckets by chain length (first come, first served within a bucket)
  const size_t cap = size_t(std::max(1, workers / 2));
  int32_t maxrank = 0;
  for (int32_t r : rank) maxrank = std::max(maxrank, r);
  std::vector<std::vector<int32_t>> bucket(size_t(maxrank) + 1);
  std::vector<size_t> head(size_t(maxrank) + 1, 0);
  int32_t top = 0;  // highest bucket that may hold ready items
  auto push = [&](int32_t i) {
    bucket[size_t(rank[size_t(i)])].push_back(i);
    top = std::max(top, rank[size_t(i)]);
  };
  for (int32_t i = 0; i < n; ++i)
    if (indeg[size_t(i)] == 0) push(i);
  std::vector<int32_t> round, next;
  out.reserve(size_t(n));
  for (;;) {
    round.clear();
    while (round.size() < cap && top > 0) {
      const size_t r = size_t(top);
      if (head[r] < bucket[r].size()) round.push_back(bucket[r][head[r]++]);
      else --top;
    }
    if (round.empty()) break;
    for (int32_t i : round) {
      out.push_back(items[size_t(i)]);
      for (int32_t k = sfirst[size_t(i)]; k < sfirst[size_t(i) + 1]; ++k)
        if (--indeg[size_t(succ[size_t(k)])] == 0) next.push_back(succ[size_t(k)]);
    }
    for (int32_t j : next) push(j);
    next.clear();
  }
  return out.size() == size_t(n);
}

// Build all host tables and the byte layout of the split region.
// `workers`: CTAs of the persistent launch (its ticket order is scheduled
// for them; the layout does not depend on it).
// Items of Steps 1-4 in a work list (the tasks of the persistent schedule).
size_t stage_items(const std::vector<int64_t>& loff, const std::vector<int>& lkind) {
  size_t c = 0;
  for (size_t l = 0; l < lkind.size(); ++l)
    if (lkind[l] != LC_K_FINAL) c += size_t(loff[l + 1] - loff[l]);
  return c;
}

// schedule = false builds only what the byte layout needs (no task graph).
void build_host(const lc_plan_s* p, SplitHost& h, int workers, bool schedule) {
  h.S = p->opt.slices;
  h.s = p->g.s;
  h.Lmax = p->g.L;
  h.Nmax = p->g.N;
  h.count = p->count;
  std::vector<int64_t> len(h.count), off(h.count);
  int64_t acc = 0;
  for (int64_t m = 0; m < h.count; ++m) {
    len[m] = p->ragged ? p->h_len[m] : p->g.n;
    off[m] = acc;
    acc += len[m];
  }
  std::vector<int64_t> order(h.count);
  for (int64_t m = 0; m < h.count; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return len[a] > len[b]; });
  h.len_sorted.resize(h.count);
  h.orig.resize(h.count);
  h.off_sorted.resize(h.count);
  h.Lm.resize(h.count);
  for (int64_t r = 0; r < h.count; ++r) {
    h.orig[r] = order[r];
    h.len_sorted[r] = len[order[r]];
    h.off_sorted[r] = off[order[r]];
    h.Lm[r] = (h.Lmax > 0) ? member_levels(h.len_sorted[r], h.s) : 0;
  }
  h.Lcount.assign(h.Lmax + 2, 0);
  for (int64_t r = 0; r < h.count; ++r)
    for (int l = 0; l <= h.Lm[r] && l < h.Lmax + 2; ++l) h.Lcount[l]++;
  auto cnt = [&](int d, int64_t g) -> int64_t {
    const int64_t th = seg_threshold(d, g);
    return th < int64_t(h.Lcount.size()) ? h.Lcount[th] : 0;
  };
  h.nstrips = (h.Nmax + 2 * h.s - 1) / (2 * h.s);
  h.cntN.assign(h.nstrips, 0);
  {  // members longer than 2 s t: a prefix of the descending order, shrinking with t
    int64_t c = h.count;
    for (int64_t t = 0; t < h.nstrips; ++t) {
      while (c > 0 && h.len_sorted[c - 1] <= 2 * int64_t(h.s) * t) --c;
      h.cntN[t] = c;
    }
  }
  // row bases: per d, per g < 2^(Lmax+1-d): 2 x cnt(d, g) rows (sigma-major)
  h.rowbase.clear();
  h.rows = 0;
  for (int d = 0; d < h.Lmax; ++d) {
    const int64_t nseg = int64_t(1) << (h.Lmax + 1 - d);
    for (int64_t g = 0; g < nseg; ++g) {
      h.rowbase.push_back(h.rows);
      h.rows += 2 * cnt(d, g);
    }
  }
  if (h.rowbase.empty()) h.rowbase.push_back(0);
  // work lists
  h.work.clear();
  h.launch_off.assign(1, 0);
  h.launch_kind.clear();
  h.launch_level.clear();
  auto add_items = [&](int d, int64_t seg, int64_t members) {
    for (int64_t t0 = 0; t0 < members; t0 += kRows) h.work.push_back(Work{d, int32_t(seg), int32_t(t0 / kRows)});
  };
  auto close_launch = [&](int kind, int level) {
    h.launch_off.push_back(int64_t(h.work.size()));
    h.launch_kind.push_back(kind);
    h.launch_level.push_back(level);
  };
  if (h.Lmax > 0) {
    for (int64_t g = 2; g < (int64_t(2) << h.Lmax); ++g) add_items(0, g, cnt(0, g));
    close_launch(LC_K_LEAF, 0);
    for (int d = 0; d + 1 < h.Lmax; ++d) {  // parents at d+1
      for (int64_t G = 2; G < (int64_t(1) << (h.Lmax - d)); ++G) add_items(d + 1, G, cnt(d + 1, G));
      close_launch(LC_K_UP, d);
    }
    for (int d = 0; d < h.Lmax; ++d)
      for (int64_t v = 0; v + 2 < (int64_t(1) << (h.Lmax + 1 - d)); ++v) add_items(d, v, cnt(d, v + 2));
    close_launch(LC_K_COUPLE, 0);
    for (int d = h.Lmax - 2; d >= 0; --d) {  // children at d
      for (int64_t v = 0; v + 4 < (int64_t(1) << (h.Lmax + 1 - d)); ++v) add_items(d, v, cnt(d, v + 4));
      close_launch(LC_K_DOWN, d);
    }
  }
  for (int64_t t = 0; t < h.nstrips; ++t) add_items(0, t, h.cntN[t]);
  close_launch(LC_K_FINAL, 0);
  // transposed pass: row tree up, coupling per column segment, column tree down
  h.awork.clear();
  h.alaunch_off.assign(1, 0);
  h.alaunch_kind.clear();
  auto aadd = [&](int d, int64_t seg, int64_t members) {
    for (int64_t t0 = 0; t0 < members; t0 += kRows) h.awork.push_back(Work{d, int32_t(seg), int32_t(t0 / kRows)});
  };
  auto aclose = [&](int kind) {
    h.alaunch_off.push_back(int64_t(h.awork.size()));
    h.alaunch_kind.push_back(kind);
  };
  if (h.Lmax > 0) {
    for (int64_t v = 0; v + 2 < (int64_t(2) << h.Lmax); ++v) aadd(0, v, cnt(0, v + 2));
    aclose(LC_K_LEAF);
    for (int d = 0; d + 1 < h.Lmax; ++d) {  // parents at d+1
      for (int64_t V = 0; V + 2 < (int64_t(1) << (h.Lmax - d)); ++V) aadd(d + 1, V, cnt(d + 1, V + 2));
      aclose(LC_K_UP);
    }
    for (int d = 0; d < h.Lmax; ++d)
      for (int64_t g = 2; g < (int64_t(1) << (h.Lmax + 1 - d)); ++g) aadd(d, g, cnt(d, g));
    aclose(LC_K_COUPLE);
    for (int d = h.Lmax - 2; d >= 0; --d) {  // children at d
      for (int64_t g = 4; g < (int64_t(1) << (h.Lmax + 1 - d)); ++g) aadd(d, g, cnt(d, g));
      aclose(LC_K_DOWN);
    }
  }
  for (int64_t t = 0; t < h.nstrips; ++t) aadd(0, t, h.cntN[t]);
  aclose(LC_K_FINAL);
  h.persist = schedule && build_ptasks(false, h.Lmax, h.work, h.launch_off, h.launch_kind, workers, h.ptask) &&
              build_ptasks(true, h.Lmax, h.awork, h.alaunch_off, h.alaunch_kind, workers, h.aptask);
  const size_t nfwd = stage_items(h.launch_off, h.launch_kind), nadj = stage_items(h.alaunch_off, h.alaunch_kind);

  // Y tables
  const int s = h.s;
  auto ktab = [&](YKind k, int items, int K) {
    h.y[k].items = items;
    h.y[k].K = K;
    h.y[k].KP = std::max(32, (K + 15) / 16 * 16);
  };
  int64_t nrowseg = 0;
  for (int G = 0; G < h.Lmax; ++G) nrowseg += (int64_t(4) << G) - 2;
  ktab(Y_LEAF, 2, s);
  ktab(Y_SPREAD, 2, LC_M);
  ktab(Y_UP, 1, 2 * LC_M);
  ktab(Y_DOWN, 2, LC_M);
  ktab(Y_COUPLE, int(nrowseg), 2 * LC_M);
  ktab(Y_NEAR, int(2 * h.nstrips), 2 * s);
  ktab(Y_COUPLE_T, int(nrowseg), 2 * LC_M);
  ktab(Y_NEAR_T, int(2 * h.nstrips), 2 * s);

  size_t o = 0;
  auto take = [&](size_t bytes) {
    o = align256(o);
    size_t r = o;
    o += bytes;
    return r;
  };
  for (int k = 0; k < Y_KINDS; ++k) {
    YTable& y = h.y[k];
    y.off_q = take(size_t(y.items) * h.S * kNP * y.KP * 2);  // laid out as in shared memory
    y.off_e = take(size_t(y.items) * kNP * 4);
  }
  h.off_len = take(size_t(h.count) * 8);
  h.off_orig = take(size_t(h.count) * 8);
  h.off_off = take(size_t(h.count) * 8);
  h.off_Lcount = take(h.Lcount.size() * 8);
  h.off_cntN = take(size_t(h.nstrips) * 8);
  h.off_rowbase = take(h.rowbase.size() * 8);
  h.off_work = take(h.work.size() * sizeof(Work));
  h.off_awork = take(h.awork.size() * sizeof(Work));
  h.off_ptask = take(nfwd * sizeof(PTask));
  h.off_aptask = take(nadj * sizeof(PTask));
  h.off_sched = take((4 + 2 * std::max(nfwd, nadj)) * sizeof(int));
  h.off_W = take(size_t(h.rows) * LC_M * 8);
  h.off_We = take(size_t(h.rows) * 4);
  h.off_C = take(size_t(h.rows) * LC_M * 8);
  h.off_Ce = take(size_t(h.rows) * 4);
  h.total = align256(o) + 256;
}

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ float pow2f(int k) {
  return (k < -126) ? 0.0f : (k > 127 ? __int_as_float(0x7f800000) : __uint_as_float(uint32_t(k + 127) << 23));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Exponent k of a positive normal float v with v in [2^(k-1), 2^k).
__device__ __forceinline__ int exp_of(float v) { return int((__float_as_uint(v) >> 23) & 0xff) - 126; }

// Biased exponent of |x| as if normalised (below 1 for subnormals); kNoExp
// for zero, infinity and NaN.
constexpr int kNoExp = -(1 << 20);
__device__ __forceinline__ int exp_field(double x) {
  const uint64_t u = __double_as_longlong(x);
  const int E = int((u >> 52) & 0x7ff);
  const uint64_t m = u & ((uint64_t(1) << 52) - 1);
  if (E == 2047) return kNoExp;
  if (E == 0) return m ? 1 - (__clzll(m) - 11) : kNoExp;
  return E;
}

// x * 2^-e_row as a double-float, built from the bit pattern (no FP64 op).
// Subnormal doubles are normalised first; results below 2^-126 (far below
// the row's largest entry, whose exponent e_row is) are flushed to zero.
__device__ __forceinline__ void d2df_scaled(double x, int e_row, float& hi, float& lo) {
  const uint64_t u = __double_as_longlong(x);
  int E = int((u >> 52) & 0x7ff);
  uint64_t m = u & ((uint64_t(1) << 52) - 1);
  if (E == 0) {
    if (m == 0) {
      hi = lo = 0.0f;
      return;
    }
    const int sh = __clzll(m) - 11;
    m <<= sh;
    E = 1 - sh;
  } else {
    m |= uint64_t(1) << 52;
  }
  const int k = E - 1075 - e_row;  // value = m * 2^k
  const uint32_t mh = uint32_t(m >> 29);
  const uint32_t ml = uint32_t(m & 0x1fffffffu);
  const int eh = k + 29 + 23 + 127;
  const uint32_t sgn = uint32_t(u >> 63) << 31;
  hi = (eh >= 1 && eh <= 254) ? __uint_as_float(sgn | (uint32_t(eh) << 23) | (mh & 0x7fffffu)) : 0.0f;
  float l = __uint2float_rn(ml) * pow2f(k);
  lo = (sgn ? -l : l);
  if (eh < 1) lo = 0.0f;
}

// f * 2^E as a double: from the bit pattern (exact) when the result is a
// normal FP64 number, else by a correctly rounded FP64 scaling.
__device__ __forceinline__ double f2d_scaled(float f, int E) {
  const uint32_t u = __float_as_uint(f);
  const int ef = int((u >> 23) & 0xff);
  if (ef == 0) return 0.0;
  const int64_t ed = int64_t(ef) - 127 + 1023 + E;
  const uint64_t sgn = uint64_t(u >> 31) << 63;
  if (ed >= 1 && ed <= 2046) return __longlong_as_double(sgn | (uint64_t(ed) << 52) | (uint64_t(u & 0x7fffffu) << 29));
  if (E < -2200) return 0.0;
  return ldexp(double(f), E > 2200 ? 2200 : E);
}

__device__ __forceinline__ uint16_t bf16_of_int(float q) { return uint16_t(__float_as_uint(q) >> 16); }

// Cut a normalised double-float x = hi + lo (|x| <= 1/2, |lo| <= ulp(hi)) into
// S base-2^8 digits q_1..q_S (rounded to nearest at each step):
// x = sum_s q_s 2^(-8 s) + r, |r| <= 2^(-8S-1); q[s] = bf16(q_(s+1)).
// The first two digits come from hi alone (its 24 bits are exact under the
// 8-bit shifts), lo joins once through TwoSum, and after the third digit the
// residual fits one float.  Digits stay within [-129, 129].
__device__ __forceinline__ void slice_digits(float hi, float lo, int S, uint16_t (&q)[7]) {
  float r = hi;
#pragma unroll
  for (int sl = 0; sl < 2; ++sl) {
    const float t = r * 256.0f;
    const float d = rintf(t);
    r = t - d;
    q[sl] = bf16_of_int(d);
  }
  float rh, rl;
  two_sum(r, lo * 65536.0f, rh, rl);  // residual after two digits, lo brought to the same scale
  {
    const float th = rh * 256.0f, tl = rl * 256.0f;
    const float d = rintf(th);
    r = (th - d) + tl;  // the rest fits one float
    q[2] = bf16_of_int(d);
  }
#pragma unroll
  for (int sl = 3; sl < 7; ++sl) {
    const float t = r * 256.0f;
    const float d = rintf(t);
    r = t - d;
    q[sl] = sl < S ? bf16_of_int(d) : uint16_t(0);
  }
}

// Slice the 8 double-floats hi[j] + lo[j], columns 8 ch .. 8 ch + 7 of tile
// row rr, into the S planes of an operand in the canonical K-major layout of
// lc_umma.cuh (Kp columns per row, plane_bytes apart): one 16-byte store per
// plane.  Threads that take consecutive rows at the same ch write one
// contiguous 128-byte core-matrix row group, free of bank conflicts.
__device__ __forceinline__ void put_chunk(unsigned char* X, int plane_bytes, int Kp, int rr, int ch, int S,
                                          const float (&hi)[8], const float (&lo)[8]) {
  uint32_t w[7][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    uint16_t q[7];
    slice_digits(hi[j], lo[j], S, q);
#pragma unroll
    for (int sl = 0; sl < 7; ++sl) {
      if (j & 1) w[sl][j >> 1] |= uint32_t(q[sl]) << 16;
      else w[sl][j >> 1] = q[sl];
    }
  }
  const uint32_t off = umma_offset(rr, 8 * ch, Kp);
#pragma unroll
  for (int sl = 0; sl < 7; ++sl)
    if (sl < S) *reinterpret_cast<uint4*>(X + sl * plane_bytes + off) = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
}

// Bring the Y slices of one table item (S planes of kNP x KP bf16 in the
// canonical layout) and its kNP exponents into shared memory with two bulk
// copies: y_issue starts them (thread 0), y_wait waits for them (all
// threads).  The mbarrier's phases run on across the loads of a CTA (`count`
// loads waited for so far).  Between the two the CTA stages its own operand.
// y_wait returns false if the bounded wait ran out; thread 0 then waits once
// more (bounded) so that a late copy lands before the CTA moves on, and the
// caller records the failure.
__device__ __forceinline__ void y_issue(const uint16_t* __restrict__ q, const int* __restrict__ e, int S, int KP,
                                        unsigned char* Ys, int* Ye, uint64_t* mbar) {
  const uint32_t mb = lc_smem_u32(mbar);
  const uint32_t bq = uint32_t(S) * kNP * KP * 2, be = uint32_t(kNP) * 4;
  if (threadIdx.x == 0) {
    lc_fence_proxy_async();
    lc_mbar_expect(mb, bq + be);
    lc_bulk_g2s(Ys, q, bq, mb);
    lc_bulk_g2s(Ye, e, be, mb);
  }
}
__device__ __forceinline__ bool y_wait(uint64_t* mbar, uint32_t& count) {
  const uint32_t mb = lc_smem_u32(mbar);
  const uint32_t phase = count & 1u;
  ++count;
  const bool ok = lc_mbar_wait_bounded(mb, phase);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) lc_mbar_wait_bounded(mb, phase);
    return false;
  }
  return true;
}

struct Dev {
  int S, s, Lmax;
  int64_t count, Nmax, nstrips;
  const int64_t* len;
  const int64_t* orig;
  const int64_t* off;
  const int64_t* Lcount;
  const int64_t* cntN;
  const int64_t* rowbase;
  const Work* work;
  float2* W;
  int* We;
  float2* C;
  int* Ce;
  const uint16_t* yq[Y_KINDS];
  const int* ye[Y_KINDS];
  int yKP[Y_KINDS];
  int dir;
  int ragged;
  int adj;  // transposed pass
  int* err;
  // persistent schedule: per-block write counters, the ticket counter and the
  // abort word of one execution (zeroed before the launch)
  int* cnt;
  unsigned* head;
  int* abort;
  // I/O
  const double* in;
  double* out;
  int64_t ib, ie, ob, oe;
  int64_t inner, iob, oob;  // two-level batches (lc_layout)
};

// Lcount in shared memory, loaded by every stage kernel at its start
// (ctx_begin): the member counts every task looks up first.
constexpr int kMaxLcount = 64;
__shared__ int64_t s_lcount[kMaxLcount];
__device__ __forceinline__ int64_t dcnt(const Dev& D, int d, int64_t g) {
  const int lg = g >= 2 ? 63 - __clzll(g) : 0;  // floor(log2 g)
  const int th = d + (lg > 1 ? lg : 1);
  return th <= D.Lmax + 1 ? s_lcount[th] : 0;
}
__device__ __forceinline__ int64_t drow(const Dev& D, int d, int64_t g, int sigma, int64_t r) {
  const int64_t db = (int64_t(4) << D.Lmax) - (int64_t(4) << (D.Lmax - d));  // sum_{d'<d} 2^(Lmax+1-d')
  return D.rowbase[db + g] + sigma * dcnt(D, d, g) + r;
}

// Shared memory of the stage kernels: the per-vector operand X (S planes of
// kRows x KPx, staged kXCols columns at a time at most), the shared operand
// Y (S planes of kNP x KP), and small per-row / per-column arrays.
struct Smem {
  unsigned char* X;
  unsigned char* Y;
  int xplane, yplane;  // bytes per slice plane
  int KPx, KP;         // columns of the staged X chunk and of the Y item
  int* Xe;             // [kRows] exponent of each staged row
  int* Ye;             // [kNP]   exponent of each Y row (output column)
  int* re;             // [2 kRows] stored exponents of the source rows
  float* rmax;         // [2 kRows] row maxima of the two column halves
};
__device__ __forceinline__ Smem carve(unsigned char* base, int S, int KPx, int KP) {
  Smem m;
  m.KPx = KPx;
  m.KP = KP;
  m.xplane = kRows * KPx * 2;
  m.yplane = kNP * KP * 2;
  m.X = base;
  m.Y = base + S * m.xplane;
  m.Xe = reinterpret_cast<int*>(m.Y + S * m.yplane);
  m.Ye = m.Xe + kRows;
  m.re = m.Ye + kNP;
  m.rmax = reinterpret_cast<float*>(m.re + 2 * kRows);
  return m;
}
__host__ __device__ __forceinline__ size_t smem_bytes(int S, int KPx, int KP) {
  return size_t(S) * kRows * KPx * 2 + size_t(S) * kNP * KP * 2 + size_t(kRows + kNP + 4 * kRows) * 4 + 16;
}

// Make this thread's shared-memory operand writes visible to the tensor
// cores and order its earlier TMEM reads, then synchronise the CTA.
__device__ __forceinline__ void sync_for_mma() {
  lc_fence_proxy_async();
  umma_fence_before();
  __syncthreads();
}

// Stage up to two 18-wide double-float row blocks (rows A0 and, if two, A1
// for the same members) side by side as one operand row of 18 or 36 columns,
// in a common exponent frame (from the stored row exponents), sliced into X.
// Rows beyond `valid` are zero.  In a persistent launch the rows were
// written by other CTAs: dep_wait's acquire and the CTA barrier after it
// order these loads after those writes.
__device__ __forceinline__ void stage_rows_df(const Dev& D, const float2* A, const int* Ae, int64_t rowA0,
                                              int64_t rowA1, int two, int64_t tile0, int64_t valid, Smem& m) {
  const int parts = two ? 2 : 1;
  for (int i = threadIdx.x; i < kRows * parts; i += blockDim.x) {
    const int part = i / kRows, rr = i % kRows;
    const int64_t r = tile0 + rr;
    m.re[i] = (r < valid) ? Ae[(part ? rowA1 : rowA0) + r] : -100000;
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < kRows; rr += blockDim.x)
    m.Xe[rr] = two ? max(m.re[rr], m.re[kRows + rr]) : m.re[rr];
  __syncthreads();
  const int nch = m.KPx / 8;
  for (int i = threadIdx.x; i < kRows * nch; i += blockDim.x) {
    const int rr = i % kRows, ch = i / kRows;
    const bool ok = tile0 + rr < valid;
    const float sc0 = ok ? pow2f(m.re[rr] - m.Xe[rr]) : 0.0f;
    const float sc1 = (ok && two) ? pow2f(m.re[kRows + rr] - m.Xe[rr]) : 0.0f;
    float hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * ch + j;
      hi[j] = lo[j] = 0.0f;
      if (ok && c < LC_M * parts) {
        const int part = c >= LC_M;
        const float2 v = A[((part ? rowA1 : rowA0) + tile0 + rr) * LC_M + (c - part * LC_M)];
        const float sc = part ? sc1 : sc0;
        hi[j] = v.x * sc;
        lo[j] = v.y * sc;
      }
    }
    put_chunk(m.X, m.xplane, m.KPx, rr, ch, D.S, hi, lo);
  }
  sync_for_mma();
}

// FP64 input value j of a member (zero outside [0, len)); cinv != 0
// multiplies it by C^{-1} (2/pi, 1/pi at index 0) first (transposed L2C pass).
__device__ __forceinline__ double in_value(const Dev& D, int64_t rb, int64_t j, int64_t len, int cinv) {
  if (j < 0 || j >= len) return 0.0;
  const double x = D.in[rb + j * D.ie];
  return cinv ? x * (j == 0 ? 0.31830988618379067154 : 0.63661977236758134308) : x;
}
// Exponent of each tile row's largest input value among columns c < ncols
// (column c of member row rr is x_r[j0 + 2c]); m.Xe receives the row frame
// exponent (largest entry brought into [1/4, 1/2)).
__device__ __forceinline__ void input_frames(const Dev& D, int64_t tile0, int64_t valid, int64_t j0, int ncols, Smem& m,
                                             const int64_t* rbase, const int64_t* rlen, int cinv) {
  for (int rr = threadIdx.x; rr < kRows; rr += blockDim.x) m.Xe[rr] = kNoExp;
  __syncthreads();
  const int nch = (ncols + 7) / 8;
  for (int i = threadIdx.x; i < kRows * nch; i += blockDim.x) {
    const int rr = i % kRows, ch = i / kRows;
    if (tile0 + rr >= valid) continue;
    int E = kNoExp;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * ch + j;
      if (c < ncols) E = max(E, exp_field(in_value(D, rbase[rr], j0 + 2 * c, rlen[rr], cinv)));
    }
    if (E > kNoExp) atomicMax(&m.Xe[rr], E);
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < kRows; rr += blockDim.x) m.Xe[rr] = (m.Xe[rr] > kNoExp ? m.Xe[rr] : -4000) - 1021;
  __syncthreads();
}
// Slice columns [c0, c0 + KPx) of the input operand (zero at c >= ncols) into X
// in the frame of m.Xe.
__device__ __forceinline__ void stage_input(const Dev& D, int64_t tile0, int64_t valid, int64_t j0, int ncols, int c0,
                                            Smem& m, const int64_t* rbase, const int64_t* rlen, int cinv) {
  const int nch = m.KPx / 8;
  for (int i = threadIdx.x; i < kRows * nch; i += blockDim.x) {
    const int rr = i % kRows, ch = i / kRows;
    const bool ok = tile0 + rr < valid;
    float hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + 8 * ch + j;
      const double x = (ok && c < ncols) ? in_value(D, rbase[rr], j0 + 2 * c, rlen[rr], cinv) : 0.0;
      d2df_scaled(x, m.Xe[rr], hi[j], lo[j]);
    }
    put_chunk(m.X, m.xplane, m.KPx, rr, ch, D.S, hi, lo);
  }
  sync_for_mma();
}

// Per-row input/output bases and lengths of a member tile.
__device__ __forceinline__ void row_info(const Dev& D, int64_t tile0, int64_t valid, int64_t* rbase, int64_t* obase,
                                         int64_t* rlen) {
  for (int rr = threadIdx.x; rr < kRows; rr += blockDim.x) {
    const int64_t r = tile0 + rr;
    const bool ok = r < valid;
    rbase[rr] = ok ? (D.ragged ? D.off[r] : lc_boff(D.orig[r], D.ib, D.inner, D.iob)) : 0;
    if (obase) obase[rr] = ok ? (D.ragged ? D.off[r] : lc_boff(D.orig[r], D.ob, D.inner, D.oob)) : 0;
    rlen[rr] = ok ? D.len[r] : 0;
  }
  __syncthreads();
}

// ---- tensor-core stage: TMEM holds one kNP-column accumulator per slice
// diagonal u = s + t (u = 2 .. S + 1), at columns (u - 2) kNP.  TMEM is
// taken only once the first operand is staged (tc_acquire): a CTA resident
// beside two others that hold TMEM stages its operands meanwhile and waits
// in the allocation, instead of idling from its start.
struct TcState {
  uint32_t* tslot;  // shared: TMEM base address
  uint64_t* mbar;   // shared: MMA completion barrier
  uint32_t tmem;
  uint32_t phase;
  bool held;
};
// Shared state of a CTA across its tasks.
struct CtaShared {
  uint64_t mbar_y, mbar_mma;
  uint32_t tslot;
  int ticket;
  int ye_near[kNP];
};
// Per-row input/output bases and lengths of the leaf and final stages, in
// dynamic shared memory after the stage's operands (`off` bytes from its
// start): [3][kRows] int64.

struct RowArrays {
  int64_t* rbase;
  int64_t* obase;
  int64_t* rlen;
};
__device__ __forceinline__ RowArrays row_arrays(unsigned char* base, size_t off) {
  int64_t* p = reinterpret_cast<int64_t*>(base + ((off + 15) & ~size_t(15)));
  return RowArrays{p, p + kRows, p + 2 * kRows};
}
// Per-CTA state of the stage bodies: the Y-copy mbarrier's running phase
// count and the MMA state (mbarrier phase, TMEM).
struct Ctx {
  CtaShared* sh;
  TcState tc;
  uint32_t ycount;
};
__device__ __forceinline__ Ctx ctx_begin(const Dev& D, CtaShared& sh) {
  for (int i = threadIdx.x; i <= D.Lmax + 1; i += blockDim.x) s_lcount[i] = D.Lcount[i];
  if (threadIdx.x == 0) {
    lc_mbar_init(lc_smem_u32(&sh.mbar_y));
    lc_mbar_init(lc_smem_u32(&sh.mbar_mma));
  }
  __syncthreads();
  return Ctx{&sh, TcState{&sh.tslot, &sh.mbar_mma, 0u, 0u, false}, 0u};
}
__device__ __forceinline__ void tc_acquire(TcState& tc) {
  if (tc.held) return;
  if (threadIdx.x < 32) {
    umma_alloc(tc.tslot, kTmemCols);
    umma_relinquish();
  }
  umma_fence_before();
  __syncthreads();
  umma_fence_after();
  tc.tmem = *tc.tslot;
  tc.held = true;
}
__device__ __forceinline__ void tc_end(const TcState& tc) {
  if (!tc.held) return;
  umma_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) umma_dealloc(tc.tmem, kTmemCols);
}

// Slice products of the staged X (its K slices [xkt0, xkt0 + KPx/16) of the
// full operand) with the Y item over the K slices [kt0, kt1): thread 0 issues
// one tcgen05.mma (M = kRows, N = kNP, K = 16) per slice pair and K slice into
// the diagonal's accumulator -- acc_first: add to what it holds -- and
// commits them to the mbarrier; every thread waits for that phase (bounded).
// A timeout returns false after a second bounded wait, so that no MMA is in
// flight when the caller releases TMEM.
__device__ __forceinline__ bool tc_products(const Smem& m, int S, int xkt0, int kt0, int kt1, TcState& tc,
                                            bool acc_first) {
  tc_acquire(tc);
  const uint32_t tmem = tc.tmem;
  uint32_t& phase = tc.phase;
  const uint32_t mb = lc_smem_u32(tc.mbar);
  if (threadIdx.x == 0) {
    umma_fence_after();
    const uint32_t xs = lc_smem_u32(m.X), ys = lc_smem_u32(m.Y);
    constexpr uint32_t idesc = umma_idesc_bf16(kRows, kNP);
    for (int u = 2; u <= S + 1; ++u) {
      uint32_t acc = acc_first ? 1u : 0u;
      const int s0 = u - S > 1 ? u - S : 1, s1 = u - 1 < S ? u - 1 : S;
      for (int sx = s0; sx <= s1; ++sx) {
        const uint32_t xa = xs + uint32_t(sx - 1) * m.xplane, ya = ys + uint32_t(u - sx - 1) * m.yplane;
        for (int kt = kt0; kt < kt1; ++kt) {
          umma_bf16(tmem + uint32_t(u - 2) * kNP, umma_desc_kslice(xa, m.KPx, kt - xkt0),
                    umma_desc_kslice(ya, m.KP, kt), idesc, acc);
          acc = 1u;
        }
      }
    }
    umma_commit(mb);
  }
  const bool ok = lc_mbar_wait_bounded(mb, phase);
  const bool bad = __syncthreads_or(!ok);
  if (bad && threadIdx.x == 0) lc_mbar_wait_bounded(mb, phase);
  phase ^= 1u;
  umma_fence_after();
  return !bad;
}

// This thread's place in the accumulators: tile row ep_row() (TMEM lane
// 32 (warp % 4) + lane), columns ep_col0() .. + kCols - 1.
__device__ __forceinline__ int ep_row() { return ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31); }
__device__ __forceinline__ int ep_col0() { return int(threadIdx.x >> 7) * kCols; }

// Recombine the diagonals of this thread's row and columns:
// hi + lo = sum_u P_u 2^(-8 (u - 2)), the product times 2^16 in units of
// 2^(e_x + e_y), by a Horner sum in base 2^8 in double-float.
// The diagonals are read in groups of up to two loads in flight, one wait
// per group (more would cost the registers of a third resident CTA).
__device__ __forceinline__ void horner_step(float (&hi)[kCols], float (&lo)[kCols], const uint32_t (&p)[kCols],
                                            bool first) {
#pragma unroll
  for (int j = 0; j < kCols; ++j) {
    const float pj = __uint_as_float(p[j]);
    if (first) {
      hi[j] = pj;
      lo[j] = 0.0f;
    } else {
      float sh, se;
      two_sum(hi[j] * (1.0f / 256.0f), pj, sh, se);
      fast_two_sum(sh, lo[j] * (1.0f / 256.0f) + se, hi[j], lo[j]);
    }
  }
}
__device__ __forceinline__ void tc_recombine(uint32_t tmem, int S, float (&hi)[kCols], float (&lo)[kCols]) {
  const uint32_t base = tmem + (uint32_t(32 * ((threadIdx.x >> 5) & 3)) << 16) + uint32_t(ep_col0());
  int u = S + 1;
  while (u >= 2) {
    const int g = u - 1 < 2 ? u - 1 : 2;  // diagonals u (and u - 1) in this group
    uint32_t p[2][kCols];
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (q < g) umma_ld16_async(base + uint32_t(u - q - 2) * kNP, p[q]);
    umma_wait_ld();
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (q < g) horner_step(hi, lo, p[q], u - q == S + 1);
    u -= g;
  }
}

// Value frame of this thread's row: hi/lo hold P 2^16 in units of
// 2^(e_x + e_y(col)); scale them to value 2^-e_row so that the row's largest
// of its `valid_cols` columns lies in [1/4, 1/2) and return e_row.  The two
// threads that share a row (column halves) exchange their maxima through
// shared memory.
__device__ __forceinline__ int tc_frame(float (&hi)[kCols], float (&lo)[kCols], const int* Ye, int ex,
                                        int valid_cols, float* rmax) {
  const int r = ep_row(), c0 = ep_col0();
  float mx = 0.0f;
#pragma unroll
  for (int j = 0; j < kCols; ++j)
    if (c0 + j < valid_cols) mx = fmaxf(mx, fabsf(hi[j]) * pow2f(Ye[c0 + j]));
  rmax[(threadIdx.x >> 7) * kRows + r] = mx;
  __syncthreads();
  mx = fmaxf(rmax[r], rmax[kRows + r]);
  const int k = (mx > 0.0f) ? exp_of(mx) : 0;
#pragma unroll
  for (int j = 0; j < kCols; ++j) {
    const float sc = (c0 + j < valid_cols) ? pow2f(Ye[c0 + j] - k - 1) : 0.0f;
    hi[j] *= sc;
    lo[j] *= sc;
  }
  __syncthreads();  // rmax is free again
  return ex - 16 + k + 1;
}

// Store this thread's part of a framed row to a double-float row array.
__device__ __forceinline__ void tc_store_row(float2* Out, int* OutE, int64_t row_base, int64_t tile0, int64_t valid,
                                             const float (&hi)[kCols], const float (&lo)[kCols], int er) {
  const int r = ep_row(), c0 = ep_col0();
  const int64_t row = tile0 + r;
  if (row >= valid) return;
#pragma unroll
  for (int j = 0; j < kCols; ++j)
    if (c0 + j < LC_M) Out[(row_base + row) * LC_M + c0 + j] = make_float2(hi[j], lo[j]);
  if (c0 == 0) OutE[row_base + row] = er;
}

// ------------------------------------------------------------ stage bodies
// Every body: one (segment or strip, parity sigma, tile of kRows members);
// `pt` is the persistent task (its dependencies), null for level-by-level
// launches.  A body returns false if a bounded wait ran out (no MMA or copy
// of its own is then in flight).

// Persistent schedule: wait until the blocks the task reads are complete.
// Thread 0 polls their write counters (relaxed loads, both at once), then
// one acquire fence; the CTA barrier passes the ordering on to every thread.
// False if the execution was aborted or the bounded wait (about a second)
// ran out.
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool dep_wait(const Dev& D, const PTask* pt, int sigma) {
  if (!pt || pt->rd[0] < 0) return true;  // (rd[1] is set only with rd[0])
  bool ok = true;
  if (threadIdx.x == 0) {
    const int* c0 = D.cnt + 2 * int64_t(pt->rd[0]) + sigma;
    const int* c1 = pt->rd[1] >= 0 ? D.cnt + 2 * int64_t(pt->rd[1]) + sigma : c0;
    const int n0 = pt->need[0], n1 = pt->rd[1] >= 0 ? pt->need[1] : 0;
    const long long t0 = clock64();
    for (;;) {
      const int v0 = ld_relaxed(c0), v1 = ld_relaxed(c1);
      if (v0 >= n0 && v1 >= n1) break;
      if (*reinterpret_cast<volatile int*>(D.abort) || clock64() - t0 > (1ll << 31)) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
    asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
  }
  return !__syncthreads_or(!ok);
}

// Steps 1-4, one product each (kind = LC_K_LEAF, _UP, _COUPLE or _DOWN):
//   leaf    W(0, g)   = F(g, sigma) T(sigma)                      (Step 1)
//   up      W(d+1, G) = [W(d, 2G) W(d, 2G+1)] [B(0) B(1)]^T       (Step 2)
//   couple  C(d, v)   = [W(d, v+2) W(d, v+3)] [A-hat(b,0) A-hat(b,1)]^T (v even),
//                       W(d, v+2) A-hat(b,2)^T (v odd)           (Step 3)
//   down    C(d, v)  += C(d+1, v/2) B(v mod 2)                    (Step 4)
// (the transposed pass: the roles of its header comment).  One code path
// for the four, so that a persistent CTA that runs all of them needs the
// registers of one.
__device__ __forceinline__ bool s_stage(const Dev& D, int kind, Work it, int sigma, unsigned char* sm_raw, Ctx& c,
                                        const PTask* pt) {
  const int d = it.d;
  const int64_t v = it.seg, tile0 = int64_t(it.tile) * kRows;
  YKind yk = Y_LEAF;
  int64_t yitem = 0, valid = 0, r0 = 0, r1 = 0, orow = 0;
  int two = 0;
  const float2* A = D.W;
  const int* Ae = D.We;
  float2* Out = D.W;
  int* OutE = D.We;
  switch (kind) {
    case LC_K_LEAF:  // column segment v (transposed: row strip)
      yitem = sigma;
      valid = dcnt(D, 0, D.adj ? v + 2 : v);
      orow = drow(D, 0, v, sigma, 0);
      break;
    case LC_K_UP:  // parent G = v at level d (transposed: row tree)
      yk = Y_UP;
      valid = dcnt(D, d, D.adj ? v + 2 : v);
      r0 = drow(D, d - 1, 2 * v, sigma, 0);
      r1 = drow(D, d - 1, 2 * v + 1, sigma, 0);
      two = 1;
      orow = drow(D, d, v, sigma, 0);
      break;
    case LC_K_COUPLE: {
      // forward: row segment v from column segments v+2 (and v+3);
      // transposed: column segment v from row segments v-2 (and v-3)
      yk = D.adj ? Y_COUPLE_T : Y_COUPLE;
      const int Gam = D.Lmax - 1 - d;  // level in the shared table
      yitem = (int64_t(4) * ((int64_t(1) << Gam) - 1) - 2 * Gam) + (D.adj ? v - 2 : v);
      valid = dcnt(D, d, D.adj ? v : v + 2);
      two = D.adj ? int(v & 1) : ((v & 1) == 0 ? 1 : 0);
      r0 = drow(D, d, D.adj ? v - 2 : v + 2, sigma, 0);
      r1 = two ? drow(D, d, D.adj ? v - 3 : v + 3, sigma, 0) : 0;
      Out = D.C;
      OutE = D.Ce;
      orow = drow(D, d, v, sigma, 0);
      break;
    }
    default:  // down: child v at level d (transposed: column segment)
      yk = Y_DOWN;
      yitem = v & 1;
      valid = dcnt(D, d, D.adj ? v : v + 4);
      A = D.C;
      Ae = D.Ce;
      r0 = drow(D, d + 1, v >> 1, sigma, 0);
      Out = D.C;
      OutE = D.Ce;
      orow = drow(D, d, v, sigma, 0);
      break;
  }
  const int KP = D.yKP[yk];
  Smem m = carve(sm_raw, D.S, KP, KP);
  y_issue(D.yq[yk] + size_t(yitem) * D.S * kNP * KP, D.ye[yk] + yitem * kNP, D.S, KP, m.Y, m.Ye, &c.sh->mbar_y);
  const bool ready = dep_wait(D, pt, sigma);
  if (ready) {
    if (kind == LC_K_LEAF) {
      const int s = D.s;
      const int cinv = D.adj && D.dir == LC_L2C;
      const RowArrays ra = row_arrays(sm_raw, smem_bytes(D.S, KP, KP));
      row_info(D, tile0, valid, ra.rbase, nullptr, ra.rlen);
      input_frames(D, tile0, valid, 2 * int64_t(s) * v + sigma, s, m, ra.rbase, ra.rlen, cinv);
      stage_input(D, tile0, valid, 2 * int64_t(s) * v + sigma, s, 0, m, ra.rbase, ra.rlen, cinv);
    } else {
      stage_rows_df(D, A, Ae, r0, r1, two, tile0, valid, m);
    }
  }
  bool ok = y_wait(&c.sh->mbar_y, c.ycount) && ready;
  if (ok) ok = tc_products(m, D.S, 0, 0, KP / 16, c.tc, false);
  if (!ok) return false;
  float hi[kCols], lo[kCols];
  tc_recombine(c.tc.tmem, D.S, hi, lo);
  const int er = tc_frame(hi, lo, m.Ye, m.Xe[ep_row()], LC_M, m.rmax);
  if (kind != LC_K_DOWN) {
    tc_store_row(Out, OutE, orow, tile0, valid, hi, lo, er);
    return true;
  }
  // down: add the existing row (the coupling result) in a common frame
  const int r = ep_row(), c0 = ep_col0();
  const int64_t row = tile0 + r;
  const int eo = row < valid ? OutE[orow + row] : 0;
  const int F = max(er, eo) + 1;
  const float sa = pow2f(er - F), sb = pow2f(eo - F);
  __syncthreads();  // both halves of every row have read the old exponent
  if (row < valid) {
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int col = c0 + j;
      if (col >= LC_M) continue;
      const float2 o = Out[(orow + row) * LC_M + col];
      float sh, se, nh, nl;
      two_sum(hi[j] * sa, o.x * sb, sh, se);
      fast_two_sum(sh, se + lo[j] * sa + o.y * sb, nh, nl);
      Out[(orow + row) * LC_M + col] = make_float2(nh, nl);
    }
    if (c0 == 0) OutE[orow + row] = F;
  }
  return true;
}

// Steps 5-7 for strip t and parity sigma, kRows members per CTA:
//   Z = F(strip) E^T + C(0, t) T(sigma)^T, then C^{-1} (L2C), store.
// The near-field product (K = 2s, staged kXCols columns at a time) and the
// spread (K = 18) reuse the same shared memory and TMEM one after the other;
// their results meet in the FP64 Step 7.
__device__ __forceinline__ bool s_final(const Dev& D, Work it, int sigma, unsigned char* sm_raw, Ctx& c) {
  CtaShared& sh = *c.sh;
  const int64_t t = it.seg, tile0 = int64_t(it.tile) * kRows;
  const int64_t validN = D.cntN[t];
  // far field of strip t: row segment t (forward), column segment t (transposed)
  const int64_t validF = D.Lmax <= 0 ? 0
                         : D.adj ? ((t >= 2 && t < (int64_t(2) << D.Lmax)) ? dcnt(D, 0, t) : 0)
                                 : ((t + 2 < (int64_t(2) << D.Lmax)) ? dcnt(D, 0, t + 2) : 0);
  const int s = D.s;
  const int KPn = D.yKP[Y_NEAR];
  const int KPx = KPn < kXCols ? KPn : kXCols;
  const int KPs = D.yKP[Y_SPREAD];
  Smem m = carve(sm_raw, D.S, KPx, KPn);
  // after the larger of the near-field and spread operands
  const RowArrays ra = row_arrays(sm_raw, max(smem_bytes(D.S, KPx, KPn), smem_bytes(D.S, KPs, KPs)));
  const int r = ep_row(), c0 = ep_col0();
  float nh[kCols], nl[kCols], fh[kCols], fl[kCols];
  int enx = 0, efx = 0;
  // ---- near field
  const int64_t item = 2 * t + sigma;
  const YKind yk = D.adj ? Y_NEAR_T : Y_NEAR;
  y_issue(D.yq[yk] + size_t(item) * D.S * kNP * KPn, D.ye[yk] + item * kNP, D.S, KPn, m.Y, m.Ye, &sh.mbar_y);
  bool ok = true;
  {
    // forward: columns of strips t, t+1 of the band of rows in strip t;
    // transposed: rows of strips t-1, t (times C^{-1} for L2C) for columns in strip t
    const int cinv = D.adj && D.dir == LC_L2C;
    const int64_t j0 = 2 * int64_t(s) * (D.adj ? t - 1 : t) + sigma;
    row_info(D, tile0, validN, ra.rbase, ra.obase, ra.rlen);
    input_frames(D, tile0, validN, j0, 2 * s, m, ra.rbase, ra.rlen, cinv);
    for (int cc = 0; cc < KPn && ok; cc += KPx) {
      stage_input(D, tile0, validN, j0, 2 * s, cc, m, ra.rbase, ra.rlen, cinv);
      if (cc == 0) ok = y_wait(&sh.mbar_y, c.ycount);
      const int kt1 = (cc + KPx < KPn ? cc + KPx : KPn) / 16;
      if (ok) ok = tc_products(m, D.S, cc / 16, cc / 16, kt1, c.tc, cc > 0);
    }
  }
  if (ok) {
    tc_recombine(c.tc.tmem, D.S, nh, nl);
    enx = m.Xe[r];
    if (threadIdx.x < kNP) sh.ye_near[threadIdx.x] = m.Ye[threadIdx.x];
    sync_for_mma();  // every TMEM read of the near field is done; Y and Xe may be overwritten
  }
  // ---- far field (spread)
  const bool far_tile = validF > tile0;
  if (ok && far_tile) {
    Smem m2 = carve(sm_raw, D.S, KPs, KPs);
    y_issue(D.yq[Y_SPREAD] + size_t(sigma) * D.S * kNP * KPs, D.ye[Y_SPREAD] + sigma * kNP, D.S, KPs, m2.Y, m2.Ye,
            &sh.mbar_y);
    stage_rows_df(D, D.C, D.Ce, drow(D, 0, t, sigma, 0), 0, 0, tile0, validF, m2);
    ok = y_wait(&sh.mbar_y, c.ycount);
    if (ok) ok = tc_products(m2, D.S, 0, 0, KPs / 16, c.tc, false);
    if (ok) {
      tc_recombine(c.tc.tmem, D.S, fh, fl);
      efx = m2.Xe[r];
      m.Ye = m2.Ye;
    }
  }
  // ---- Step 7 in FP64 and the store
  if (ok) {
    const int64_t row = tile0 + r;
    const bool l2c = (D.dir == LC_L2C) && !D.adj;  // (the transposed pass applied C^{-1} first)
    const bool far = far_tile && row < validF;
    if (row < validN) {
#pragma unroll
      for (int j = 0; j < kCols; ++j) {
        const int col = c0 + j;  // local row m of the strip
        if (col >= s) continue;
        const int64_t row_i = 2 * int64_t(s) * t + 2 * col + sigma;
        if (row_i >= ra.rlen[r]) continue;
        const int E1 = enx + sh.ye_near[col] - 16;
        const int E2 = efx + (far ? m.Ye[col] : 0) - 16;
        // near (nh + nl) 2^E1 and far (fh + fl) 2^E2, each word brought to
        // FP64 exactly, summed and scaled by C^{-1} (L2C) in FP64
        const double cf = l2c ? ((row_i == 0) ? 0.31830988618379067154 : 0.63661977236758134308) : 1.0;
        const double lo_sum = f2d_scaled(nl[j], E1) + (far ? f2d_scaled(fl[j], E2) : 0.0);
        const double hi_far = far ? f2d_scaled(fh[j], E2) : 0.0;
        D.out[ra.obase[r] + row_i * D.oe] = fma(cf, f2d_scaled(nh[j], E1), fma(cf, hi_far, cf * lo_sum));
      }
    }
  }
  return ok;
}

// ------------------------------------------------------------------ kernels
// Level-by-level launches: one task per CTA (item w0 + blockIdx.x / 2,
// parity blockIdx.x % 2); TMEM taken once the first operand is staged and
// released at the end on every path; a failed bounded wait sets the plan's
// status word.
template <int KIND>
__device__ __forceinline__ void level_task(const Dev& D, int64_t w0) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ __align__(16) CtaShared sh;
  Ctx c = ctx_begin(D, sh);
  const Work it = D.work[w0 + (blockIdx.x >> 1)];
  const int sigma = int(blockIdx.x & 1);
  const bool ok = KIND == LC_K_FINAL ? s_final(D, it, sigma, sm_raw, c)
                                     : s_stage(D, KIND, it, sigma, sm_raw, c, nullptr);
  if (!ok && threadIdx.x == 0) atomicOr(D.err, 1);
  tc_end(c.tc);
}
__global__ void __launch_bounds__(kThreads) k_s_leaf(Dev D, int64_t w0) { level_task<LC_K_LEAF>(D, w0); }
__global__ void __launch_bounds__(kThreads) k_s_up(Dev D, int64_t w0) { level_task<LC_K_UP>(D, w0); }
__global__ void __launch_bounds__(kThreads) k_s_couple(Dev D, int64_t w0) { level_task<LC_K_COUPLE>(D, w0); }
// (three CTAs of the down stage fit an SM by shared memory: keep their registers to a third)
__global__ void __launch_bounds__(kThreads, 3) k_s_down(Dev D, int64_t w0) { level_task<LC_K_DOWN>(D, w0); }
__global__ void __launch_bounds__(kThreads) k_s_final(Dev D, int64_t w0) { level_task<LC_K_FINAL>(D, w0); }

// Steps 1-4 of an execution in one persistent launch.  Each CTA takes TMEM
// once, before its first task, then draws tickets (task = ticket / 2,
// parity = ticket % 2) from a global counter until they run out, always one
// ticket ahead: thread 64 draws the next ticket and loads its task while the
// current task runs, off the path of thread 0, which issues the copies and
// MMAs.  A task waits only for blocks written by tasks of smaller tickets;
// the smallest unfinished ticket is always the current task of the CTA
// holding it, and its inputs are complete, so the launch finishes whatever
// the number of resident CTAs.  After the task's
// stores, thread 32 publishes its block (a release increment of its counter)
// while thread 0 starts the next task's copies.  A failed wait sets the abort
// word: every CTA then stops drawing tickets and every waiter gives up, and
// the plan's status word reports it.  (The final stage, Steps 5-7, is the
// next launch: its register needs would spill here.)
__device__ __forceinline__ int draw(const Dev& D, int n) {
  return *reinterpret_cast<volatile int*>(D.abort) ? n : int(atomicAdd(D.head, 1u));
}
__global__ void __launch_bounds__(kThreads, 2) k_s_persist(Dev D, const PTask* __restrict__ tasks, int ntickets) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ __align__(16) CtaShared sh;
  __shared__ int tk[2];
  __shared__ PTask ptk[2];
  if (threadIdx.x == 0) {
    tk[0] = draw(D, ntickets);
    if (tk[0] < ntickets) ptk[0] = tasks[tk[0] >> 1];
  }
  Ctx c = ctx_begin(D, sh);
  tc_acquire(c.tc);
  for (int it = 0;; ++it) {
    const int t = tk[it & 1];
    if (t >= ntickets) break;
    if (threadIdx.x == 64) {  // the next ticket and its task, off thread 0's path; read after the barrier below
      const int tn = draw(D, ntickets);
      tk[(it + 1) & 1] = tn;
      if (tn < ntickets) ptk[(it + 1) & 1] = tasks[tn >> 1];
    }
    const PTask pt = ptk[it & 1];
    const bool ok = s_stage(D, pt.kind, Work{pt.d, pt.seg, pt.tile}, t & 1, sm_raw, c, &pt);
    __syncthreads();  // the task's stores are issued; the next ticket is visible
    if (threadIdx.x == 32) {
      if (!ok) {
        atomicOr(D.abort, 1);
        atomicOr(D.err, 1);
      } else if (pt.wr >= 0) {  // release: the CTA's stores (ordered by the barrier) before the count
        asm volatile("red.release.gpu.global.add.s32 [%0], 1;\n" ::"l"(D.cnt + 2 * int64_t(pt.wr) + (t & 1))
                     : "memory");
      }
    }
  }
  tc_end(c.tc);
}

// ------------------------------------------------------------ plan kernels
__device__ double y_value(int kind, int64_t item, int k, int n, const lc_plan_s& P, int s, int L, int64_t N,
                          int dir) {
  switch (kind) {
    case Y_LEAF:  // Y[m][k'] = T[sigma][m][k']
      return (n < LC_M && k < s) ? P.T[(item * s + k) * LC_M + n] : 0.0;
    case Y_SPREAD:  // Y[k'][m] = T[sigma][m][k']
      return (k < LC_M && n < s) ? P.T[(item * s + n) * LC_M + k] : 0.0;
    case Y_UP: {  // Y[c*18+j][k'] = B(c)[k'][j]
      if (n >= LC_M || k >= 2 * LC_M) return 0.0;
      const int c = k / LC_M, j = k % LC_M;
      const double b = P.B[n * LC_M + j];
      return (c == 1 && ((n - j) & 1)) ? -b : b;
    }
    case Y_DOWN: {  // Y[j][k'] = B(p)[j][k']
      if (n >= LC_M || k >= LC_M) return 0.0;
      const double b = P.B[k * LC_M + n];
      return (item == 1 && ((k - n) & 1)) ? -b : b;
    }
    case Y_COUPLE: {
      if (n >= LC_M || k >= 2 * LC_M) return 0.0;
      int G = 0;
      while (G + 1 < L && item >= 4 * ((int64_t(1) << (G + 1)) - 1) - 2 * (G + 1)) ++G;
      const int64_t v = item - (4 * ((int64_t(1) << G) - 1) - 2 * G);
      const int64_t b = v >> 1;
      const int64_t aoff = lc_ahat_offset(G);
      if ((v & 1) == 0) {
        const int c = k / LC_M, l = k % LC_M;
        return P.Ahat[(aoff + 3 * b + c) * (LC_M * LC_M) + n * LC_M + l];
      }
      if (k >= LC_M) return 0.0;
      return P.Ahat[(aoff + 3 * b + 2) * (LC_M * LC_M) + n * LC_M + k];
    }
    case Y_COUPLE_T: {  // column segment g: Y[c*18 + k][l] = A-hat(b, c')[k][l]
      if (n >= LC_M || k >= 2 * LC_M) return 0.0;
      int G = 0;
      while (G + 1 < L && item >= 4 * ((int64_t(1) << (G + 1)) - 1) - 2 * (G + 1)) ++G;
      const int64_t g = item - (4 * ((int64_t(1) << G) - 1) - 2 * G) + 2;
      const int64_t aoff = lc_ahat_offset(G);
      const int c = k / LC_M, kk = k % LC_M;
      if ((g & 1) == 0) {  // from row segment g-2 (even): A-hat(b, 0), b = (g-2)/2
        if (c) return 0.0;
        return P.Ahat[(aoff + 3 * ((g - 2) >> 1)) * (LC_M * LC_M) + kk * LC_M + n];
      }
      // from row segments g-2 (odd, A-hat(b, 2)) and g-3 (even, A-hat(b, 1)), b = (g-3)/2
      return P.Ahat[(aoff + 3 * ((g - 3) >> 1) + (c ? 1 : 2)) * (LC_M * LC_M) + kk * LC_M + n];
    }
    case Y_NEAR_T: {  // column strip t: Y[k][m] = entry (row 2s(t-1)+2k+sigma, column 2st+2m+sigma)
      if (n >= s || k >= 2 * s) return 0.0;
      const int64_t t = item >> 1;
      const int sigma = int(item & 1);
      const int64_t i = 2 * int64_t(s) * (t - 1) + 2 * k + sigma;
      const int64_t j = 2 * int64_t(s) * t + 2 * n + sigma;
      if (i < 0 || j < i || j >= N) return 0.0;
      const int64_t kk = (j - i) / 2;
      if (dir == LC_L2C) return P.lam[kk] * P.lam2[i + kk];
      double e = (double(2 * i) + P.geg.two_alpha) * double(j) * P.lam[kk] * P.lam2[i + kk];
      if (i == 0 && j == 0) e += 1.0;
      return e;
    }
    case Y_NEAR: {  // Y[jj][m] = E(t, sigma)[m][jj]
      if (n >= s || k >= 2 * s) return 0.0;
      const int64_t t = item >> 1;
      const int sigma = int(item & 1);
      const int64_t i = 2 * int64_t(s) * t + 2 * n + sigma;
      const int64_t j = 2 * int64_t(s) * t + 2 * k + sigma;
      if (j < i || j >= N || i >= N) return 0.0;
      const int64_t kk = (j - i) / 2;
      if (dir == LC_L2C) return P.lam[kk] * P.lam2[i + kk];
      double e = (double(2 * i) + P.geg.two_alpha) * double(j) * P.lam[kk] * P.lam2[i + kk];
      if (i == 0 && j == 0) e += 1.0;
      return e;
    }
  }
  return 0.0;
}

// Slice planes of the shared operands, item by item: plane sl of item it
// holds digit sl of every entry (row n < kNP, column k < KP) in the canonical
// K-major layout of lc_umma.cuh, scaled by the row's exponent e[it][n].
__global__ void k_make_y(int kind, int items, int K, int KP, int S, lc_plan_s P, int s, int L, int64_t N,
                         int dir, uint16_t* __restrict__ q, int* __restrict__ e) {
  constexpr int NP = kNP;
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(items) * NP) return;
  const int64_t item = tid / NP;
  const int n = int(tid % NP);
  double mx = 0.0;
  for (int k = 0; k < K; ++k) mx = fmax(mx, fabs(y_value(kind, item, k, n, P, s, L, N, dir)));
  int ey = 0;
  if (mx > 0.0) {
    int ex;
    frexp(mx, &ex);  // mx in [2^(ex-1), 2^ex)
    ey = ex + 1;
  }
  e[item * NP + n] = ey;
  unsigned char* dst = reinterpret_cast<unsigned char*>(q) + size_t(item) * S * NP * KP * 2;
  for (int k = 0; k < KP; ++k) {
    double y = (k < K) ? ldexp(y_value(kind, item, k, n, P, s, L, N, dir), -ey) : 0.0;
    for (int sl = 0; sl < S; ++sl) {
      const double tt = y * 256.0;
      const double qq = rint(tt);
      y = tt - qq;
      *reinterpret_cast<uint16_t*>(dst + size_t(sl) * NP * KP * 2 + umma_offset(n, k, KP)) =
          uint16_t(__float_as_uint(float(qq)) >> 16);
    }
  }
}

Dev make_dev(const lc_plan_s* p, const SplitHost& h) {
  char* base = static_cast<char*>(p->split);
  Dev D;
  memset(&D, 0, sizeof(D));
  D.S = h.S;
  D.s = h.s;
  D.Lmax = h.Lmax;
  D.count = h.count;
  D.Nmax = h.Nmax;
  D.nstrips = h.nstrips;
  D.len = reinterpret_cast<const int64_t*>(base + h.off_len);
  D.orig = reinterpret_cast<const int64_t*>(base + h.off_orig);
  D.off = reinterpret_cast<const int64_t*>(base + h.off_off);
  D.Lcount = reinterpret_cast<const int64_t*>(base + h.off_Lcount);
  D.cntN = reinterpret_cast<const int64_t*>(base + h.off_cntN);
  D.rowbase = reinterpret_cast<const int64_t*>(base + h.off_rowbase);
  D.work = reinterpret_cast<const Work*>(base + h.off_work);
  D.W = reinterpret_cast<float2*>(base + h.off_W);
  D.We = reinterpret_cast<int*>(base + h.off_We);
  D.C = reinterpret_cast<float2*>(base + h.off_C);
  D.Ce = reinterpret_cast<int*>(base + h.off_Ce);
  for (int k = 0; k < Y_KINDS; ++k) {
    D.yq[k] = reinterpret_cast<const uint16_t*>(base + h.y[k].off_q);
    D.ye[k] = reinterpret_cast<const int*>(base + h.y[k].off_e);
    D.yKP[k] = h.y[k].KP;
  }
  D.dir = int(p->dir);
  D.ragged = p->ragged;
  D.adj = 0;
  D.err = p->err;
  return D;
}

// Dynamic shared memory of each stage (kind) and of the persistent kernel
// (the largest stage).
size_t stage_smem(const SplitHost& h, int kind) {
  auto sq = [&](YKind k) { return smem_bytes(h.S, h.y[k].KP, h.y[k].KP); };
  switch (kind) {
    case LC_K_LEAF: return sq(Y_LEAF) + 16 + kRowBytes;
    case LC_K_UP: return sq(Y_UP);
    case LC_K_COUPLE: return std::max(sq(Y_COUPLE), sq(Y_COUPLE_T));
    case LC_K_DOWN: return sq(Y_DOWN);
    default: {
      const int kpn = h.y[Y_NEAR].KP, kpx = kpn < kXCols ? kpn : kXCols;
      return std::max(smem_bytes(h.S, kpx, kpn), sq(Y_SPREAD)) + 16 + kRowBytes;
    }
  }
}
size_t persist_smem(const SplitHost& h) {
  size_t b = 0;
  for (int k : {LC_K_LEAF, LC_K_UP, LC_K_COUPLE, LC_K_DOWN}) b = std::max(b, stage_smem(h, k));
  return b;
}

}  // namespace

size_t lc_split_bytes(const lc_plan_s* p) {
  SplitHost h;
  build_host(p, h, 2, false);
  return h.total;
}

lc_status lc_split_prepare(lc_plan p, char* base, size_t bytes, cudaStream_t st) {
  if (p->g.s > 32) return LC_ERR_UNSUPPORTED;  // K tiles sized for s <= 32
  if (p->g.L + 2 > kMaxLcount) return LC_ERR_UNSUPPORTED;
  int dev = 0, sms = 0;
  LC_CUDA_TRY(cudaGetDevice(&dev));
  LC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SplitHost* h = new (std::nothrow) SplitHost;
  if (!h) return LC_ERR_HOST_ALLOC;
  build_host(p, *h, 2 * sms, true);
  if (h->total > bytes) {
    delete h;
    return LC_ERR_WORKSPACE_TOO_SMALL;
  }
  p->ragged_dev = h;  // host tables stay alive with the plan (freed by lc_split_release)
  auto up = [&](size_t off, const void* src, size_t n) -> lc_status {
    if (n) LC_CUDA_TRY(cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st));
    return LC_OK;
  };
  lc_status s2;
  if ((s2 = up(h->off_len, h->len_sorted.data(), h->count * 8)) != LC_OK) return s2;
  if ((s2 = up(h->off_orig, h->orig.data(), h->count * 8)) != LC_OK) return s2;
  if ((s2 = up(h->off_off, h->off_sorted.data(), h->count * 8)) != LC_OK) return s2;
  if ((s2 = up(h->off_Lcount, h->Lcount.data(), h->Lcount.size() * 8)) != LC_OK) return s2;
  if ((s2 = up(h->off_cntN, h->cntN.data(), h->cntN.size() * 8)) != LC_OK) return s2;
  if ((s2 = up(h->off_rowbase, h->rowbase.data(), h->rowbase.size() * 8)) != LC_OK) return s2;
  if ((s2 = up(h->off_work, h->work.data(), h->work.size() * sizeof(Work))) != LC_OK) return s2;
  if ((s2 = up(h->off_awork, h->awork.data(), h->awork.size() * sizeof(Work))) != LC_OK) return s2;
  if (h->persist && (p->opt.debug_flags & 2)) {
    // testing only: one task in the second half of each list waits for one
    // write more than its block ever receives, so its bounded wait runs out
    for (std::vector<PTask>* tl : {&h->ptask, &h->aptask})
      for (size_t i = tl->size() / 2; i < tl->size(); ++i)
        if ((*tl)[i].rd[0] >= 0) {
          (*tl)[i].need[0] += 1;
          break;
        }
  }
  if ((s2 = up(h->off_ptask, h->ptask.data(), h->ptask.size() * sizeof(PTask))) != LC_OK) return s2;
  if ((s2 = up(h->off_aptask, h->aptask.data(), h->aptask.size() * sizeof(PTask))) != LC_OK) return s2;
  const int Ks[Y_KINDS] = {h->s, LC_M, 2 * LC_M, LC_M, 2 * LC_M, 2 * h->s, 2 * LC_M, 2 * h->s};
  for (int k = 0; k < Y_KINDS; ++k) {
    const YTable& y = h->y[k];
    if (y.items == 0) continue;
    const int64_t threads = int64_t(y.items) * kNP;
    k_make_y<<<unsigned((threads + 127) / 128), 128, 0, st>>>(
        k, y.items, Ks[k], y.KP, h->S, *p, h->s, h->Lmax, h->Nmax, int(p->dir),
        reinterpret_cast<uint16_t*>(base + y.off_q), reinterpret_cast<int*>(base + y.off_e));
    LC_LAUNCH_CHECK();
  }
  const size_t big = smem_bytes(7, 64, 64) + 16 + kRowBytes;  // the largest configuration any kernel takes
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, int(big)));
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_up, cudaFuncAttributeMaxDynamicSharedMemorySize, int(big)));
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_couple, cudaFuncAttributeMaxDynamicSharedMemorySize, int(big)));
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_down, cudaFuncAttributeMaxDynamicSharedMemorySize, int(big)));
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_final, cudaFuncAttributeMaxDynamicSharedMemorySize, int(big)));
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, int(big)));
  LC_CUDA_TRY(cudaFuncSetAttribute(k_s_persist, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   int(cudaSharedmemCarveoutMaxShared)));
  // the persistent launch: shared memory of the largest stage, two CTAs per
  // SM (their registers fill the register file, their TMEM all of TMEM).
  // The schedule needs no co-residency: a CTA that finds no SM room starts
  // when another exits, finds no tickets left and exits.
  p->split_grid = h->persist ? 2 * sms : 0;
  return LC_OK;
}

void lc_split_release(lc_plan p) {
  if (p && p->dtype == LC_F64_SPLIT && p->ragged_dev) {
    delete static_cast<SplitHost*>(p->ragged_dev);
    p->ragged_dev = nullptr;
  }
}

int lc_exec_split_launches(const lc_plan_s* p) {
  const SplitHost* h = static_cast<const SplitHost*>(p->ragged_dev);
  if (!h) return 0;
  if (!lc_split_persistent(p)) return int(h->launch_kind.size());
  return (h->ptask.empty() ? 0 : 1) + 1;  // the persistent launch (if there are levels) and the final one
}

bool lc_split_persistent(const lc_plan_s* p) {
  const SplitHost* h = static_cast<const SplitHost*>(p->ragged_dev);
  return h && h->persist && p->split_grid > 0 && p->split_sched == 1;
}

lc_status lc_exec_split(lc_plan p, const void* in, void* out, const lc_layout& lay, cudaStream_t st,
                        int adjoint) {
  const SplitHost* h = static_cast<const SplitHost*>(p->ragged_dev);
  if (!h) return LC_ERR_INVALID_ARG;
  Dev D = make_dev(p, *h);
  if (adjoint) {
    D.adj = 1;
    D.work = reinterpret_cast<const Work*>(static_cast<char*>(p->split) + h->off_awork);
  }
  const std::vector<int64_t>& loff = adjoint ? h->alaunch_off : h->launch_off;
  const std::vector<int>& lkind = adjoint ? h->alaunch_kind : h->launch_kind;
  D.in = static_cast<const double*>(in);
  D.out = static_cast<double*>(out);
  D.ib = lay.ib;
  D.ie = lay.ie;
  D.ob = lay.ob;
  D.oe = lay.oe;
  D.inner = lay.inner;
  D.iob = lay.iob;
  D.oob = lay.oob;
  lc_timer_begin(p);
  size_t first = 0;  // first launch of the level schedule still to run
  if (lc_split_persistent(p)) {  // Steps 1-4 in one persistent launch, then the final launch
    const std::vector<PTask>& tl = adjoint ? h->aptask : h->ptask;
    char* base = static_cast<char*>(p->split);
    int* sched = reinterpret_cast<int*>(base + h->off_sched);
    D.head = reinterpret_cast<unsigned*>(sched);
    D.abort = sched + 1;
    D.cnt = sched + 4;
    const int ntickets = int(2 * tl.size());
    lc_timer_mark(p, st, LC_K_OTHER);
    LC_CUDA_TRY(cudaMemsetAsync(sched, 0, (4 + 2 * tl.size()) * sizeof(int), st));
    if (ntickets > 0) {
      const int grid = std::min(p->split_grid, ntickets);
      k_s_persist<<<grid, kThreads, persist_smem(*h), st>>>(
          D, reinterpret_cast<const PTask*>(base + (adjoint ? h->off_aptask : h->off_ptask)), ntickets);
      LC_LAUNCH_CHECK();
    }
    first = lkind.size() - 1;  // the final launch
  }
  for (size_t l = first; l < lkind.size(); ++l) {
    const int64_t w0 = loff[l], nitems = loff[l + 1] - w0;
    if (nitems <= 0) continue;
    const int kind = lkind[l];
    // the two parities of an item are neighbouring CTAs, and neighbouring
    // items share input lines, so CTAs that read the same data run together
    // (the second read hits L2)
    dim3 grid(unsigned(2 * nitems), 1);
    lc_timer_mark(p, st, kind);
    switch (kind) {
      case LC_K_LEAF: k_s_leaf<<<grid, kThreads, stage_smem(*h, kind), st>>>(D, w0); break;
      case LC_K_UP: k_s_up<<<grid, kThreads, stage_smem(*h, kind), st>>>(D, w0); break;
      case LC_K_COUPLE: k_s_couple<<<grid, kThreads, stage_smem(*h, kind), st>>>(D, w0); break;
      case LC_K_DOWN: k_s_down<<<grid, kThreads, stage_smem(*h, kind), st>>>(D, w0); break;
      case LC_K_FINAL: k_s_final<<<grid, kThreads, stage_smem(*h, kind), st>>>(D, w0); break;
    }
    LC_LAUNCH_CHECK();
  }
  lc_timer_end(p, st);
  return LC_OK;
}

