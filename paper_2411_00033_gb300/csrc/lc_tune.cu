// lc_tune.cu -- autotuning of the chunk geometry of the CUDA-core tiers.
//
// The subtree pipeline (lc_exec_kernels.cuh) has two shape parameters: the
// number of levels the first up chunk climbs (and the last down chunk
// descends), and the number of levels per coarse chunk.  Deeper leaf chunks
// mean fewer, larger CTAs and a shorter coarse chain; shallower ones more
// parallelism and less shared memory per CTA.  lc_plan_autotune times every
// candidate on the caller's data with CUDA events, keeps the fastest in the
// plan and in a process-wide cache keyed by the plan's shape, which later
// plans of the same shape pick up at creation.
#include <map>
#include <mutex>
#include <tuple>

#include "lc_internal.cuh"

namespace {
typedef std::tuple<int64_t, int64_t, int, int, int, int> Key;  // n, batch, L, s, dtype, direction
std::mutex g_mu;
std::map<Key, std::pair<int, int>> g_cache;

Key key_of(const lc_plan_s* p) {
  return Key(p->g.n, p->batch, p->g.L, p->g.s, int(p->dtype), int(p->dir));
}
bool tunable(const lc_plan_s* p) {
  return !p->ragged && (p->dtype == LC_F64 || p->dtype == LC_F32 || p->dtype == LC_F64_DF) && p->g.L > 1;
}
}  // namespace

void lc_tune_apply_cached(lc_plan p) {
  if (!tunable(p)) return;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(key_of(p));
  if (it != g_cache.end()) {
    p->leaf_depth = it->second.first;
    p->chunk_depth = it->second.second;
  }
}

extern "C" {

lc_status lc_plan_set_config(lc_plan plan, int32_t leaf_depth, int32_t chunk_depth) {
  // Depth 8 is the deepest coarse chunk whose subtree (511 nodes of 2M values,
  // plus the work array of the upward pass) fits the 227 KB of shared memory
  // of one CTA in the 8-byte types.
  if (!plan || leaf_depth < 1 || leaf_depth > 6 || chunk_depth < 1 || chunk_depth > 8) return LC_ERR_INVALID_ARG;
  plan->leaf_depth = leaf_depth;
  plan->chunk_depth = chunk_depth;
  return LC_OK;
}

lc_status lc_plan_set_band(lc_plan plan, int32_t ctas, int32_t after_leaf) {
  if (!plan || ctas < 0 || ctas > (1 << 24) || (after_leaf != 0 && after_leaf != 1)) return LC_ERR_INVALID_ARG;
  plan->band_ctas = ctas;
  plan->band_after_leaf = after_leaf;
  return LC_OK;
}

lc_status lc_plan_set_split_schedule(lc_plan plan, int32_t persistent) {
  if (!plan || (persistent != 0 && persistent != 1)) return LC_ERR_INVALID_ARG;
  if (plan->dtype != LC_F64_SPLIT) return LC_ERR_UNSUPPORTED;
  const int old = plan->split_sched;
  plan->split_sched = persistent;
  if (persistent && !lc_split_persistent(plan)) {
    plan->split_sched = old;
    return LC_ERR_UNSUPPORTED;
  }
  return LC_OK;
}

lc_status lc_plan_autotune(lc_plan plan, const void* in, void* out, int64_t in_batch_stride, int64_t in_elem_stride,
                           int64_t out_batch_stride, int64_t out_elem_stride, lc_stream stream, int32_t* leaf_depth,
                           int32_t* chunk_depth, float* best_ms) {
  if (!plan || !in || !out) return LC_ERR_INVALID_ARG;
  if (!tunable(plan)) {
    if (leaf_depth) *leaf_depth = plan->leaf_depth;
    if (chunk_depth) *chunk_depth = plan->chunk_depth;
    if (best_ms) *best_ms = 0.0f;
    return LC_OK;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  LC_CUDA_TRY(cudaEventCreate(&e0));
  LC_CUDA_TRY(cudaEventCreate(&e1));
  const int leafs[3] = {3, 4, 5};
  const int chunks[3] = {3, 4, 6};
  float best = 1e30f;
  int bl = plan->leaf_depth, bc = plan->chunk_depth;
  lc_status status = LC_OK;
  for (int a = 0; a < 3 && status == LC_OK; ++a) {
    for (int c = 0; c < 3 && status == LC_OK; ++c) {
      plan->leaf_depth = leafs[a];
      plan->chunk_depth = chunks[c];
      float tot = 0.0f;
      for (int rep = 0; rep < 4 && status == LC_OK; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        status = lc_execute(plan, in, out, in_batch_stride, in_elem_stride, out_batch_stride, out_elem_stride, stream);
      }
      if (status != LC_OK) break;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&tot, e0, e1) != cudaSuccess) {
        status = LC_ERR_CUDA;
        break;
      }
      if (tot < best) {
        best = tot;
        bl = leafs[a];
        bc = chunks[c];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->leaf_depth = bl;
  plan->chunk_depth = bc;
  if (status != LC_OK) return status;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key_of(plan)] = std::make_pair(bl, bc);
  }
  if (leaf_depth) *leaf_depth = bl;
  if (chunk_depth) *chunk_depth = bc;
  if (best_ms) *best_ms = best / 3.0f;
  return LC_OK;
}

}  // extern "C"
