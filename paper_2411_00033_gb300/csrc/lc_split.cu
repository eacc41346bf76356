// lc_split.cu -- split-precision tensor-core tier, LC_F64_SPLIT.
#include "lc_internal.cuh"

size_t lc_split_bytes(const lc_plan_s*) { return 0; }
lc_status lc_split_prepare(lc_plan, char*, size_t, cudaStream_t) { return LC_ERR_UNSUPPORTED; }
lc_status lc_exec_split(lc_plan, const void*, void*, int64_t, int64_t, int64_t, int64_t, cudaStream_t, int) {
  return LC_ERR_UNSUPPORTED;
}
int lc_exec_split_launches(const lc_plan_s*) { return 0; }

extern "C" {
lc_status lc_plan_workspace_size_ragged(const int64_t*, int64_t, lc_direction, lc_dtype, const lc_plan_options*,
                                        size_t*) {
  return LC_ERR_UNSUPPORTED;
}
lc_status lc_plan_create_ragged(lc_plan*, const int64_t*, int64_t, lc_direction, lc_dtype, const lc_plan_options*,
                                void*, size_t, lc_stream) {
  return LC_ERR_UNSUPPORTED;
}
}
