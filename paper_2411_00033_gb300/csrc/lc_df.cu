// lc_df.cu -- double-float (FP32 pair) tier, LC_F64_DF.
#include "lc_internal.cuh"

size_t lc_df_bytes(const lc_geom&, int64_t) { return 0; }
lc_status lc_df_prepare(lc_plan, cudaStream_t) { return LC_ERR_UNSUPPORTED; }
lc_status lc_exec_df(lc_plan, const void*, void*, int64_t, int64_t, int64_t, int64_t, cudaStream_t, int) {
  return LC_ERR_UNSUPPORTED;
}
