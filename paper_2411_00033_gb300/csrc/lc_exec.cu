// lc_exec.cu -- Algorithm 4 on the CUDA cores in FP64 (LC_F64) and FP32
// (LC_F32), forward and transposed (lc_adjoint).  The kernels live in
// lc_exec_kernels.cuh.
#include "lc_exec_kernels.cuh"

using namespace lc_exec;


int lc_exec_cuda_cores_launches(const lc_plan_s* p) {
  return launches_for<double>(p->g.L, p->leaf_depth, p->chunk_depth, p->batch);
}

lc_status lc_exec_cuda_cores(lc_plan p, const void* in, void* out, int64_t ib, int64_t ie, int64_t ob,
                             int64_t oe, cudaStream_t st, int adjoint) {
  if (p->ragged) return LC_ERR_UNSUPPORTED;
  if (p->dtype == LC_F64) {
    Args<double> a;
    a.in = static_cast<const double*>(in);
    a.out = static_cast<double*>(out);
    a.ib = ib; a.ie = ie; a.ob = ob; a.oe = oe;
    a.n = p->g.n; a.N = p->g.N; a.L = p->g.L; a.s = p->g.s; a.nseg = p->g.nseg;
    a.batch = p->batch; a.dir = int(p->dir);
    a.t = lc_tables<double>{p->lam, p->lam2, p->T, p->B, p->Ahat, p->W, p->Cc, p->err, p->opt.debug_flags};
    return run<double>(p, a, st, adjoint);
  } else {
    Args<float> a;
    a.in = static_cast<const float*>(in);
    a.out = static_cast<float*>(out);
    a.ib = ib; a.ie = ie; a.ob = ob; a.oe = oe;
    a.n = p->g.n; a.N = p->g.N; a.L = p->g.L; a.s = p->g.s; a.nseg = p->g.nseg;
    a.batch = p->batch; a.dir = int(p->dir);
    a.t = lc_tables<float>{p->lamf, p->lam2f, p->Tf, p->Bf, p->Ahatf, p->Wf, p->Ccf, p->err, p->opt.debug_flags};
    return run<float>(p, a, st, adjoint);
  }
}
