// lc_exec.cu -- Algorithm 4 on the CUDA cores in FP64 (LC_F64) and FP32
// (LC_F32), forward and transposed (lc_adjoint).  The kernels live in
// lc_exec_kernels.cuh.
#include "lc_exec_kernels.cuh"

using namespace lc_exec;


int lc_exec_cuda_cores_launches(const lc_plan_s* p) {
  // + the exponent pre-pass of the double-float tier's far-field chain
  return launches_for<double>(p->g.L, p->leaf_depth, p->chunk_depth, p->batch) +
         (p->dtype == LC_F64_DF && p->g.L > 0 ? 1 : 0);
}

lc_status lc_exec_cuda_cores(lc_plan p, const void* in, void* out, const lc_layout& lay, cudaStream_t st,
                             int adjoint) {
  if (p->ragged) return LC_ERR_UNSUPPORTED;
  if (p->dtype == LC_F64) {
    Args<double> a;
    a.in = static_cast<const double*>(in);
    a.out = static_cast<double*>(out);
    a.ib = lay.ib; a.ie = lay.ie; a.ob = lay.ob; a.oe = lay.oe;
    a.inner = lay.inner; a.iob = lay.iob; a.oob = lay.oob;
    a.n = p->g.n; a.N = p->g.N; a.L = p->g.L; a.s = p->g.s; a.nseg = p->g.nseg;
    a.batch = p->batch; a.dir = int(p->dir); a.two_alpha = p->geg.two_alpha; a.nodal = p->opt.nodal;
    a.trigger = 0;
    a.t = lc_tables<double>{p->lam, p->lam2, p->T, p->B, p->Ahat, p->W, p->Cc, p->err, p->opt.debug_flags};
    a.xe = a.xe_part = nullptr;
    a.xe_cnt = nullptr;
    return run<double>(p, a, st, adjoint);
  } else {
    Args<float> a;
    a.in = static_cast<const float*>(in);
    a.out = static_cast<float*>(out);
    a.ib = lay.ib; a.ie = lay.ie; a.ob = lay.ob; a.oe = lay.oe;
    a.inner = lay.inner; a.iob = lay.iob; a.oob = lay.oob;
    a.n = p->g.n; a.N = p->g.N; a.L = p->g.L; a.s = p->g.s; a.nseg = p->g.nseg;
    a.batch = p->batch; a.dir = int(p->dir); a.two_alpha = p->geg.two_alpha; a.nodal = p->opt.nodal;
    a.trigger = 0;
    a.t = lc_tables<float>{p->lamf, p->lam2f, p->Tf, p->Bf, p->Ahatf, p->Wf, p->Ccf, p->err, p->opt.debug_flags};
    a.xe = a.xe_part = nullptr;
    a.xe_cnt = nullptr;
    return run<float>(p, a, st, adjoint);
  }
}
