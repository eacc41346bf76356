// lc_noalloc.cu -- a transform entry point that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc themselves or let a
// library do it -- for example plugins inside a host application whose memory
// pool owns all device memory and offers no allocation hook, latency-critical
// loops where cudaMalloc's implicit device-wide synchronisation would stall
// other streams, and deployments that reserve every byte of device memory at
// load time and forbid allocation afterwards.  lc_plan_create needs a
// caller-provided workspace; this entry point needs none.
//
// How: the direct O(n^2) sum over the whole upper triangle (the near-field
// band of lc_execute extended to every column), with its scratch -- the table
// of Lambda(k) (L2C) or of the C2L factors u_k, v_m -- in a file-scope
// __device__ array of LC_STATIC_MAX_N x 2 doubles (256 KiB).  Every GPU that
// loads the library holds that array until the process exits.
#include <mutex>

#include "lc_internal.cuh"

// Plan-builder kernels of lc_plan.cu, reused to fill the table.
__global__ void k_plan_lambda(int64_t N, double* __restrict__ lam);
__global__ void k_plan_c2l_tables(int64_t N, double* __restrict__ u, double* __restrict__ v);

static __device__ __align__(256) double lc_static_scratch[2 * LC_STATIC_MAX_N];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of lc_static_scratch on the current device; looked up once
// per device (the name is only a host-side stand-in in host code).
lc_status scratch_address(double** out) {
  int dev = 0;
  LC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return LC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    LC_CUDA_TRY(cudaGetSymbolAddress(&p, lc_static_scratch));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LC_OK;
}

// One thread per output row i: z_i = sum over j >= i, j - i even, of M_ij x_j,
// with M = C^{-1}A (L2C, eq:hik then Step 7) or L(i,j) of eq:Lxymod (C2L,
// factorised as (2i+1) j u_k v_{i+k}, L(0,0) = 1).  tab holds [u | v] (C2L)
// or lambda in both halves' roles (L2C: u = v = lambda).
__global__ void k_direct_static(const double* __restrict__ tab_u, const double* __restrict__ tab_v, int dir,
                                int64_t n, int64_t batch, const double* __restrict__ in, double* __restrict__ out,
                                int64_t ib, int64_t ie, int64_t ob, int64_t oe) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
    const double* f = in + b * ib;
    double acc = 0.0;
    int64_t k = 0;
    if (dir == LC_L2C) {
      for (int64_t j = i; j < n; j += 2, ++k) acc = fma(tab_u[k] * tab_v[i + k], f[j * ie], acc);
      acc *= (i == 0) ? 0.31830988618379067154 : 0.63661977236758134308;  // C^{-1}
    } else {
      for (int64_t j = i; j < n; j += 2, ++k) acc = fma(tab_u[k] * tab_v[i + k], double(j) * f[j * ie], acc);
      acc *= double(2 * i + 1);
      if (i == 0) acc += f[0];
    }
    out[b * ob + i * oe] = acc;
  }
}

}  // namespace

extern "C" lc_status lc_direct_static(lc_direction direction, int64_t n, int64_t batch, const double* in,
                                      double* out, int64_t in_batch_stride, int64_t in_elem_stride,
                                      int64_t out_batch_stride, int64_t out_elem_stride, lc_stream stream) {
  if (direction != LC_L2C && direction != LC_C2L) return LC_ERR_INVALID_ARG;
  if (n < 1 || n > LC_STATIC_MAX_N || batch < 1 || batch > (int64_t(1) << 31)) return LC_ERR_INVALID_ARG;
  if (!in || !out || in == static_cast<const double*>(out)) return LC_ERR_INVALID_ARG;
  if (in_batch_stride < 0 || in_elem_stride < 0 || out_batch_stride < 0 || out_elem_stride < 0)
    return LC_ERR_INVALID_ARG;
  // as lc_execute: a zero output stride would make several rows (or vectors)
  // write one address
  if ((out_elem_stride == 0 && n > 1) || (out_batch_stride == 0 && batch > 1)) return LC_ERR_INVALID_ARG;
  double* scratch = nullptr;
  lc_status st = scratch_address(&scratch);
  if (st != LC_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* u = scratch;
  double* v = scratch + LC_STATIC_MAX_N;
  // The table for this n is rewritten in full before it is read: no entry
  // needs to start at zero, whatever an earlier call left in the array.
  if (direction == LC_L2C) {
    k_plan_lambda<<<unsigned((n + 7) / 8 + 255) / 256, 256, 0, s>>>(n, u);
    LC_LAUNCH_CHECK();
    v = u;
  } else {
    k_plan_lambda<<<unsigned((n + 7) / 8 + 255) / 256, 256, 0, s>>>(n, v);
    LC_LAUNCH_CHECK();
    k_plan_c2l_tables<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, u, v);
    LC_LAUNCH_CHECK();
  }
  dim3 grid(unsigned((n + 127) / 128), unsigned(batch < 65535 ? batch : 65535));
  k_direct_static<<<grid, 128, 0, s>>>(u, v, int(direction), n, batch, in, out, in_batch_stride, in_elem_stride,
                                        out_batch_stride, out_elem_stride);
  LC_LAUNCH_CHECK();
  return LC_OK;
}
