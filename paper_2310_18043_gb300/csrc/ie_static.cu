// ie_apply_G_static: G(V) = sum_i w_i K_i^{-1} B V with the call's scratch in a file-scope
// device array instead of memory allocated by the library. For callers that must not make
// the library allocate device memory at call time (a host application whose allocator owns
// the device memory budget, or a latency-critical loop that cannot take cudaMalloc's
// implicit synchronisation). The kernels are the same as ie_apply_G's.
#include <mutex>

#include "ie_internal.cuh"

namespace {
constexpr size_t kScratchElems = IE_STATIC_SCRATCH_BYTES / sizeof(cplx);

// One array per device that loads the library, kept until the process exits.
static __device__ __align__(256) cplx g_static_scratch[kScratchElems];

// Device address of g_static_scratch, looked up once per device. In host code the symbol
// is only a host-side handle: it must never be passed to a kernel as a pointer.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
cplx* g_dev_ptr[kMaxDevices] = {};

cudaError_t scratch_ptr_for(int dev, cplx** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);   // device `dev` is current
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = (cplx*)p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

// Device memory of GPU `dev` itself (a block on another GPU would be read through a peer
// mapping), or managed memory.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}
}  // namespace

extern "C" ie_status ie_apply_G_static(ie_handle h, const ie_complex* d_V, int64_t ldv, int32_t k,
                                       ie_complex* d_GV, int64_t ldgv, void* stream) {
  IeFactorsView f;
  if (!ie_internal_factors(h, &f) || !d_V || !d_GV || k < 1 || ldv < f.n || ldgv < f.n)
    return IE_ERR_ARG;
  if (!f.L64 || !f.U64) return IE_ERR_ARG;   // complex128 handles only (precision = 0)
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != f.dev) return IE_ERR_ARG;
  if (!on_device(d_V, f.dev) || !on_device(d_GV, f.dev)) return IE_ERR_ARG;
  // scratch: B V (n x k) followed by the q per-pole solve buffers (n x k each)
  const unsigned long long need =
      (unsigned long long)(f.q + 1) * (unsigned long long)f.n * (unsigned long long)k;
  if (need > kScratchElems) return IE_ERR_SCRATCH_LIMIT;
  cplx* base = nullptr;
  cudaError_t e = scratch_ptr_for(f.dev, &base);
  if (e != cudaSuccess) return IE_ERR_CUDA;
  cplx* BV = base;
  cplx* Xp = base + (int64_t)f.n * k;
  cudaStream_t s = (cudaStream_t)stream;
  // every element of BV and Xp read below is written first by this call
  launch_spmv(f.P, make_double2(0, 0), make_double2(1, 0), (const cplx*)d_V, ldv, nullptr, k, BV,
              f.n, s);
  e = launch_band_solve(f.q, f.n, f.kl, f.n_pad, f.L64, f.U64, f.piv, f.dinv, f.Tb, f.Hb, f.Ub,
                        f.weights, BV, f.n, k, Xp, f.n, f.n * (int64_t)k, f.status, s);
  if (e != cudaSuccess) return IE_ERR_CUDA;
  launch_pole_sum(f.q, f.n, k, Xp, f.n, f.n * (int64_t)k, (cplx*)d_GV, ldgv, s);
  if (cudaGetLastError() != cudaSuccess) return IE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return IE_ERR_CUDA;
  int st[ST_COUNT];
  if (cudaMemcpy(st, f.status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return IE_ERR_CUDA;
  return st[ST_TIMEOUT] ? IE_ERR_TIMEOUT : IE_OK;
}
