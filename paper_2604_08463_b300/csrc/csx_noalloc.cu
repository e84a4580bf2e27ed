// csx_spectral_grad_noalloc: the likelihood + adjoint gradient of csx_spectral_grad for callers
// that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: applications whose device memory is owned by
// their own pool allocator (a cudaMalloc behind its back can fail once the pool holds the memory,
// or fragment it), and latency-critical loops with a fixed memory budget, where a first-call
// allocation (and the device synchronisation cudaMalloc/cudaFree can imply) is not acceptable.
// This entry point keeps the only scratch csx_spectral_grad needs -- the per-problem SED tables --
// in a statically sized device array that is part of the loaded library, so the call allocates
// nothing. Inputs and outputs are still the caller's buffers.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "csx_host.h"

namespace csx {
namespace {

// Capacity of the static table buffer, in floats: problems x (K_d + 2 K_T + K_s) x 16 must fit.
constexpr size_t kNoAllocTableFloats = size_t(1) << 20;  // 4 MiB

// Lives on every device that loads the library, until the process exits. Every call on a device
// shares it and it keeps the last call's contents; calls whose work overlaps on that device race.
static __device__ __align__(256) float g_noalloc_tables[kNoAllocTableFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_dev_ptr[kMaxDevices] = {};

// Device address of g_noalloc_tables on the current device. In host code the symbol's name is only
// a host-side handle, so the address is looked up with that device current: on the first call on
// the device, and again on every call made while `stream` is not capturing, so that a context that
// was torn down and re-created (cudaDeviceReset) gets its own module's address. During a capture
// the address found by an earlier call is used; the first call on a device must not be captured.
int table_buffer(cudaStream_t stream, float** out) {
  int dev = 0;
  CSX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CSX_EINVAL, "device index out of range");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CSX_CUDA(cudaStreamIsCapturing(stream, &cap));
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_dev_ptr[dev]) {
    if (cap != cudaStreamCaptureStatusNone)
      return fail(CSX_EINVAL, "csx_spectral_grad_noalloc: the first call on a device must not be "
                              "made during a stream capture");
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tables);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_tables)");
    g_dev_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_dev_ptr[dev];
  return CSX_OK;
}

}  // namespace
}  // namespace csx

using namespace csx;

extern "C" int csx_spectral_grad_noalloc(const csx_model* m, const csx_sky* sky,
                                         const int32_t* labels, const int32_t K[3],
                                         int32_t nprob, const float* beta, double* L,
                                         float* grad, void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (!K) return fail(CSX_EINVAL, "K is NULL");
  if ((rc = check_K(K))) return rc;
  if ((rc = check_align(labels, 4, "labels")) || (rc = check_align(beta, 4, "beta")) ||
      (rc = check_align(L, 8, "L")) || (rc = check_align(grad, 4, "grad")))
    return rc;
  if (nprob < 0 || nprob > sky->nreal) return fail(CSX_EINVAL, "nprob must be in [0, sky->nreal]");
  if (nprob == 0) return CSX_OK;
  if (!beta || !L || !grad || (sky->npix > 0 && !labels))
    return fail(CSX_EINVAL, "beta, L, grad and labels must not be NULL");
  // sizes in 64-bit arithmetic (K_j <= CSX_MAX_K keeps P and the row count within int)
  const long long P = (long long)K[0] + K[1] + K[2];
  const long long rows = (long long)K[0] + 2LL * K[1] + K[2];
  const long long need = (long long)nprob * rows * NB;
  if (need > (long long)kNoAllocTableFloats)
    return fail(CSX_EINVAL, "csx_spectral_grad_noalloc: nprob x (K_d + 2 K_T + K_s) x 16 = " +
                                std::to_string(need) + " table floats exceed the static buffer of " +
                                std::to_string(kNoAllocTableFloats) +
                                "; split the problems over several calls or use csx_spectral_grad");
  cudaStream_t s = (cudaStream_t)stream;
  float* tables = nullptr;
  if ((rc = table_buffer(s, &tables))) return rc;
  const Bands b = make_bands(*m);
  // the tables are fully rewritten; L and grad are accumulated and so start from zero
  if ((rc = launch_tables(b, nprob, K[0], K[1], K[2], beta, tables, s))) return rc;
  CSX_CUDA(cudaMemsetAsync(L, 0, (size_t)nprob * sizeof(double), s));
  CSX_CUDA(cudaMemsetAsync(grad, 0, (size_t)nprob * (size_t)P * sizeof(float), s));
  if (sky->npix == 0) return CSX_OK;
  SpecArgs a;
  std::memset(&a, 0, sizeof(a));
  a.bands = b;
  a.npix = sky->npix;
  a.nprob = nprob;
  a.Kd = K[0];
  a.KT = K[1];
  a.Ks = K[2];
  a.P = (int)P;
  a.rows = (int)rows;
  a.noise_kind = sky->noise_kind;
  a.d = sky->d;
  a.w = sky->w;
  a.ninv_pix = sky->ninv_pix;
  for (int f = 0; f < NB; ++f) a.ninv_band[f] = (f < m->nfreq) ? sky->ninv_band[f] : 0.f;
  a.labels = labels;
  a.beta = beta;
  a.tables = tables;
  a.L = L;
  a.grad = grad;
  return launch_spectral(a, true, s);
}
