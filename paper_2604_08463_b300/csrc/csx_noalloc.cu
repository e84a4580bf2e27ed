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

#include <cmath>
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
// a host-side handle, so the address is looked up once per device (with that device current).
int table_buffer(float** out) {
  int dev = 0;
  CSX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CSX_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
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
  if (!m) return fail(CSX_EINVAL, "model is NULL");
  if (m->nfreq < 1 || m->nfreq > 15) return fail(CSX_EINVAL, "nfreq must be in 1..15");
  if (m->units != 0 && m->units != 1) return fail(CSX_EINVAL, "units must be 0 (K_CMB) or 1 (RJ)");
  if (!(m->nu0_dust_ghz > 0) || !(m->nu0_sync_ghz > 0) || (m->units == 0 && !(m->t_cmb > 0)))
    return fail(CSX_EINVAL, "reference frequencies and t_cmb must be > 0");
  for (int f = 0; f < m->nfreq; ++f)
    if (!(m->nu_ghz[f] > 0)) return fail(CSX_EINVAL, "band frequencies must be > 0");
  if (!sky) return fail(CSX_EINVAL, "sky is NULL");
  if (sky->npix < 0 || sky->nreal < 0) return fail(CSX_EINVAL, "npix and nreal must be >= 0");
  if (sky->noise_kind < 0 || sky->noise_kind > 2) return fail(CSX_EINVAL, "unknown noise_kind");
  if (sky->npix > 0 && sky->nreal > 0 && !sky->d) return fail(CSX_EINVAL, "sky->d is NULL");
  if (sky->noise_kind == CSX_NOISE_SEPARABLE && sky->npix > 0 && !sky->w)
    return fail(CSX_EINVAL, "separable noise needs sky->w");
  if (sky->noise_kind == CSX_NOISE_PERPIXEL && sky->npix > 0 && !sky->ninv_pix)
    return fail(CSX_EINVAL, "per-pixel noise needs sky->ninv_pix");
  {
    int rc0;
    if ((rc0 = check_align(sky->d, 16, "sky->d")) || (rc0 = check_align(sky->ninv_pix, 16, "sky->ninv_pix")) ||
        (rc0 = check_align(sky->w, 4, "sky->w")) || (rc0 = check_align(labels, 4, "labels")) ||
        (rc0 = check_align(beta, 4, "beta")) || (rc0 = check_align(L, 8, "L")) ||
        (rc0 = check_align(grad, 4, "grad")))
      return rc0;
  }
  if (sky->noise_kind != CSX_NOISE_PERPIXEL)
    for (int f = 0; f < m->nfreq; ++f)
      if (!(sky->ninv_band[f] >= 0.f) || !std::isfinite(sky->ninv_band[f]))
        return fail(CSX_EINVAL, "ninv_band must be finite and >= 0");
  if (!K || K[0] < 1 || K[1] < 1 || K[2] < 1) return fail(CSX_EINVAL, "every K_j must be >= 1");
  if (nprob < 0 || nprob > sky->nreal) return fail(CSX_EINVAL, "nprob must be in [0, sky->nreal]");
  if (nprob == 0) return CSX_OK;
  if (!beta || !L || !grad || (sky->npix > 0 && !labels))
    return fail(CSX_EINVAL, "beta, L, grad and labels must not be NULL");
  const int P = K[0] + K[1] + K[2];
  const int rows = K[0] + 2 * K[1] + K[2];
  const size_t need = (size_t)nprob * rows * NB;
  if (need > kNoAllocTableFloats)
    return fail(CSX_EINVAL, "csx_spectral_grad_noalloc: nprob x (K_d + 2 K_T + K_s) x 16 = " +
                                std::to_string(need) + " table floats exceed the static buffer of " +
                                std::to_string(kNoAllocTableFloats) +
                                "; split the problems over several calls or use csx_spectral_grad");
  float* tables = nullptr;
  int rc = table_buffer(&tables);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Bands b = make_bands(*m);
  // the tables are fully rewritten; L and grad are accumulated and so start from zero
  if ((rc = launch_tables(b, nprob, K[0], K[1], K[2], beta, tables, s))) return rc;
  CSX_CUDA(cudaMemsetAsync(L, 0, (size_t)nprob * sizeof(double), s));
  CSX_CUDA(cudaMemsetAsync(grad, 0, (size_t)nprob * P * sizeof(float), s));
  if (sky->npix == 0) return CSX_OK;
  SpecArgs a;
  std::memset(&a, 0, sizeof(a));
  a.bands = b;
  a.npix = sky->npix;
  a.nprob = nprob;
  a.Kd = K[0];
  a.KT = K[1];
  a.Ks = K[2];
  a.P = P;
  a.rows = rows;
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
