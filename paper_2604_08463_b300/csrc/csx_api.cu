// C ABI of the csx library (include/csx.h): argument checks, per-device scratch, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>
#include <chrono>
#include <cstdio>
#include <cstdlib>

#include "csx_host.h"

namespace csx {

// ------------------------------------------------------------------------------ tracing --------
// CSX_TRACE=1 in the environment: every traced span synchronises its stream and prints its GPU
// time (CUDA events) and host time to stderr. Off by default; diagnostic only.
static bool trace_on() {
  static const bool on = [] {
    const char* e = std::getenv("CSX_TRACE");
    return e && *e && *e != '0';
  }();
  return on;
}

struct TraceSpan {
  const char* name;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  std::chrono::steady_clock::time_point t0;
  TraceSpan(const char* n, cudaStream_t st) : name(n), s(st) {
    if (!trace_on()) return;
    t0 = std::chrono::steady_clock::now();
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  ~TraceSpan() {
    if (!a) return;
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double host =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::fprintf(stderr, "csx trace: %-24s gpu %9.3f ms  host %9.3f ms\n", name, ms, host);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// ------------------------------------------------------------------------------ errors ---------
static thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? CSX_ENOMEM : CSX_ECUDA;
}

// ------------------------------------------------------------------------------ scratch --------
namespace {
constexpr int kMaxDev = 64;
struct Buf {
  void* p = nullptr;
  size_t n = 0;
};
std::mutex g_mu;
Buf g_buf[kMaxDev][SCR_COUNT];
}  // namespace

void* scratch(ScratchId id, size_t bytes, int* err) {
  int dev = 0;
  *err = CSX_OK;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    *err = fail(CSX_ECUDA, "cudaGetDevice failed");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  Buf& b = g_buf[dev][id];
  if (bytes == 0) bytes = 1;
  if (b.n < bytes) {
    if (b.p) {
      cudaError_t e = cudaFree(b.p);
      b.p = nullptr;
      b.n = 0;
      if (e != cudaSuccess) {
        *err = cuda_fail(e, "cudaFree(scratch)");
        return nullptr;
      }
    }
    const size_t want = bytes + bytes / 4;  // headroom against repeated growth
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
      b.p = nullptr;
      *err = cuda_fail(e, "cudaMalloc(scratch)");
      return nullptr;
    }
    b.n = want;
  }
  return b.p;
}

void scratch_release_all() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < SCR_COUNT; ++i) {
    if (g_buf[dev][i].p) cudaFree(g_buf[dev][i].p);
    g_buf[dev][i] = Buf();
  }
}

// ------------------------------------------------------------------------------ model ----------
// RJ -> K_CMB factor u(nu) = (e^x - 1)^2 / (x^2 e^x), x = h nu / (k T_CMB).
static double rj_to_kcmb(double nu_ghz, double t_cmb) {
  const double h_over_k = 6.62607015e-34 / 1.380649e-23 * 1e9;  // K per GHz
  const double x = h_over_k * nu_ghz / t_cmb;
  const double em1 = std::expm1(x);
  return em1 * em1 / (x * x * std::exp(x));
}

Bands make_bands(const csx_model& m) {
  Bands b;
  std::memset(&b, 0, sizeof(b));
  const double h_over_k = 6.62607015e-34 / 1.380649e-23 * 1e9;
  b.nf = m.nfreq;
  b.xk0 = (float)(h_over_k * m.nu0_dust_ghz);
  const bool kcmb = (m.units == 0);
  const double ud = kcmb ? rj_to_kcmb(m.nu0_dust_ghz, m.t_cmb) : 1.0;
  const double us = kcmb ? rj_to_kcmb(m.nu0_sync_ghz, m.t_cmb) : 1.0;
  for (int f = 0; f < m.nfreq; ++f) {
    const double nu = m.nu_ghz[f];
    const double u = kcmb ? rj_to_kcmb(nu, m.t_cmb) : 1.0;
    b.lnd[f] = (float)std::log(nu / m.nu0_dust_ghz);
    b.lns[f] = (float)std::log(nu / m.nu0_sync_ghz);
    b.xk[f] = (float)(h_over_k * nu);
    b.cd[f] = (float)(nu / m.nu0_dust_ghz * u / ud);
    b.cs[f] = (float)(u / us);
  }
  return b;
}

Bands64 make_bands64(const csx_model& m) {
  Bands64 b;
  std::memset(&b, 0, sizeof(b));
  const double h_over_k = 6.62607015e-34 / 1.380649e-23 * 1e9;
  b.nf = m.nfreq;
  b.xk0 = h_over_k * m.nu0_dust_ghz;
  const bool kcmb = (m.units == 0);
  const double ud = kcmb ? rj_to_kcmb(m.nu0_dust_ghz, m.t_cmb) : 1.0;
  const double us = kcmb ? rj_to_kcmb(m.nu0_sync_ghz, m.t_cmb) : 1.0;
  for (int f = 0; f < m.nfreq; ++f) {
    const double nu = m.nu_ghz[f];
    const double u = kcmb ? rj_to_kcmb(nu, m.t_cmb) : 1.0;
    b.lnd[f] = std::log(nu / m.nu0_dust_ghz);
    b.lns[f] = std::log(nu / m.nu0_sync_ghz);
    b.xk[f] = h_over_k * nu;
    b.cd[f] = nu / m.nu0_dust_ghz * u / ud;
    b.cs[f] = u / us;
  }
  return b;
}

// ------------------------------------------------------------------------------ checks ---------
int check_model(const csx_model* m) {
  if (!m) return fail(CSX_EINVAL, "model is NULL");
  if (m->nfreq < 1 || m->nfreq > 15) return fail(CSX_EINVAL, "nfreq must be in 1..15");
  if (m->units != 0 && m->units != 1) return fail(CSX_EINVAL, "units must be 0 (K_CMB) or 1 (RJ)");
  if (!(m->nu0_dust_ghz > 0) || !(m->nu0_sync_ghz > 0)) return fail(CSX_EINVAL, "reference frequencies must be > 0");
  if (m->units == 0 && !(m->t_cmb > 0)) return fail(CSX_EINVAL, "t_cmb must be > 0 for K_CMB units");
  for (int f = 0; f < m->nfreq; ++f)
    if (!(m->nu_ghz[f] > 0)) return fail(CSX_EINVAL, "band frequencies must be > 0");
  return CSX_OK;
}

int check_align(const void* p, size_t align, const char* what) {
  if (p && (reinterpret_cast<uintptr_t>(p) % align) != 0)
    return fail(CSX_EINVAL, std::string(what) + " must be " + std::to_string(align) +
                                "-byte aligned");
  return CSX_OK;
}

#define CSX_ALIGN(p, n)                                    \
  do {                                                     \
    const int rc_ = check_align((p), (n), #p);             \
    if (rc_) return rc_;                                   \
  } while (0)

int check_sky(const csx_sky* s, int nfreq) {
  if (!s) return fail(CSX_EINVAL, "sky is NULL");
  // pixel rows are read as 16-byte vectors (and staged by tensor copies): 16-byte alignment
  int rc;
  if ((rc = check_align(s->d, 16, "sky->d")) || (rc = check_align(s->ninv_pix, 16, "sky->ninv_pix")) ||
      (rc = check_align(s->w, 4, "sky->w")))
    return rc;
  if (s->npix < 0 || s->nreal < 0) return fail(CSX_EINVAL, "npix and nreal must be >= 0");
  if (s->npix > 0 && s->nreal > 0 && !s->d) return fail(CSX_EINVAL, "sky->d is NULL");
  if (s->noise_kind < 0 || s->noise_kind > 2) return fail(CSX_EINVAL, "unknown noise_kind");
  if (s->noise_kind == CSX_NOISE_SEPARABLE && !s->w && s->npix > 0)
    return fail(CSX_EINVAL, "separable noise needs sky->w");
  if (s->noise_kind == CSX_NOISE_PERPIXEL && !s->ninv_pix && s->npix > 0)
    return fail(CSX_EINVAL, "per-pixel noise needs sky->ninv_pix");
  if (s->noise_kind != CSX_NOISE_PERPIXEL) {
    for (int f = 0; f < nfreq; ++f)
      if (!(s->ninv_band[f] >= 0.f) || !std::isfinite(s->ninv_band[f]))
        return fail(CSX_EINVAL, "ninv_band must be finite and >= 0");
  }
  return CSX_OK;
}

int check_K(const int32_t* K) {
  for (int j = 0; j < 3; ++j)
    if (K[j] < 1 || K[j] > CSX_MAX_K)
      return fail(CSX_EINVAL, "every K_j must be in [1, " + std::to_string(CSX_MAX_K) + "]");
  return CSX_OK;
}

static void copy_band_weights(const csx_sky* s, int nfreq, float* out) {
  for (int f = 0; f < NB; ++f) out[f] = (f < nfreq) ? s->ninv_band[f] : 0.f;
}

}  // namespace csx

using namespace csx;

extern "C" {

const char* csx_version(void) { return "csx 0.1.0 (sm_103a)"; }

const char* csx_last_error(void) { return g_err.c_str(); }

int csx_release(void) {
  CSX_CUDA(cudaDeviceSynchronize());
  scratch_release_all();
  return CSX_OK;
}

int csx_device_status(void* stream) {
  unsigned n = 0;
  int rc = device_timeouts((cudaStream_t)stream, &n);
  if (rc) return rc;
  if (n) return fail(CSX_ETIMEOUT, std::to_string(n) + " bounded device wait(s) gave up since the "
                                   "last check (the affected problems' L is NaN)");
  return CSX_OK;
}

int csx_stream_schedule(int32_t tile, int32_t stages, int32_t* current) {
  if (tile != -1 || stages != -1) {
    const int rc = set_stream_schedule(tile, stages);
    if (rc) return rc;
  }
  if (current) get_stream_schedule(&current[0], &current[1]);
  return CSX_OK;
}

int csx_fit_defaults(csx_fit_opts* o) {
  if (!o) return fail(CSX_EINVAL, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->max_iter = 500;
  o->history = 8;
  o->max_ls = 20;
  o->path = CSX_PATH_AUTO;
  o->grad_mode = CSX_GRAD_ADJOINT;
  o->threads = 0;
  const float lo[3] = {0.5f, 5.f, -5.f}, hi[3] = {3.f, 60.f, -1.f}, xt[3] = {1e-4f, 1e-3f, 1e-4f};
  for (int j = 0; j < 3; ++j) {
    o->lower[j] = lo[j];
    o->upper[j] = hi[j];
    o->xtol[j] = xt[j];
  }
  o->fd_step = 1e-3f;
  o->solver = CSX_SOLVER_LBFGS;
  o->topk = 0.f;
  return CSX_OK;
}

int csx_mixing(const csx_model* m, int32_t n, const float* beta, float* A, float* dA, void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if (n < 0) return fail(CSX_EINVAL, "n must be >= 0");
  if (n > 0 && (!beta || !A)) return fail(CSX_EINVAL, "beta and A must not be NULL");
  CSX_ALIGN(beta, 4);
  CSX_ALIGN(A, 4);
  CSX_ALIGN(dA, 4);
  return launch_mixing(make_bands(*m), n, beta, A, dA, (cudaStream_t)stream);
}

static int spectral_common(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                           const int32_t K[3], int32_t nprob, const float* beta, double* L,
                           float* grad, bool want_grad, void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (!K) return fail(CSX_EINVAL, "K is NULL");
  if ((rc = check_K(K))) return rc;
  if (nprob < 0 || nprob > sky->nreal) return fail(CSX_EINVAL, "nprob must be in [0, sky->nreal]");
  if (nprob == 0) return CSX_OK;
  if (!beta) return fail(CSX_EINVAL, "beta is NULL");
  if (sky->npix > 0 && !labels) return fail(CSX_EINVAL, "labels is NULL");
  if (want_grad && !grad) return fail(CSX_EINVAL, "grad is NULL");
  if (!want_grad && !L) return fail(CSX_EINVAL, "L is NULL");
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(beta, 4);
  CSX_ALIGN(L, 8);
  CSX_ALIGN(grad, 4);
  cudaStream_t s = (cudaStream_t)stream;
  const int P = K[0] + K[1] + K[2];
  const int rows = K[0] + 2 * K[1] + K[2];
  const Bands b = make_bands(*m);
  float* tables = (float*)scratch(SCR_TABLES, (size_t)nprob * rows * NB * sizeof(float), &rc);
  if (rc) return rc;
  double* Lbuf = L;
  if (!Lbuf) {
    Lbuf = (double*)scratch(SCR_MISC, (size_t)nprob * sizeof(double), &rc);
    if (rc) return rc;
  }
  if ((rc = launch_tables(b, nprob, K[0], K[1], K[2], beta, tables, s))) return rc;
  CSX_CUDA(cudaMemsetAsync(Lbuf, 0, (size_t)nprob * sizeof(double), s));
  if (want_grad) CSX_CUDA(cudaMemsetAsync(grad, 0, (size_t)nprob * P * sizeof(float), s));
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
  copy_band_weights(sky, m->nfreq, a.ninv_band);
  a.labels = labels;
  a.beta = beta;
  a.tables = tables;
  a.L = Lbuf;
  a.grad = want_grad ? grad : nullptr;
  if (sky->npix == 0) return CSX_OK;
  return launch_spectral(a, want_grad, s);
}

int csx_spectral_like(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                      const int32_t K[3], int32_t nprob, const float* beta, double* L, void* stream) {
  return spectral_common(m, sky, labels, K, nprob, beta, L, nullptr, false, stream);
}

int csx_spectral_grad(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                      const int32_t K[3], int32_t nprob, const float* beta, double* L, float* grad,
                      void* stream) {
  return spectral_common(m, sky, labels, K, nprob, beta, L, grad, true, stream);
}

struct csx_spectral_plan {
  int device;
  int npix;
  int K[3];
  int ncell;
  int* pcell;      // [npix] cell of each pixel
  int4* cell_lab;  // [ncell] (l_d, l_T, l_s, 0)
};

int csx_spectral_plan_create(int32_t npix, const int32_t* labels, const int32_t K[3], void* stream,
                             csx_spectral_plan** plan) {
  if (!plan) return fail(CSX_EINVAL, "plan is NULL");
  *plan = nullptr;
  if (npix < 0) return fail(CSX_EINVAL, "npix must be >= 0");
  if (!K) return fail(CSX_EINVAL, "K is NULL");
  int rc = check_K(K);
  if (rc) return rc;
  if (npix > 0 && !labels) return fail(CSX_EINVAL, "labels is NULL");
  CSX_ALIGN(labels, 4);
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  CSX_CUDA(cudaGetDevice(&dev));
  // temporaries of the cell sort: perm [npix], offsets [npix + 1], count, K
  int* tmp = nullptr;
  CSX_CUDA(cudaMalloc(&tmp, ((size_t)2 * npix + 8) * sizeof(int)));
  int* perm = tmp;
  int* off = tmp + npix;
  int* nc = off + npix + 1;
  int* Kd = nc + 1;
  int ncell = 0;
  auto cleanup = [&](int code) {
    cudaFree(tmp);
    return code;
  };
  if (cudaMemcpyAsync(Kd, K, 3 * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return cleanup(fail(CSX_ECUDA, "copy of K"));
  if (npix > 0 && (rc = launch_cells(npix, 1, labels, Kd, perm, off, nc, s))) return cleanup(rc);
  if (npix > 0) {
    if (cudaMemcpyAsync(&ncell, nc, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return cleanup(fail(CSX_ECUDA, "cell count"));
  }
  if (ncell < 0) return cleanup(fail(CSX_EINVAL, "a label is outside [0, K_j)"));
  csx_spectral_plan* p = new csx_spectral_plan();
  p->device = dev;
  p->npix = npix;
  for (int j = 0; j < 3; ++j) p->K[j] = K[j];
  p->ncell = ncell;
  void* mem = nullptr;
  const size_t lab_off = (((size_t)npix * sizeof(int)) + 15) & ~size_t(15);
  if (cudaMalloc(&mem, lab_off + (size_t)ncell * sizeof(int4) + 16) != cudaSuccess) {
    delete p;
    return cleanup(fail(CSX_ECUDA, "plan allocation"));
  }
  p->pcell = (int*)mem;
  p->cell_lab = (int4*)((char*)mem + lab_off);
  if ((rc = launch_plan_cells(npix, ncell, labels, perm, off, p->pcell, p->cell_lab, s)) ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaFree(mem);
    delete p;
    return cleanup(rc ? rc : fail(CSX_ECUDA, "plan construction"));
  }
  *plan = p;
  return cleanup(CSX_OK);
}

int csx_spectral_plan_destroy(csx_spectral_plan* plan) {
  if (!plan) return CSX_OK;
  int cur = 0;
  CSX_CUDA(cudaGetDevice(&cur));
  if (cur != plan->device) CSX_CUDA(cudaSetDevice(plan->device));
  const cudaError_t e = cudaFree(plan->pcell);
  if (cur != plan->device) cudaSetDevice(cur);
  delete plan;
  if (e != cudaSuccess) return cuda_fail(e, "cudaFree(plan)");
  return CSX_OK;
}

int csx_spectral_plan_ncell(const csx_spectral_plan* plan, int32_t* ncell) {
  if (!plan || !ncell) return fail(CSX_EINVAL, "NULL argument");
  *ncell = plan->ncell;
  return CSX_OK;
}

int csx_spectral_grad_plan(const csx_spectral_plan* plan, const csx_model* m, const csx_sky* sky,
                           int32_t nprob, const float* beta, double* L, float* grad, void* stream) {
  if (!plan) return fail(CSX_EINVAL, "plan is NULL");
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (sky->noise_kind == CSX_NOISE_PERPIXEL)
    return fail(CSX_EINVAL, "the cell plan needs homogeneous or separable noise");
  if (sky->npix != plan->npix) return fail(CSX_EINVAL, "sky->npix differs from the plan's npix");
  if (nprob < 0 || nprob > sky->nreal) return fail(CSX_EINVAL, "nprob must be in [0, sky->nreal]");
  if (nprob == 0) return CSX_OK;
  if (!beta || !L) return fail(CSX_EINVAL, "beta and L must not be NULL");
  CSX_ALIGN(beta, 4);
  CSX_ALIGN(L, 8);
  CSX_ALIGN(grad, 4);
  int dev = 0;
  CSX_CUDA(cudaGetDevice(&dev));
  if (dev != plan->device) return fail(CSX_EINVAL, "the plan belongs to another device");
  cudaStream_t s = (cudaStream_t)stream;
  const int* K = plan->K;
  const int P = K[0] + K[1] + K[2];
  const int rows = K[0] + 2 * K[1] + K[2];
  const Bands b = make_bands(*m);
  float* tables = (float*)scratch(SCR_TABLES, (size_t)nprob * rows * NB * sizeof(float), &rc);
  if (rc) return rc;
  float* ctab = (float*)scratch(SCR_CELLTAB, (size_t)nprob * plan->ncell * CELL_TAB * sizeof(float), &rc);
  if (rc) return rc;
  if ((rc = launch_tables(b, nprob, K[0], K[1], K[2], beta, tables, s))) return rc;
  CSX_CUDA(cudaMemsetAsync(L, 0, (size_t)nprob * sizeof(double), s));
  if (grad) CSX_CUDA(cudaMemsetAsync(grad, 0, (size_t)nprob * P * sizeof(float), s));
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
  copy_band_weights(sky, m->nfreq, a.ninv_band);
  a.beta = beta;
  a.tables = tables;
  a.L = L;
  a.grad = grad;
  a.pcell = plan->pcell;
  a.cell_lab = plan->cell_lab;
  a.ncell = plan->ncell;
  if ((rc = launch_cell_tables(a, grad != nullptr, ctab, s))) return rc;
  a.ctab = ctab;
  return launch_spectral(a, grad != nullptr, s);
}

int csx_spectral_grad_f64(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                          const int32_t K[3], int32_t nprob, const double* beta, double* L,
                          double* grad, void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (!K) return fail(CSX_EINVAL, "K is NULL");
  if ((rc = check_K(K))) return rc;
  if (nprob < 0 || nprob > sky->nreal) return fail(CSX_EINVAL, "nprob must be in [0, sky->nreal]");
  if (nprob == 0) return CSX_OK;
  if (!beta || !L) return fail(CSX_EINVAL, "beta and L must not be NULL");
  if (sky->npix > 0 && !labels) return fail(CSX_EINVAL, "labels is NULL");
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(beta, 8);
  CSX_ALIGN(L, 8);
  CSX_ALIGN(grad, 8);
  cudaStream_t s = (cudaStream_t)stream;
  const long long P = (long long)K[0] + K[1] + K[2];
  const long long rows = (long long)K[0] + 2LL * K[1] + K[2];
  double* tables = (double*)scratch(SCR_TABLES, (size_t)nprob * rows * NB * sizeof(double), &rc);
  if (rc) return rc;
  CSX_CUDA(cudaMemsetAsync(L, 0, (size_t)nprob * sizeof(double), s));
  if (grad) CSX_CUDA(cudaMemsetAsync(grad, 0, (size_t)nprob * P * sizeof(double), s));
  Spec64Args a;
  std::memset(&a, 0, sizeof(a));
  a.bands = make_bands64(*m);
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
  copy_band_weights(sky, m->nfreq, a.ninv_band);
  a.labels = labels;
  a.beta = beta;
  a.tables = tables;
  a.L = L;
  a.grad = grad;
  return launch_spectral64(a, grad != nullptr, s);
}

int csx_build_cells(int32_t npix, int32_t nconf, const int32_t* labels, const int32_t* K,
                    int32_t* perm, int32_t* cell_off, int32_t* ncell, void* stream) {
  if (npix < 0 || nconf < 0) return fail(CSX_EINVAL, "npix and nconf must be >= 0");
  if (nconf == 0) return CSX_OK;
  if (!K || !perm || !cell_off || !ncell || (npix > 0 && !labels))
    return fail(CSX_EINVAL, "NULL argument");
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(perm, 4);
  CSX_ALIGN(cell_off, 4);
  CSX_ALIGN(ncell, 4);
  for (int c = 0; c < nconf; ++c) {
    int rc = check_K(K + 3 * c);
    if (rc) return rc;
  }
  int rc = CSX_OK;
  int* Kd = (int*)scratch(SCR_MISC, (size_t)nconf * 3 * sizeof(int), &rc);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CSX_CUDA(cudaMemcpyAsync(Kd, K, (size_t)nconf * 3 * sizeof(int), cudaMemcpyHostToDevice, s));
  return launch_cells(npix, nconf, labels, Kd, perm, cell_off, ncell, s);
}

int csx_fit_batch(const csx_model* m, const csx_sky* sky, int32_t nconf, const int32_t* labels,
                  const int32_t* K, const csx_fit_opts* opts, const float* beta0, float* beta_out,
                  double* L_out, int32_t* status, int32_t* iters, int32_t* nevals,
                  void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (nconf < 0) return fail(CSX_EINVAL, "nconf must be >= 0");
  const long long nprob = (long long)nconf * sky->nreal;
  if (nprob == 0) return CSX_OK;
  if (nprob > (1LL << 30)) return fail(CSX_EINVAL, "too many problems");
  if (!K || !opts || !beta0 || !beta_out || !L_out || !status || !iters)
    return fail(CSX_EINVAL, "NULL argument");
  if (sky->npix > 0 && !labels) return fail(CSX_EINVAL, "labels is NULL");
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(beta0, 4);
  CSX_ALIGN(beta_out, 4);
  CSX_ALIGN(L_out, 8);
  CSX_ALIGN(status, 4);
  CSX_ALIGN(iters, 4);
  CSX_ALIGN(nevals, 4);
  const csx_fit_opts& o = *opts;
  if (o.history < 1 || o.history > 16) return fail(CSX_EINVAL, "history must be in 1..16");
  if (o.max_iter < 0 || o.max_ls < 1) return fail(CSX_EINVAL, "max_iter >= 0 and max_ls >= 1 required");
  if (o.grad_mode != CSX_GRAD_ADJOINT && o.grad_mode != CSX_GRAD_FD) return fail(CSX_EINVAL, "unknown grad_mode");
  for (int j = 0; j < 3; ++j) {
    if (!(o.lower[j] < o.upper[j])) return fail(CSX_EINVAL, "lower < upper required");
    if (!(o.xtol[j] > 0)) return fail(CSX_EINVAL, "xtol must be > 0");
  }
  if (o.lower[1] <= 0.f) return fail(CSX_EINVAL, "T_d lower bound must be > 0");
  if (o.grad_mode == CSX_GRAD_FD && !(o.fd_step > 0)) return fail(CSX_EINVAL, "fd_step must be > 0");
  if (o.solver != CSX_SOLVER_LBFGS && o.solver != CSX_SOLVER_ADATOPK)
    return fail(CSX_EINVAL, "unknown solver");
  if (o.solver == CSX_SOLVER_ADATOPK && o.grad_mode != CSX_GRAD_ADJOINT)
    return fail(CSX_EINVAL, "AdaTopK needs the adjoint gradient");
  if (!(o.topk >= 0.f && o.topk <= 1.f)) return fail(CSX_EINVAL, "topk must be in [0, 1]");
  int path = o.path;
  if (path == CSX_PATH_AUTO)
    path = (sky->noise_kind != CSX_NOISE_PERPIXEL && o.grad_mode == CSX_GRAD_ADJOINT) ? CSX_PATH_MOMENT
                                                                                     : CSX_PATH_STREAM;
  if (path != CSX_PATH_MOMENT && path != CSX_PATH_STREAM) return fail(CSX_EINVAL, "unknown path");
  if (path == CSX_PATH_MOMENT && sky->noise_kind == CSX_NOISE_PERPIXEL)
    return fail(CSX_EINVAL, "the moment path needs homogeneous or separable noise");
  if (path == CSX_PATH_MOMENT && o.grad_mode == CSX_GRAD_FD)
    return fail(CSX_EINVAL, "the finite-difference plain form uses the stream path");
  cudaStream_t s = (cudaStream_t)stream;
  const int npix = sky->npix;

  // Sizes from the host-known K only: nothing is read back from the device, so the call returns
  // once its work is enqueued. Problem descriptors and the longest-first queue order are formed on
  // the device; the per-slot moment scratch is sized from the bound ncell <= min(npix, K_d K_T K_s).
  int Pmax = 0, rows_max = 0, ncell_max = 0;
  std::vector<long long> cost((size_t)nconf);
  for (int c = 0; c < nconf; ++c) {
    if ((rc = check_K(K + 3 * c))) return rc;
    const long long kd = K[3 * c], kt = K[3 * c + 1], ks = K[3 * c + 2];
    Pmax = std::max(Pmax, (int)(kd + kt + ks));
    rows_max = std::max(rows_max, (int)(kd + 2 * kt + ks));
    const long long bound = std::min<long long>((long long)npix, kd * kt * ks);
    if (path == CSX_PATH_MOMENT) ncell_max = std::max(ncell_max, (int)bound);
    cost[(size_t)c] = (path == CSX_PATH_MOMENT ? bound : 0) + 8 * (kd + kt + ks);
  }
  Pmax = (Pmax + 3) & ~3;
  const bool device_order = nconf <= FIT_ORDER_MAX;
  const size_t desc_b = ((size_t)nprob * sizeof(ProbDesc) + 255) & ~size_t(255);
  const size_t order_b = ((size_t)nprob * sizeof(int) + 255) & ~size_t(255);
  char* db = (char*)scratch(SCR_FIT_DESC, desc_b + order_b + 256 + (size_t)nconf * 3 * sizeof(int), &rc);
  if (rc) return rc;
  ProbDesc* probs_d = (ProbDesc*)db;
  int* order_d = (int*)(db + desc_b);
  int* head_d = (int*)(db + desc_b + order_b);
  int* Kdev = (int*)(db + desc_b + order_b + 256);
  int *perm = nullptr, *coffs = nullptr, *ncell = nullptr;
  {
    TraceSpan tr("fit: descriptors + cells", s);
    CSX_CUDA(cudaMemcpyAsync(Kdev, K, (size_t)nconf * 3 * sizeof(int), cudaMemcpyHostToDevice, s));
    if ((rc = launch_fit_desc(nconf, sky->nreal, Kdev, probs_d, s))) return rc;
    if (path == CSX_PATH_MOMENT) {
      const size_t per = (size_t)npix;
      char* cb = (char*)scratch(SCR_CELLS, (size_t)nconf * (2 * per + 2) * sizeof(int) + 256, &rc);
      if (rc) return rc;
      perm = (int*)cb;
      coffs = perm + (size_t)nconf * per;
      ncell = coffs + (size_t)nconf * (per + 1);
      if ((rc = launch_cells(npix, nconf, labels, Kdev, perm, coffs, ncell, s))) return rc;
    }
    if (device_order) {
      if ((rc = launch_fit_order(nconf, sky->nreal, Kdev, ncell, order_d, s))) return rc;
    } else {
      // longest-first queue order from the host-known estimate (more configurations than the
      // device sort takes)
      std::vector<int> order((size_t)nprob);
      std::iota(order.begin(), order.end(), 0);
      const int nr = sky->nreal;
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return cost[(size_t)(x / nr)] > cost[(size_t)(y / nr)]; });
      CSX_CUDA(cudaMemcpyAsync(order_d, order.data(), (size_t)nprob * sizeof(int), cudaMemcpyHostToDevice, s));
    }
  }

  long long slot_floats = 0;
  fit_slot_floats(Pmax, rows_max, ncell_max, o.history, path, &slot_floats);
  int grid = 0;
  if ((rc = fit_grid(o.threads, path, o.grad_mode, o.solver, &grid))) return rc;
  if ((long long)grid > nprob) grid = (int)nprob;
  float* slots = (float*)scratch(SCR_FIT_SLOTS, (size_t)grid * slot_floats * sizeof(float), &rc);
  if (rc) return rc;

  FitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.bands = make_bands(*m);
  a.npix = npix;
  a.nreal = sky->nreal;
  a.noise_kind = sky->noise_kind;
  a.d = sky->d;
  a.w = sky->w;
  a.ninv_pix = sky->ninv_pix;
  copy_band_weights(sky, m->nfreq, a.ninv_band);
  a.labels = labels;
  a.perm = perm;
  a.cell_off = coffs;
  a.ncell = ncell;
  a.probs = probs_d;
  a.order = order_d;
  a.nprob = (int)nprob;
  a.head = head_d;
  a.beta0 = beta0;
  a.beta_out = beta_out;
  a.L_out = L_out;
  a.status = status;
  a.iters = iters;
  a.nevals = nevals;
  a.slots = slots;
  a.slot_floats = slot_floats;
  a.Pmax = Pmax;
  a.rows_max = rows_max;
  a.ncell_max = ncell_max;
  a.history = o.history;
  a.max_iter = o.max_iter;
  a.max_ls = o.max_ls;
  a.path = path;
  a.grad_mode = o.grad_mode;
  for (int j = 0; j < 3; ++j) {
    a.lower[j] = o.lower[j];
    a.upper[j] = o.upper[j];
    a.xtol[j] = o.xtol[j];
  }
  a.fd_step = o.fd_step;
  a.solver = o.solver;
  a.topk = o.topk;
  TraceSpan tr("fit: kernel", s);
  return launch_fit(a, o.threads, grid, s);
}

int csx_cell_like_grad(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                       const int32_t K[3], int32_t nprob, const float* beta_ref, const float* beta,
                       double* L, float* grad, void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (!K) return fail(CSX_EINVAL, "K is NULL");
  if ((rc = check_K(K))) return rc;
  if (sky->noise_kind == CSX_NOISE_PERPIXEL)
    return fail(CSX_EINVAL, "the cell-moment evaluation needs homogeneous or separable noise");
  if (nprob < 0 || nprob > sky->nreal) return fail(CSX_EINVAL, "nprob must be in [0, sky->nreal]");
  if (nprob == 0) return CSX_OK;
  if (!beta_ref || !beta || !L || !grad) return fail(CSX_EINVAL, "NULL argument");
  if (sky->npix > 0 && !labels) return fail(CSX_EINVAL, "labels is NULL");
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(beta_ref, 4);
  CSX_ALIGN(beta, 4);
  CSX_ALIGN(L, 8);
  CSX_ALIGN(grad, 4);
  cudaStream_t s = (cudaStream_t)stream;
  const int npix = sky->npix;
  const int P = K[0] + K[1] + K[2];
  const int rows = K[0] + 2 * K[1] + K[2];
  const int Pmax = (P + 3) & ~3;
  const int bound = (int)std::min<long long>((long long)npix, (long long)K[0] * K[1] * K[2]);
  char* cb = (char*)scratch(SCR_CELLS, (size_t)(2 * npix + 2) * sizeof(int) + 256, &rc);
  if (rc) return rc;
  int* perm = (int*)cb;
  int* coffs = perm + npix;
  int* ncell = coffs + npix + 1;
  int* Kdev = (int*)(cb + (((size_t)(2 * npix + 2) * sizeof(int) + 15) & ~size_t(15)));
  std::vector<ProbDesc> probs((size_t)nprob);
  for (int q = 0; q < nprob; ++q) {
    ProbDesc& d = probs[(size_t)q];
    d.conf = 0;
    d.real = q;
    d.Kd = K[0];
    d.KT = K[1];
    d.Ks = K[2];
    d.P = P;
    d.poff = (long long)q * P;
    d.toff = 0;
  }
  ProbDesc* probs_d = (ProbDesc*)scratch(SCR_FIT_DESC, (size_t)nprob * sizeof(ProbDesc), &rc);
  if (rc) return rc;
  long long slot_floats = 0;
  fit_slot_floats(Pmax, rows, bound, 1, CSX_PATH_MOMENT, &slot_floats);
  int grid = 0;
  if ((rc = fit_grid(128, CSX_PATH_MOMENT, CSX_GRAD_ADJOINT, CSX_SOLVER_LBFGS, &grid))) return rc;
  if (grid > nprob) grid = nprob;
  float* slots = (float*)scratch(SCR_FIT_SLOTS, (size_t)grid * slot_floats * sizeof(float), &rc);
  if (rc) return rc;
  CSX_CUDA(cudaMemcpyAsync(Kdev, K, 3 * sizeof(int), cudaMemcpyHostToDevice, s));
  CSX_CUDA(cudaMemcpyAsync(probs_d, probs.data(), (size_t)nprob * sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
  if ((rc = launch_cells(npix, 1, labels, Kdev, perm, coffs, ncell, s))) return rc;
  FitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.bands = make_bands(*m);
  a.npix = npix;
  a.nreal = sky->nreal;
  a.noise_kind = sky->noise_kind;
  a.d = sky->d;
  a.w = sky->w;
  copy_band_weights(sky, m->nfreq, a.ninv_band);
  a.labels = labels;
  a.perm = perm;
  a.cell_off = coffs;
  a.ncell = ncell;
  a.probs = probs_d;
  a.nprob = nprob;
  a.beta0 = beta_ref;
  a.beta_eval = beta;
  a.L_out = L;
  a.grad_out = grad;
  a.slots = slots;
  a.slot_floats = slot_floats;
  a.Pmax = Pmax;
  a.rows_max = rows;
  a.ncell_max = bound;
  a.history = 1;
  a.path = CSX_PATH_MOMENT;
  return launch_cell_eval(a, grid, s);
}

int csx_reconstruct(const csx_model* m, const csx_sky* sky, int32_t nconf, const int32_t* labels,
                    const int32_t* K, const float* beta, const float* d_fg, float* s_hat,
                    float* sigma2, float* r_sys, double* metrics, void* stream) {
  int rc = check_model(m);
  if (rc) return rc;
  if ((rc = check_sky(sky, m->nfreq))) return rc;
  if (nconf < 0) return fail(CSX_EINVAL, "nconf must be >= 0");
  const long long nprob = (long long)nconf * sky->nreal;
  if (nprob == 0) return CSX_OK;
  if (!K || !beta) return fail(CSX_EINVAL, "NULL argument");
  if (sky->npix > 0 && !labels) return fail(CSX_EINVAL, "labels is NULL");
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(beta, 4);
  CSX_ALIGN(d_fg, 16);
  CSX_ALIGN(s_hat, 4);
  CSX_ALIGN(sigma2, 4);
  CSX_ALIGN(r_sys, 4);
  CSX_ALIGN(metrics, 8);
  cudaStream_t s = (cudaStream_t)stream;
  // descriptors formed on the device from K (no pageable per-problem copy, so the call does not
  // wait for earlier work on the stream)
  long long toff = 0;
  for (int c = 0; c < nconf; ++c) {
    if ((rc = check_K(K + 3 * c))) return rc;
    toff += (long long)sky->nreal * ((long long)K[3 * c] + 2LL * K[3 * c + 1] + K[3 * c + 2]);
  }
  const size_t desc_b = ((size_t)nprob * sizeof(ProbDesc) + 255) & ~size_t(255);
  char* db = (char*)scratch(SCR_RECON_DESC, desc_b + (size_t)nconf * 3 * sizeof(int), &rc);
  if (rc) return rc;
  ProbDesc* probs_d = (ProbDesc*)db;
  int* Kdev = (int*)(db + desc_b);
  float* tables = (float*)scratch(SCR_TABLES, (size_t)toff * NB * sizeof(float), &rc);
  if (rc) return rc;
  CSX_CUDA(cudaMemcpyAsync(Kdev, K, (size_t)nconf * 3 * sizeof(int), cudaMemcpyHostToDevice, s));
  if ((rc = launch_fit_desc(nconf, sky->nreal, Kdev, probs_d, s))) return rc;
  const Bands b = make_bands(*m);
  if ((rc = launch_recon_tables(b, (int)nprob, probs_d, beta, tables, toff, s))) return rc;
  if (metrics) CSX_CUDA(cudaMemsetAsync(metrics, 0, (size_t)nprob * CSX_NMETRIC * sizeof(double), s));
  if (sky->npix == 0) return CSX_OK;
  ReconArgs a;
  std::memset(&a, 0, sizeof(a));
  a.bands = b;
  a.npix = sky->npix;
  a.nreal = sky->nreal;
  a.noise_kind = sky->noise_kind;
  a.nprob = (int)nprob;
  a.d = sky->d;
  a.w = sky->w;
  a.ninv_pix = sky->ninv_pix;
  copy_band_weights(sky, m->nfreq, a.ninv_band);
  a.labels = labels;
  a.probs = probs_d;
  a.tables = tables;
  a.d_fg = d_fg;
  a.s_hat = s_hat;
  a.sigma2 = sigma2;
  a.r_sys = r_sys;
  a.metrics = metrics;
  TraceSpan tr("reconstruct: kernel", s);
  return launch_recon(a, s);
}

int csx_kmeans(const double* vec, int32_t n, int32_t nlab, const int32_t* K, const int32_t* init,
               int32_t max_iter, int32_t* labels, int32_t* iters, void* stream) {
  if (n < 1 || nlab < 0) return fail(CSX_EINVAL, "n must be >= 1 and nlab >= 0");
  if (nlab == 0) return CSX_OK;
  if (!vec || !K || !labels) return fail(CSX_EINVAL, "NULL argument");
  if (max_iter < 1) return fail(CSX_EINVAL, "max_iter must be >= 1");
  CSX_ALIGN(vec, 8);
  CSX_ALIGN(init, 4);
  CSX_ALIGN(labels, 4);
  CSX_ALIGN(iters, 4);
  std::vector<long long> ioff((size_t)nlab);
  long long total = 0;
  int kmax = 1;
  for (int L = 0; L < nlab; ++L) {
    if (K[L] < 1) return fail(CSX_EINVAL, "every K must be >= 1");
    ioff[L] = total;
    if (K[L] > 1 && K[L] < n) {
      if (K[L] > KMEANS_KMAX)
        return fail(CSX_EINVAL, "K above " + std::to_string(KMEANS_KMAX) + " (and below n)");
      total += K[L];
      kmax = std::max(kmax, (int)K[L]);
    }
  }
  if (total > 0 && !init) return fail(CSX_EINVAL, "init is NULL");
  int rc = CSX_OK;
  const size_t best_b = (size_t)nlab * n * sizeof(double);
  const size_t k_b = ((size_t)nlab * sizeof(int) + 15) & ~size_t(15);
  const size_t mem_b = ((size_t)nlab * n * sizeof(int) + 15) & ~size_t(15);
  char* scr = (char*)scratch(SCR_KMEANS, best_b + mem_b + k_b + (size_t)nlab * sizeof(long long), &rc);
  if (rc) return rc;
  double* best = (double*)scr;
  int* members = (int*)(scr + best_b);
  int* K_dev = (int*)(scr + best_b + mem_b);
  long long* ioff_dev = (long long*)(scr + best_b + mem_b + k_b);
  cudaStream_t s = (cudaStream_t)stream;
  CSX_CUDA(cudaMemcpyAsync(K_dev, K, (size_t)nlab * sizeof(int), cudaMemcpyHostToDevice, s));
  CSX_CUDA(cudaMemcpyAsync(ioff_dev, ioff.data(), (size_t)nlab * sizeof(long long),
                           cudaMemcpyHostToDevice, s));
  return launch_kmeans(vec, n, nlab, K_dev, ioff_dev, init, max_iter, kmax, labels, best, members,
                       iters, s);
}

int csx_select(int32_t nconf, int32_t nreal, const double* metrics, double* vtot, int32_t* best,
               void* stream) {
  if (nconf < 1 || nreal < 1) return fail(CSX_EINVAL, "nconf and nreal must be >= 1");
  if (!metrics || !vtot || !best) return fail(CSX_EINVAL, "NULL argument");
  CSX_ALIGN(metrics, 8);
  CSX_ALIGN(vtot, 8);
  CSX_ALIGN(best, 4);
  return launch_select(nconf, nreal, metrics, vtot, best, (cudaStream_t)stream);
}

}  // extern "C"
