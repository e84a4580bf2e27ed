/*
 * csx -- clustered parametric component separation on NVIDIA B300 (sm_103a).
 *
 * C ABI of the hot path of the parametric spectral-likelihood method of arxiv 2604.08463:
 * the mixing matrix (Eq. 5), the clustered spectral likelihood (Eq. 4 over the patches of
 * Sec. 2.2), its adjoint gradient (Sec. 3.3.1), the batched box-bounded fit over patch
 * configurations x noise realizations (Eq. 7, Sec. 3.1, App. A), the reconstruction
 * s_hat = W d with its residual diagnostics (Eqs. 3, 8-11, 14-15), the pseudo-C_ell residual
 * spectra (Sec. 2.5) and the seeded spherical K-means patches (Sec. 2.2).
 *
 * Conventions shared by every call
 *   - Plain pointers and sizes only. "device" pointers are CUDA device memory of the current
 *     device, "host" pointers are ordinary host memory. The caller owns every buffer; no pointer is
 *     retained after a call returns.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *     stream) unless stated otherwise. Outputs are valid once the stream has been synchronised.
 *   - Return value: CSX_OK (0) or a negative CSX_E* code; csx_last_error() gives a message.
 *     No exception or abort crosses the ABI. Argument checks happen before anything is enqueued.
 *   - The library keeps per-device scratch buffers between calls (grown on demand with
 *     cudaMalloc, released by csx_release()). Calls that use the same scratch must not overlap
 *     in time on different streams.
 *   - Band axis: every per-pixel vector has 16 float slots; bands nfreq..15 must hold zeros.
 *   - Data d: float32 [nreal][npix][2][16], Stokes Q then U: one 128-byte line per pixel.
 *   - Alignment: d, ninv_pix and d_fg must be 16-byte aligned (pixel rows are read as 16-byte
 *     vectors and staged by tensor copies); every other array its element size (4 bytes, 8 for
 *     double). A misaligned pointer is refused with CSX_EINVAL before anything is enqueued.
 *   - Patch labels: int32 [3][npix] per configuration (beta_d, T_d, beta_s labelings), values in
 *     [0, K_j). Labels out of range make the affected problem's likelihood NaN (spectral calls,
 *     reconstruction) or its fit status CSX_FIT_BADLABEL / CSX_FIT_NONPHYSICAL with L NaN (fit).
 *   - Parameters of one problem are packed [beta_d (K_d) | T_d (K_T) | beta_s (K_s)], P = sum K_j.
 */
#ifndef CSX_H
#define CSX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSX_MAX_BANDS 16
#define CSX_NMETRIC 8
#define CSX_MAX_K (1 << 24) /* largest patch count per parameter (larger K_j: CSX_EINVAL) */

/* return codes */
#define CSX_OK 0
#define CSX_EINVAL (-1)   /* null or misaligned pointer, bad size or option */
#define CSX_ECUDA (-2)    /* a CUDA runtime call failed */
#define CSX_ENOMEM (-3)   /* scratch allocation failed */
#define CSX_ETIMEOUT (-4) /* a bounded device wait gave up (reported by csx_device_status) */
#define CSX_ELABEL (-5)   /* a label outside [0, K_j) was found */

/* noise models: N_p^-1 = diag(ninv_band) | w_p diag(ninv_band) | diag(ninv_pix[p]) */
#define CSX_NOISE_HOMOGENEOUS 0
#define CSX_NOISE_SEPARABLE 1
#define CSX_NOISE_PERPIXEL 2

/* per-problem fit status */
#define CSX_FIT_CONVERGED 0
#define CSX_FIT_MAXITER 1
#define CSX_FIT_NONPHYSICAL 2   /* non-finite likelihood at the start (e.g. singular A^T N^-1 A) */
#define CSX_FIT_LINESEARCH 3    /* no acceptable step from the current point */
#define CSX_FIT_BADLABEL 4      /* the configuration has a label outside [0, K_j) (moment path) */

/* optimiser of csx_fit_batch: L-BFGS in Gauss-Newton-scaled variables, or AdaTopK (App. A:
 * AdaBelief directions, Top-K release of bound constraints, dynamic rescaling, backtracking) */
#define CSX_SOLVER_LBFGS 0
#define CSX_SOLVER_ADATOPK 1

/* likelihood evaluation inside the fit (AUTO: MOMENT for homogeneous or separable noise with the
 * adjoint gradient, STREAM otherwise) */
#define CSX_PATH_AUTO 0
#define CSX_PATH_STREAM 1  /* per pixel, any noise model */
#define CSX_PATH_MOMENT 2  /* per cell of equal (l_d, l_T, l_s); separable/homogeneous noise */

/* gradient inside the fit */
#define CSX_GRAD_ADJOINT 0 /* Sec. 3.3.1 */
#define CSX_GRAD_FD 1      /* central finite differences of the forward likelihood (plain form) */

/* selection-metric slots of csx_reconstruct (per problem, float64 sums over its pixels) */
#define CSX_M_SYS_SQ 0      /* sum_{p,s} r_sys^2,  r_sys = [W d_fg]_cmb (Eq. 15) */
#define CSX_M_STAT 1        /* sum_p [M_p^-1]_00 (statistical residual variance) */
#define CSX_M_CMB_Q 2       /* sum_p s_hat_cmb,Q */
#define CSX_M_CMB_Q2 3      /* sum_p s_hat_cmb,Q^2 */
#define CSX_M_CMB_U 4       /* sum_p s_hat_cmb,U */
#define CSX_M_CMB_U2 5      /* sum_p s_hat_cmb,U^2 */
#define CSX_M_NPIX 6        /* number of pixels */

/* Spectral model of Eq. 5: CMB column 1; dust modified blackbody normalised at nu0_dust;
 * synchrotron power law normalised at nu0_sync. units 0: K_CMB (each foreground column times
 * g(nu)/g(nu0), g = (e^x-1)^2/(x^2 e^x), x = h nu / k t_cmb); units 1: Rayleigh-Jeans. */
typedef struct csx_model {
  int32_t nfreq;          /* 1 .. 15 */
  int32_t units;          /* 0 K_CMB, 1 RJ */
  double nu_ghz[CSX_MAX_BANDS];
  double nu0_dust_ghz;    /* 353 */
  double nu0_sync_ghz;    /* 23 */
  double t_cmb;           /* 2.7255 K */
} csx_model;

/* Data and noise (Eq. 1). */
typedef struct csx_sky {
  int32_t npix;
  int32_t nreal;                       /* realizations stored in d */
  int32_t noise_kind;                  /* CSX_NOISE_* */
  int32_t reserved;
  const float* d;                      /* device [nreal][npix][2][16], 16-byte aligned */
  float ninv_band[CSX_MAX_BANDS];      /* host values: 1/sigma_f^2 (HOMOGENEOUS, SEPARABLE) */
  const float* w;                      /* device [npix] hit-count weights (SEPARABLE), else NULL */
  const float* ninv_pix;               /* device [npix][16] (PERPIXEL), 16-byte aligned, else NULL */
} csx_sky;

/* Options of csx_fit_batch. csx_fit_defaults() fills the values quoted here. */
typedef struct csx_fit_opts {
  int32_t max_iter;     /* 500: quasi-Newton iterations per problem */
  int32_t history;      /* 8: L-BFGS memory m, 1..16 */
  int32_t max_ls;       /* 20: likelihood evaluations per line search */
  int32_t path;         /* CSX_PATH_AUTO */
  int32_t grad_mode;    /* CSX_GRAD_ADJOINT */
  int32_t threads;      /* 0 = automatic CTA size */
  float lower[3];       /* box bounds (beta_d, T_d [K], beta_s): 0.5, 5, -5 */
  float upper[3];       /* 3, 60, -1 */
  float xtol[3];        /* 1e-4, 1e-3 K, 1e-4: stop once the quasi-Newton step and the last step of
                           every free parameter are below these (physical units) */
  float fd_step;        /* 1e-3: central-difference step in Gauss-Newton-scaled units (FD mode) */
  int32_t solver;       /* CSX_SOLVER_LBFGS; CSX_SOLVER_ADATOPK (App. A) needs CSX_GRAD_ADJOINT and
                           stops once the last two steps of every parameter are below 0.003 xtol */
  float topk;           /* 0: AdaTopK's Top-K fraction of releasable bound constraints freed per
                           iteration (0 = the single highest score, 1 = all) */
} csx_fit_opts;

/* Library version string. */
const char* csx_version(void);

/* Message of the last error on this host thread ("" if none). */
const char* csx_last_error(void);

/* Free the scratch buffers of the current device. Synchronises the device. */
int csx_release(void);

/*
 * Device-side failures found since the last call on the current device: synchronises `stream`,
 * then returns CSX_ETIMEOUT if any bounded wait of a streaming-kernel launch gave up (a tensor
 * copy that did not arrive within about 2 s; that problem's L was set to NaN and the kernel
 * returned), CSX_ECUDA if the synchronisation failed, else CSX_OK. The record is cleared.
 */
int csx_device_status(void* stream);

/*
 * Tile schedule of the streaming likelihood kernel (csx_spectral_like, csx_spectral_grad and
 * csx_spectral_grad_noalloc): pixels per tile (= threads per CTA) and tensor-copy pipeline stages,
 * for the launches that follow, in every thread and on every device. Built schedules:
 * (128, 2) (the default), (64, 2), (64, 3), (128, 3), (128, 4), (256, 2); (0, 0) restores the
 * default; (-1, -1) changes nothing. current: host int32[2] receiving the schedule in force, or
 * NULL. The results do not depend on the schedule beyond FP32 rounding. Errors: CSX_EINVAL for a
 * pair that is not built. A host-only call.
 */
int csx_stream_schedule(int32_t tile, int32_t stages, int32_t* current);

/* Fill `o` with the defaults listed in csx_fit_opts. */
int csx_fit_defaults(csx_fit_opts* o);

/*
 * Mixing matrix and its parameter derivatives (Eq. 5) for n parameter triples.
 *   beta  device float [n][3]  (beta_d, T_d [K], beta_s)
 *   A     device float [n][16][3]  (bands >= nfreq are 0)
 *   dA    device float [n][3][16] or NULL: dA_dust/dbeta_d, dA_dust/dT_d, dA_sync/dbeta_s
 * T_d <= 0 gives NaN entries.
 */
int csx_mixing(const csx_model* m, int32_t n, const float* beta, float* A, float* dA, void* stream);

/*
 * Spectral likelihood L(beta) = - sum_p sum_{s=Q,U} (A^T N^-1 d)^T (A^T N^-1 A)^-1 (A^T N^-1 d)
 * (Eq. 4, negated and doubled), for one patch configuration and nprob problems; problem i uses
 * realization i of the sky (nprob <= sky->nreal) and its own parameters.
 *   labels device int32 [3][npix];  K host int32[3]
 *   beta   device float [nprob][P]
 *   L      device double [nprob]   (overwritten)
 * Streaming kernel over pixels, evaluated in the residual form L = chi2_min - sum d^T N^-1 d.
 * A pixel whose A^T N^-1 A is not positive definite makes its problem's L NaN.
 */
int csx_spectral_like(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                      const int32_t K[3], int32_t nprob, const float* beta, double* L,
                      void* stream);

/*
 * Likelihood and adjoint gradient (Sec. 3.3.1): dL/dbeta = -2 sum_p sum_s w_r^T (dA/dbeta) s_hat,
 * w_r = N^-1 (d - A s_hat), routed to the owning patch. Same arguments as csx_spectral_like plus
 *   L     device double [nprob] or NULL
 *   grad  device float [nprob][P]  (overwritten)
 */
int csx_spectral_grad(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                      const int32_t K[3], int32_t nprob, const float* beta, double* L,
                      float* grad, void* stream);

/*
 * The likelihood and adjoint gradient of csx_spectral_grad with every operation in FP64 (the data
 * are read as stored, float32, and widened; SED tables, normal equations, Cholesky solve, residuals
 * and sums in double): an on-device check of the FP32 kernels' rounding (the differentiation check
 * at nside 128). B300's FP64 rate is a small fraction of its FP32 rate; this is not a fast path.
 *   beta  device double [nprob][P];  L device double [nprob];  grad device double [nprob][P] or NULL
 * Other arguments, layouts and errors as csx_spectral_grad.
 */
int csx_spectral_grad_f64(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                          const int32_t K[3], int32_t nprob, const double* beta, double* L,
                          double* grad, void* stream);

/*
 * csx_spectral_grad without any device allocation. The paper has no counterpart: this is an
 * interface for callers that cannot let a library call cudaMalloc -- applications whose device
 * memory belongs to their own pool allocator (an allocation behind its back can fail or fragment
 * the pool), and latency-critical loops with a fixed memory budget.
 * Same arguments and results as csx_spectral_grad, except that L must not be NULL. The only
 * scratch, the SED tables, lives in a static device array of 2^20 floats (4 MiB) that stays
 * resident on every device that loads the library until the process exits;
 * nprob x (K_d + 2 K_T + K_s) x 16 must not exceed 2^20, otherwise the call returns CSX_EINVAL and
 * enqueues nothing. The array's device address is looked up (cudaGetSymbolAddress) on the first
 * call on a device and again on each later call made while `stream` is not capturing (so a
 * re-created context gets its own address); make the first call on a device before any stream
 * capture begins. All calls on a device share the array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (for example on different streams) race and must be
 * serialised by the caller. K_j above CSX_MAX_K are refused like the other argument errors.
 */
int csx_spectral_grad_noalloc(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                              const int32_t K[3], int32_t nprob, const float* beta, double* L,
                              float* grad, void* stream);

/*
 * Cell plan of a patch configuration for repeated streaming evaluations (Eqs. 3-4 over the patches
 * of Sec. 2.2, gradient of Sec. 3.3.1): the label-only part of the streaming kernel, built once for
 * labels that stay fixed while beta changes (an optimiser's loop). A cell is a set of pixels with
 * equal (l_d, l_T, l_s); with homogeneous or separable noise every pixel of a cell shares the
 * Gram-Schmidt factors of A^T N^-1 A and the band vectors of the likelihood and gradient, which
 * csx_spectral_grad_plan forms once per (problem, cell) instead of once per run of equal labels in
 * the pixel stream.
 *   labels device int32 [3][npix];  K host int32[3]
 *   plan   receives an opaque handle (owns device memory: npix + 4 ncell int32) on the current
 *          device; release it with csx_spectral_plan_destroy.
 * Synchronises `stream` (the cell count sizes the plan). Errors: CSX_EINVAL for a label outside
 * [0, K_j), bad sizes or NULL pointers (nothing is allocated then); CSX_ECUDA.
 */
typedef struct csx_spectral_plan csx_spectral_plan;
int csx_spectral_plan_create(int32_t npix, const int32_t* labels, const int32_t K[3], void* stream,
                             csx_spectral_plan** plan);

/* Frees the plan's device memory (after the device has finished any call that uses it). NULL is a
 * no-op. */
int csx_spectral_plan_destroy(csx_spectral_plan* plan);

/* Cells of the plan (host int32). */
int csx_spectral_plan_ncell(const csx_spectral_plan* plan, int32_t* ncell);

/*
 * L (and, if grad is not NULL, the adjoint gradient) of csx_spectral_like / csx_spectral_grad for
 * the plan's labels and K: the same quantities up to FP32 rounding.
 *   beta  device float [nprob][P];  L device double [nprob];  grad device float [nprob][P] or NULL
 * Must run on the plan's device. Errors: CSX_EINVAL for per-pixel noise (no shared cell basis),
 * a sky whose npix differs from the plan's, NULL or misaligned pointers.
 */
int csx_spectral_grad_plan(const csx_spectral_plan* plan, const csx_model* m, const csx_sky* sky,
                           int32_t nprob, const float* beta, double* L, float* grad, void* stream);

/*
 * L and dL/dbeta by the cell-moment evaluation that csx_fit_batch uses for homogeneous or separable
 * noise (Eq. 4 and Sec. 3.3.1 over the cells of equal (l_d, l_T, l_s), Sec. 2.2): for problem i
 * (realization i, nprob <= sky->nreal), the residual moments of each cell are formed about the
 * reference point beta_ref[i] (one pass over the pixels), then L = chi2_min - sum d^T N^-1 d and
 * the gradient are evaluated at beta[i] from the moments alone. Same values as csx_spectral_grad
 * up to FP32 rounding, which grows with |beta - beta_ref| (the moments are residuals about the
 * reference point).
 *   labels device int32 [3][npix];  K host int32[3]
 *   beta_ref, beta  device float [nprob][P]
 *   L      device double [nprob]; grad device float [nprob][P]  (overwritten; NaN for a
 *          configuration with a label outside [0, K_j))
 * Errors: CSX_EINVAL for per-pixel noise, NULL or misaligned pointers, bad sizes.
 */
int csx_cell_like_grad(const csx_model* m, const csx_sky* sky, const int32_t* labels,
                       const int32_t K[3], int32_t nprob, const float* beta_ref, const float* beta,
                       double* L, float* grad, void* stream);

/*
 * Cells of each configuration: pixels sorted stably by (l_d, l_T, l_s) (Sec. 2.2-2.3).
 *   labels   device int32 [nconf][3][npix];  K host int32 [nconf][3]
 *   perm     device int32 [nconf][npix]      sorted pixel indices
 *   cell_off device int32 [nconf][npix + 1]  start of each cell in perm; entries past ncell unused
 *   ncell    device int32 [nconf]            (-1 for a configuration with a label out of range)
 * Bit-exact: equals a stable lexicographic sort on the host.
 */
int csx_build_cells(int32_t npix, int32_t nconf, const int32_t* labels, const int32_t* K,
                    int32_t* perm, int32_t* cell_off, int32_t* ncell, void* stream);

/*
 * Batched box-bounded fit beta* = argmin L (Eq. 7) of nconf configurations x sky->nreal
 * realizations in one persistent launch; problem q = c * nreal + n.
 *   labels  device int32 [nconf][3][npix];  K host int32 [nconf][3]
 *   beta0, beta_out  device float, packed per problem: problem q starts at
 *           nreal * coff[c] + n * P_c with coff[c] = sum_{c' < c} P_c' (beta_out may alias beta0)
 *   L_out   device double [nconf * nreal] (L at beta_out), status / iters device int32 [nconf*nreal]
 *   nevals  device int32 [nconf * nreal] or NULL: likelihood evaluations performed per problem
 *           (each forward evaluation of a finite-difference gradient counts once)
 * Optimiser: L-BFGS in Gauss-Newton-scaled variables with the active-set bound handling and
 * step limit of App. A, line search on approximate Wolfe conditions. The call does not
 * synchronise: sizes come from K alone (the moment path's per-CTA scratch from the bound
 * ncell <= min(npix, K_d K_T K_s) of each configuration), the problem descriptors and the
 * longest-first work queue are formed on the device (on the host, from the bound, above 16384
 * configurations). The result is deterministic: the same inputs give the same bits on every call
 * (gradient sums are formed in a fixed order, not with floating-point atomics).
 * A configuration with a label outside [0, K_j) gives its problems status CSX_FIT_BADLABEL (moment
 * path) or CSX_FIT_NONPHYSICAL (streaming path) and L NaN.
 */
int csx_fit_batch(const csx_model* m, const csx_sky* sky, int32_t nconf, const int32_t* labels,
                  const int32_t* K, const csx_fit_opts* opts, const float* beta0, float* beta_out,
                  double* L_out, int32_t* status, int32_t* iters, int32_t* nevals,
                  void* stream);

/*
 * Reconstruction s_hat = W d, W = (A^T N^-1 A)^-1 A^T N^-1 (Eqs. 3, 8) and residual diagnostics
 * for nconf configurations x sky->nreal realizations at the parameters `beta` (packed as in
 * csx_fit_batch). Every output may be NULL.
 *   d_fg    device float [npix][2][16] noise-free foreground data, or NULL (no r_sys)
 *   s_hat   device float [nconf*nreal][npix][2][3]
 *   sigma2  device float [nconf*nreal][npix]      [M_p^-1]_00
 *   r_sys   device float [nconf*nreal][npix][2]   [W d_fg]_cmb (Eq. 15)
 *   metrics device double [nconf*nreal][CSX_NMETRIC]  (CSX_M_* slots, overwritten)
 */
int csx_reconstruct(const csx_model* m, const csx_sky* sky, int32_t nconf, const int32_t* labels,
                    const int32_t* K, const float* beta, const float* d_fg, float* s_hat,
                    float* sigma2, float* r_sys, double* metrics, void* stream);

/*
 * Selection over configurations by total residual variance:
 *   vtot[c] = mean_n ( metrics[c,n][SYS_SQ] / (2 npix) + metrics[c,n][STAT] / npix ),
 *   best = argmin_c vtot[c] (lowest index on ties; NaN never wins).
 *   metrics device double [nconf*nreal][CSX_NMETRIC]; vtot device double [nconf]; best device int32[1]
 */
int csx_select(int32_t nconf, int32_t nreal, const double* metrics, double* vtot, int32_t* best,
               void* stream);

/* Seeded spherical K-means patches (Sec. 2.2) for nlab cluster counts at once, on the device: the
 * Lloyd iterations of the input generator (assignment by the largest dot product formed as
 * (x cx + y cy) + z cz in float64 without fused multiply-add, first cluster on ties; member sums in
 * increasing pixel order; an emptied cluster re-seeded at the pixel of smallest best dot product,
 * the i-th emptied cluster taking the i-th in (value, index) order; renormalisation by
 * sqrt((x x + y y) + z z); stop when an assignment repeats or after max_iter assignments; labels
 * renumbered by first appearance), so the labels are bit-exact with that generator.
 *   vec:    device [n][3] unit vectors (float64, 8-byte aligned)
 *   K:      host [nlab] cluster counts; K <= 1 gives one patch, K >= n one pixel per patch,
 *           otherwise 2..2048
 *   init:   device int32, for each labeling with 1 < K < n (in order) its K distinct starting
 *           pixels, concatenated (the seeded draw is the caller's)
 *   labels: device [nlab][n] output; iters: device [nlab] assignments made, or NULL
 * Errors: CSX_EINVAL for bad sizes, NULL or misaligned pointers. Asynchronous on `stream`. */
int csx_kmeans(const double* vec, int32_t n, int32_t nlab, const int32_t* K, const int32_t* init,
               int32_t max_iter, int32_t* labels, int32_t* iters, void* stream);

/*
 * Pseudo-C_ell spectra of polarisation maps (Sec. 2.5: the residual spectra C_ell^tot, C_ell^syst
 * = C^BB([W d_fg]_CMB) and C_ell^stat = <C^BB([s_hat - s_true] - [W d_fg]_CMB)>_n are pseudo-spectra
 * of residual maps on the observed sky). Conventions: spin-weighted harmonics sY_lm of Goldberg
 * et al. (1967); (Q +- iU) = sum a_{+-2,lm} (+-2)Y_lm; a^E = -(a_2 + a_-2)/2, a^B = i(a_2 - a_-2)/2;
 * a_{+-2,lm} = (4 pi / (12 nside^2)) sum over the observed pixels of (Q +- iU) conj((+-2)Y_lm) (the
 * map is zero elsewhere; no f_sky division); C_l = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1);
 * C_0 = C_1 = 0.
 *
 * A plan holds the geometry of the observed pixels and the spin-2 harmonic tables of its rings
 * (float32, nring x ~lmax^2/2 x 8 bytes, computed on the device in float64).
 *   nside: 1 .. 1024; lmax: 0 .. 4 nside - 1 (and <= 1023)
 *   pix:   HOST int32 [npix], RING pixel indices, strictly increasing, in [0, 12 nside^2)
 *   plan:  receives the plan (owned by the caller; csx_sht_plan_destroy frees it)
 * The plan belongs to the current device and is used on it only. Errors: CSX_EINVAL for bad sizes
 * or an unsorted / out-of-range pix; CSX_ECUDA / CSX_ENOMEM. The call synchronises `stream`.
 */
typedef struct csx_sht_plan csx_sht_plan;
int csx_sht_plan_create(int32_t nside, int32_t lmax, const int32_t* pix, int32_t npix,
                        csx_sht_plan** plan, void* stream);
int csx_sht_plan_destroy(csx_sht_plan* plan);

/*
 * (EE, BB) pseudo-spectra of nmaps maps, averaged over consecutive groups of navg maps:
 *   map b, observed pixel p, Stokes k (0 = Q, 1 = U):
 *     X_b[p][k] = maps[b * map_stride + p * pix_stride + k * pol_stride]
 *                 - sub_common[2 p + k] (if not NULL) - sub_each[(b * npix + p) * 2 + k] (if not NULL)
 *   e.g. the CMB residual of csx_reconstruct's s_hat: map_stride = 6 npix, pix_stride = 6,
 *   pol_stride = 3, sub_common = s_true [npix][2], sub_each = r_sys [nmaps][npix][2] (for stat).
 *   maps, sub_common, sub_each: device float (4-byte aligned); strides in elements, >= 0
 *   cl:    device double [nmaps / navg][2][lmax + 1] (EE, BB), overwritten; navg >= 1 divides nmaps
 * Scratch: about min(nmaps, 256) x nring x (lmax + 1) x 16 bytes. Asynchronous on `stream`.
 * Errors: CSX_EINVAL for a NULL plan / maps / cl, bad sizes or misaligned pointers.
 */
int csx_pseudo_cl(const csx_sht_plan* plan, int32_t nmaps, const float* maps, int64_t map_stride,
                  int32_t pix_stride, int32_t pol_stride, const float* sub_common,
                  const float* sub_each, int32_t navg, double* cl, void* stream);

/*
 * The three residual spectra of Sec. 2.5 in one pass: per problem q the CMB residual
 * X_q = s_hat_q - s_true (read through the strides of csx_pseudo_cl, e.g. csx_reconstruct's s_hat:
 * map_stride = 6 npix, pix_stride = 6, pol_stride = 3) and the foreground leakage Y_q = r_sys_q;
 * their ring coefficients are taken once each and the statistical residual uses
 * a_lm(X - Y) = a_lm(X) - a_lm(Y). Averaged over groups of navg problems (the realizations):
 *   cl_tot = <C(X)>, cl_syst = <C(Y)>, cl_stat = <C(X - Y)>, each device double
 *   [nprob / navg][2][lmax + 1] (EE, BB), overwritten.
 *   s_hat: device float; s_true: device float [npix][2] or NULL (no subtraction);
 *   r_sys: device float [nprob][npix][2]. Errors as csx_pseudo_cl. Asynchronous on `stream`.
 */
int csx_residual_cl(const csx_sht_plan* plan, int32_t nprob, const float* s_hat,
                    int64_t map_stride, int32_t pix_stride, int32_t pol_stride,
                    const float* s_true, const float* r_sys, int32_t navg, double* cl_tot,
                    double* cl_syst, double* cl_stat, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CSX_H */
