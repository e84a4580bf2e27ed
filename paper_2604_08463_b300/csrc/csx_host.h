// Host-side internals of the csx library: error state, per-device scratch, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "csx_device.cuh"

namespace csx {

// ---- error reporting (thread-local message, negative return codes) ----------------------------
int fail(int code, const std::string& msg);
// CSX_EINVAL unless the (device) pointer is a multiple of `align` bytes; NULL passes.
int check_align(const void* p, size_t align, const char* what);
int cuda_fail(cudaError_t e, const char* where);
#define CSX_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// ---- per-device scratch: named grow-only buffers ----------------------------------------------
enum ScratchId {
  SCR_TABLES = 0,   // SED tables of csx_spectral_* / csx_reconstruct
  SCR_FIT_SLOTS,    // per-CTA-slot state of the persistent fit
  SCR_FIT_DESC,     // problem descriptors and queue order of the fit
  SCR_CELLS,        // cell structure of the fit (perm, offsets, counts)
  SCR_MISC,         // small counters
  SCR_RECON_DESC,
  SCR_KMEANS,       // K-means: per-labeling best dot products, cluster counts and offsets
  SCR_SHT,          // pseudo-C_ell: ring coefficients of a chunk of maps
  SCR_CELLTAB,      // per-(problem, cell) scalars and band vectors of csx_spectral_grad_plan
  SCR_COUNT
};
void* scratch(ScratchId id, size_t bytes, int* err);
void scratch_release_all();

Bands make_bands(const csx_model& m);

// Argument checks shared by the entry points (CSX_EINVAL with a message on failure).
int check_model(const csx_model* m);
int check_sky(const csx_sky* s, int nfreq);
int check_K(const int32_t* K);  // 1 <= K_j <= CSX_MAX_K

// ---- problem descriptor of the fit / reconstruction ---------------------------------------------
struct ProbDesc {
  int conf, real;
  int Kd, KT, Ks, P;
  long long poff;   // offset of the problem's parameters in the packed arrays
  long long toff;   // offset (in rows of 16 floats) of the problem's SED tables (reconstruction)
};

// ---- launchers (defined in the kernel translation units) -------------------------------------
struct SpecArgs {
  Bands bands;
  int npix, nprob, Kd, KT, Ks, P, rows;
  int noise_kind;
  const float* d;
  const float* w;
  const float* ninv_pix;
  float ninv_band[NB];
  const int* labels;
  const float* beta;
  const float* tables;   // [nprob][rows][16]
  double* L;
  float* grad;
  // cell plan (csx_spectral_plan; separable / homogeneous noise): each pixel's cell, the cells'
  // labels, and per problem and cell the Gram-Schmidt scalars and band vectors [nprob][ncell][96]
  const int* pcell;
  const int4* cell_lab;
  const float* ctab;
  int ncell;
};
// Floats of one (problem, cell) entry of the cell tables: 16 scalars (run_scalars) + 5 band vectors.
constexpr int CELL_TAB = 96;
int launch_cell_tables(const SpecArgs& a, bool grad, float* ctab, cudaStream_t s);
int launch_plan_cells(int npix, int ncell, const int* labels, const int* perm, const int* cell_off,
                      int* pcell, int4* cell_lab, cudaStream_t s);
int launch_tables(const Bands& b, int nprob, int Kd, int KT, int Ks, const float* beta,
                  float* tables, cudaStream_t s);

// All-FP64 evaluation (k_spectral64.cu): the per-band constants in double.
struct Bands64 {
  int nf;
  double xk0;
  double lnd[NB], lns[NB], xk[NB], cd[NB], cs[NB];
};
Bands64 make_bands64(const csx_model& m);
struct Spec64Args {
  Bands64 bands;
  int npix, nprob, Kd, KT, Ks, P, rows;
  int noise_kind;
  const float* d;
  const float* w;
  const float* ninv_pix;
  float ninv_band[NB];
  const int* labels;
  const double* beta;
  double* tables;   // [nprob][rows][16]
  double* L;
  double* grad;     // NULL: likelihood only
};
int launch_spectral64(const Spec64Args& a, bool grad, cudaStream_t s);
int launch_mixing(const Bands& b, int n, const float* beta, float* A, float* dA, cudaStream_t s);
int launch_spectral(const SpecArgs& a, bool grad, cudaStream_t s);
// Tile schedule of the streaming kernel for the launches that follow (process-wide).
int set_stream_schedule(int tile, int stages);
void get_stream_schedule(int* tile, int* stages);
// Synchronises `s`, returns (and clears) the count of bounded device waits that gave up.
int device_timeouts(cudaStream_t s, unsigned* count);

int launch_cells(int npix, int nconf, const int* labels, const int* K_dev, int* perm,
                 int* cell_off, int* ncell, cudaStream_t s);
constexpr int FIT_ORDER_MAX = 16384;  // configurations ordered on the device by launch_fit_order
int launch_fit_order(int nconf, int nreal, const int* K_dev, const int* ncell, int* order,
                     cudaStream_t s);
int launch_fit_desc(int nconf, int nreal, const int* K_dev, ProbDesc* probs, cudaStream_t s);

constexpr int KMEANS_KMAX = 2048;
size_t kmeans_smem(int kmax);
int launch_kmeans(const double* vec, int n, int nlab, const int* K_dev, const long long* ioff_dev,
                  const int* init, int max_iter, int kmax, int* labels, double* best, int* members,
                  int* iters, cudaStream_t s);

struct FitArgs {
  Bands bands;
  int npix, nreal, noise_kind;
  const float* d;
  const float* w;
  const float* ninv_pix;
  float ninv_band[NB];
  const int* labels;       // [nconf][3][npix]
  const int* perm;         // [nconf][npix]
  const int* cell_off;     // [nconf][npix+1]
  const int* ncell;        // [nconf]
  const ProbDesc* probs;   // [nprob]
  const int* order;        // [nprob] queue order
  int nprob;
  int* head;               // queue head counter (zeroed by the launcher)
  const float* beta0;
  float* beta_out;
  double* L_out;
  int* status;
  int* iters;
  int* nevals;             // may be NULL
  float* slots;            // per-slot scratch
  long long slot_floats;
  int Pmax, rows_max, ncell_max;
  int history, max_iter, max_ls;
  int path, grad_mode;
  float lower[3], upper[3], xtol[3], fd_step;
  int solver;
  float topk;
  const float* beta_eval;  // launch_cell_eval: evaluation points (beta0 holds the reference points)
  float* grad_out;         // launch_cell_eval: gradients [nprob][P]
};
int launch_fit(const FitArgs& a, int threads, int grid, cudaStream_t s);
int launch_cell_eval(const FitArgs& a, int grid, cudaStream_t s);
int fit_slot_floats(int Pmax, int rows_max, int ncell_max, int history, int path,
                    long long* out);
int fit_grid(int threads, int path, int grad_mode, int solver, int* grid);

struct ReconArgs {
  Bands bands;
  int npix, nreal, noise_kind, nprob;
  const float* d;
  const float* w;
  const float* ninv_pix;
  float ninv_band[NB];
  const int* labels;      // [nconf][3][npix]
  const ProbDesc* probs;
  const float* tables;    // rows per problem at probs[q].toff
  const float* d_fg;
  float* s_hat;
  float* sigma2;
  float* r_sys;
  double* metrics;
};
int launch_recon_tables(const Bands& b, int nprob, const ProbDesc* probs, const float* beta,
                        float* tables, long long total_rows, cudaStream_t s);
int launch_recon(const ReconArgs& a, cudaStream_t s);
int launch_select(int nconf, int nreal, const double* metrics, double* vtot, int* best,
                  cudaStream_t s);

}  // namespace csx
