// SED tables, the mixing matrix (Eq. 5) and the streaming likelihood / adjoint-gradient kernel
// (Eqs. 3-4 over the patches of Sec. 2.2; gradient of Sec. 3.3.1).
#include "csx_host.h"

namespace csx {

// One thread per (problem, row, band) table entry.
__global__ void k_tables(Bands b, int nprob, int Kd, int KT, int Ks, const float* __restrict__ beta,
                         float* __restrict__ tables) {
  const int P = Kd + KT + Ks;
  const int rows = Kd + 2 * KT + Ks;
  const long long total = (long long)nprob * rows * NB;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i % NB);
    const long long rq = i / NB;
    const int row = (int)(rq % rows);
    const int q = (int)(rq / rows);
    tables[i] = table_entry(b, row, f, Kd, KT, beta + (long long)q * P);
  }
}

int launch_tables(const Bands& b, int nprob, int Kd, int KT, int Ks, const float* beta,
                  float* tables, cudaStream_t s) {
  const long long total = (long long)nprob * (Kd + 2 * KT + Ks) * NB;
  if (total == 0) return CSX_OK;
  const int threads = 256;
  const long long blocks = (total + threads - 1) / threads;
  k_tables<<<(int)(blocks < 148 * 32 ? blocks : 148 * 32), threads, 0, s>>>(b, nprob, Kd, KT, Ks,
                                                                             beta, tables);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

// Mixing matrix for n parameter triples: A [n][16][3], dA [n][3][16].
__global__ void k_mixing(Bands b, int n, const float* __restrict__ beta, float* __restrict__ A,
                         float* __restrict__ dA) {
  const long long total = (long long)n * NB;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i % NB);
    const long long t = i / NB;
    const float* x = beta + 3 * t;  // (beta_d, T_d, beta_s) laid out as Kd = KT = Ks = 1
    const float pd = table_entry(b, 0, f, 1, 1, x);
    const float bt = table_entry(b, 1, f, 1, 1, x);
    const float dt = table_entry(b, 2, f, 1, 1, x);
    const float ss = table_entry(b, 3, f, 1, 1, x);
    const float ad = pd * bt;
    float* a = A + (t * NB + f) * 3;
    a[0] = (f < b.nf) ? 1.f : 0.f;
    a[1] = ad;
    a[2] = ss;
    if (dA) {
      float* g = dA + t * 3 * NB;
      g[f] = ad * b.lnd[f];
      g[NB + f] = ad * dt;
      g[2 * NB + f] = ss * b.lns[f];
    }
  }
}

int launch_mixing(const Bands& b, int n, const float* beta, float* A, float* dA, cudaStream_t s) {
  if (n == 0) return CSX_OK;
  const long long total = (long long)n * NB;
  const long long blocks = (total + 255) / 256;
  k_mixing<<<(int)(blocks < 148 * 32 ? blocks : 148 * 32), 256, 0, s>>>(b, n, beta, A, dA);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

// ---------------------------------------------------------------------------------------------
// Streaming likelihood (+ gradient): grid (pixel blocks, problems). Each thread walks pixels with a
// grid stride, evaluates the residual form in FP32 and accumulates chi2 - d^T N d. Gradients go
// to a shared-memory copy of the problem's P-vector (one shared atomic per parameter and pixel),
// flushed to global memory with one atomic per touched parameter and block. Block sums of L are
// formed in FP64 and added to L[problem] with one FP64 atomic per block.
// A label outside [0, K_j) or a non-positive-definite A^T N A poisons the problem's L with NaN.
// ---------------------------------------------------------------------------------------------
template <int NOISE, bool GRAD, bool SMEM_GRAD>
__global__ void __launch_bounds__(256) k_spectral(SpecArgs a) {
  extern __shared__ float sgrad[];
  __shared__ double sred[8];
  const int q = blockIdx.y;
  const float* tab = a.tables + (long long)q * a.rows * NB;
  const float* dq0 = a.d + (long long)q * a.npix * 2 * NB;
  float* ggl = GRAD ? a.grad + (long long)q * a.P : nullptr;
  if (GRAD && SMEM_GRAD) {
    for (int i = threadIdx.x; i < a.P; i += blockDim.x) sgrad[i] = 0.f;
    __syncthreads();
  }
  float* gacc = SMEM_GRAD ? sgrad : ggl;
  const int* ld = a.labels;
  const int* lt = a.labels + a.npix;
  const int* ls = a.labels + 2 * a.npix;
  float nb[NB];
#pragma unroll
  for (int f = 0; f < NB; ++f) nb[f] = a.ninv_band[f];
  double acc = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.npix; p += gridDim.x * blockDim.x) {
    const int kd = __ldg(ld + p), kt = __ldg(lt + p), ks = __ldg(ls + p);
    if ((unsigned)kd >= (unsigned)a.Kd || (unsigned)kt >= (unsigned)a.KT ||
        (unsigned)ks >= (unsigned)a.Ks) {
      acc += (double)nan_f();
      continue;
    }
    float dq[NB], du[NB], nn[NB];
    load_pixel(dq0 + (long long)p * 2 * NB, dq, du);
    if (NOISE == CSX_NOISE_PERPIXEL) {
      const float4* n4 = reinterpret_cast<const float4*>(a.ninv_pix + (long long)p * NB);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 v = __ldg(n4 + k);
        nn[4 * k] = v.x; nn[4 * k + 1] = v.y; nn[4 * k + 2] = v.z; nn[4 * k + 3] = v.w;
      }
    } else if (NOISE == CSX_NOISE_SEPARABLE) {
      const float wp = __ldg(a.w + p);
#pragma unroll
      for (int f = 0; f < NB; ++f) nn[f] = wp * nb[f];
    } else {
#pragma unroll
      for (int f = 0; f < NB; ++f) nn[f] = nb[f];
    }
    PixOut o;
    const bool ok = pixel_eval<GRAD, false>(dq, du, nn, tab + (long long)kd * NB,
                                            tab + (long long)(a.Kd + kt) * NB,
                                            tab + (long long)(a.Kd + a.KT + kt) * NB,
                                            tab + (long long)(a.Kd + 2 * a.KT + ks) * NB, a.bands, o);
    if (!ok) {
      acc += (double)nan_f();
      continue;
    }
    acc += (double)(o.chi2 - o.dnd);
    if (GRAD) {
      atomicAdd(gacc + kd, o.gbd);
      atomicAdd(gacc + a.Kd + kt, o.gtd);
      atomicAdd(gacc + a.Kd + a.KT + ks, o.gbs);
    }
  }
  const double tot = block_sum<256>(acc, sred);
  if (threadIdx.x == 0) atomicAdd(a.L + q, tot);
  if (GRAD && SMEM_GRAD) {
    __syncthreads();
    for (int i = threadIdx.x; i < a.P; i += blockDim.x) {
      const float v = sgrad[i];
      if (v != 0.f) atomicAdd(ggl + i, v);
    }
  }
}

template <int NOISE, bool GRAD>
static int spectral_dispatch_smem(const SpecArgs& a, dim3 grid, cudaStream_t s) {
  const size_t smem = (size_t)a.P * sizeof(float);
  if (GRAD && smem <= 48 * 1024) {
    k_spectral<NOISE, GRAD, true><<<grid, 256, smem, s>>>(a);
  } else {
    k_spectral<NOISE, GRAD, false><<<grid, 256, 0, s>>>(a);
  }
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

template <bool GRAD>
static int spectral_dispatch(const SpecArgs& a, dim3 grid, cudaStream_t s) {
  switch (a.noise_kind) {
    case CSX_NOISE_HOMOGENEOUS: return spectral_dispatch_smem<CSX_NOISE_HOMOGENEOUS, GRAD>(a, grid, s);
    case CSX_NOISE_SEPARABLE: return spectral_dispatch_smem<CSX_NOISE_SEPARABLE, GRAD>(a, grid, s);
    default: return spectral_dispatch_smem<CSX_NOISE_PERPIXEL, GRAD>(a, grid, s);
  }
}

int launch_spectral(const SpecArgs& a, bool grad, cudaStream_t s) {
  if (a.nprob == 0) return CSX_OK;
  // about 8 pixels per thread, at most 65535 problems per launch (grid.y limit)
  int bx = (a.npix + 256 * 8 - 1) / (256 * 8);
  if (bx < 1) bx = 1;
  for (int q0 = 0; q0 < a.nprob; q0 += 65535) {
    SpecArgs b = a;
    const int nq = (a.nprob - q0 < 65535) ? a.nprob - q0 : 65535;
    b.nprob = nq;
    b.tables = a.tables + (long long)q0 * a.rows * NB;
    b.d = a.d + (long long)q0 * a.npix * 2 * NB;
    b.beta = a.beta + (long long)q0 * a.P;
    b.L = a.L + q0;
    b.grad = a.grad ? a.grad + (long long)q0 * a.P : nullptr;
    dim3 grid(bx, nq);
    const int rc = grad ? spectral_dispatch<true>(b, grid, s) : spectral_dispatch<false>(b, grid, s);
    if (rc) return rc;
  }
  return CSX_OK;
}

}  // namespace csx
