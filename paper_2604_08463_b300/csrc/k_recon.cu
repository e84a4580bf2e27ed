// Reconstruction s_hat = W d, W = (A^T N^-1 A)^-1 A^T N^-1 (Eqs. 3, 8), the statistical residual
// variance [M^-1]_00, the map-space systematic residual [W d_fg]_cmb (Eq. 15), per-problem
// sums for the map variance (Eq. 9) and the selection by total residual variance.
#include "csx_host.h"

namespace csx {

#ifndef CSX_RECON_PPT
#define CSX_RECON_PPT 16  // pixels per thread of k_recon
#endif
constexpr int RECON_PPT = CSX_RECON_PPT;

// Tables for every problem of a batch: problem q's rows start at row probs[q].toff.
__global__ void k_recon_tables(Bands b, int nprob, const ProbDesc* __restrict__ probs,
                               const float* __restrict__ beta, float* __restrict__ tables,
                               long long total_rows) {
  // grid-stride over (row, band); the owning problem is found by binary search on toff
  const long long total = total_rows * NB;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / NB;
    const int f = (int)(i % NB);
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].toff <= row) lo = mid; else hi = mid - 1;
    }
    const ProbDesc pd = probs[lo];
    tables[i] = table_entry(b, (int)(row - pd.toff), f, pd.Kd, pd.KT, beta + pd.poff);
  }
}

int launch_recon_tables(const Bands& b, int nprob, const ProbDesc* probs, const float* beta,
                        float* tables, long long total_rows, cudaStream_t s) {
  if (nprob == 0 || total_rows == 0) return CSX_OK;
  const long long blocks = (total_rows * NB + 255) / 256;
  k_recon_tables<<<(int)(blocks < 148 * 64 ? blocks : 148 * 64), 256, 0, s>>>(b, nprob, probs, beta,
                                                                              tables, total_rows);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

template <int NOISE>
__global__ void __launch_bounds__(256) k_recon(ReconArgs a) {
  __shared__ double sred[7 * 8];
  const int q = blockIdx.y;
  const ProbDesc pd = a.probs[q];
  const float* tab = a.tables + pd.toff * NB;
  const int* lab = a.labels + (long long)pd.conf * 3 * a.npix;
  const float* dr = a.d + (long long)pd.real * a.npix * 2 * NB;
  float nb[NB];
#pragma unroll
  for (int f = 0; f < NB; ++f) nb[f] = a.ninv_band[f];
  // per-thread partial sums in FP32 (a thread takes a few pixels), FP64 across the warps
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.npix; p += gridDim.x * blockDim.x) {
    const int kd = lab[p], kt = lab[a.npix + p], ks = lab[2 * a.npix + p];
    float sq[3] = {nan_f(), nan_f(), nan_f()}, su[3] = {nan_f(), nan_f(), nan_f()};
    float var = nan_f(), rq = nan_f(), ru = nan_f();
    if ((unsigned)kd < (unsigned)pd.Kd && (unsigned)kt < (unsigned)pd.KT &&
        (unsigned)ks < (unsigned)pd.Ks) {
      const float* pdr = tab + kd * NB;
      const float* btr = tab + (pd.Kd + kt) * NB;
      const float* ssr = tab + (pd.Kd + 2 * pd.KT + ks) * NB;
      float nn[NB];
      if (NOISE == CSX_NOISE_PERPIXEL) {
#pragma unroll
        for (int f = 0; f < NB; ++f) nn[f] = __ldg(a.ninv_pix + (long long)p * NB + f);
      } else if (NOISE == CSX_NOISE_SEPARABLE) {
        const float wp = __ldg(a.w + p);
#pragma unroll
        for (int f = 0; f < NB; ++f) nn[f] = wp * nb[f];
      } else {
#pragma unroll
        for (int f = 0; f < NB; ++f) nn[f] = nb[f];
      }
      float ad[NB], as[NB], c1[NB], c2[NB];
#pragma unroll
      for (int f = 0; f < NB; ++f) {
        ad[f] = pdr[f] * btr[f];
        as[f] = ssr[f];
      }
      Mgs3 g;
      if (mgs3(nn, ad, as, c1, c2, g)) {
        // s_hat = R^-1 t with t the projections on the orthogonalised columns (1, c1, c2)
        auto solve = [&](const float* x, float* s) {
          float t0 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll
          for (int f = 0; f < NB; ++f) {
            const float nx = nn[f] * x[f];
            t0 += nx;
            t1 = fmaf(nx, c1[f], t1);
            t2 = fmaf(nx, c2[f], t2);
          }
          t0 *= g.i0;
          t1 *= g.i1;
          t2 *= g.i2;
          s[2] = t2;
          s[1] = fmaf(-g.nu, t2, t1);
          s[0] = t0 - g.mu1 * s[1] - g.mu2 * s[2];
        };
        float dq[NB], du[NB];
        load_pixel(dr + (long long)p * 2 * NB, dq, du);
        solve(dq, sq);
        solve(du, su);
        var = mgs3_var00(g);
        if (a.d_fg) {
          float gq[NB], gu[NB], t[3];
          load_pixel(a.d_fg + (long long)p * 2 * NB, gq, gu);
          solve(gq, t);
          rq = t[0];
          solve(gu, t);
          ru = t[0];
        } else {
          rq = ru = 0.f;
        }
      }
    }
    const long long pq = (long long)q * a.npix + p;
    if (a.s_hat) {
      float* o = a.s_hat + pq * 6;
      o[0] = sq[0]; o[1] = sq[1]; o[2] = sq[2];
      o[3] = su[0]; o[4] = su[1]; o[5] = su[2];
    }
    if (a.sigma2) a.sigma2[pq] = var;
    if (a.r_sys) {
      a.r_sys[pq * 2] = rq;
      a.r_sys[pq * 2 + 1] = ru;
    }
    acc[0] = fmaf(rq, rq, fmaf(ru, ru, acc[0]));
    acc[1] += var;
    acc[2] += sq[0];
    acc[3] = fmaf(sq[0], sq[0], acc[3]);
    acc[4] += su[0];
    acc[5] = fmaf(su[0], su[0], acc[5]);
    acc[6] += 1.f;
  }
  if (a.metrics) {
#pragma unroll
    for (int k = 0; k < 7; ++k) acc[k] = warp_sum(acc[k]);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
#pragma unroll
      for (int k = 0; k < 7; ++k) sred[k * 8 + w] = (double)acc[k];
    }
    __syncthreads();
    if (threadIdx.x < 7) {
      double t = 0.0;
      for (int j = 0; j < 8; ++j) t += sred[threadIdx.x * 8 + j];
      atomicAdd(a.metrics + (long long)q * CSX_NMETRIC + threadIdx.x, t);
    }
  }
}

int launch_recon(const ReconArgs& a, cudaStream_t s) {
  if (a.nprob == 0) return CSX_OK;
  int bx = (a.npix + 256 * RECON_PPT - 1) / (256 * RECON_PPT);
  if (bx < 1) bx = 1;
  for (int q0 = 0; q0 < a.nprob; q0 += 65535) {
    ReconArgs b = a;
    b.nprob = (a.nprob - q0 < 65535) ? a.nprob - q0 : 65535;
    b.probs = a.probs + q0;
    // outputs are indexed by the problem index inside the launch
    if (b.s_hat) b.s_hat = a.s_hat + (long long)q0 * a.npix * 6;
    if (b.sigma2) b.sigma2 = a.sigma2 + (long long)q0 * a.npix;
    if (b.r_sys) b.r_sys = a.r_sys + (long long)q0 * a.npix * 2;
    if (b.metrics) b.metrics = a.metrics + (long long)q0 * CSX_NMETRIC;
    dim3 grid(bx, b.nprob);
    switch (a.noise_kind) {
      case CSX_NOISE_HOMOGENEOUS: k_recon<CSX_NOISE_HOMOGENEOUS><<<grid, 256, 0, s>>>(b); break;
      case CSX_NOISE_SEPARABLE: k_recon<CSX_NOISE_SEPARABLE><<<grid, 256, 0, s>>>(b); break;
      default: k_recon<CSX_NOISE_PERPIXEL><<<grid, 256, 0, s>>>(b); break;
    }
    CSX_CUDA(cudaGetLastError());
  }
  return CSX_OK;
}

// vtot[c] = mean_n (sys_sq / (2 npix) + stat / npix); best = argmin (lowest index on ties).
__global__ void k_select(int nconf, int nreal, const double* __restrict__ metrics,
                         double* __restrict__ vtot, int* __restrict__ best) {
  __shared__ double sv[256];
  __shared__ int si[256];
  double bv = 0.0;
  int bi = -1;
  for (int c = threadIdx.x; c < nconf; c += blockDim.x) {
    double v = 0.0;
    for (int n = 0; n < nreal; ++n) {
      const double* m = metrics + ((long long)c * nreal + n) * CSX_NMETRIC;
      const double np = m[CSX_M_NPIX];
      v += m[CSX_M_SYS_SQ] / (2.0 * np) + m[CSX_M_STAT] / np;
    }
    v /= nreal;
    vtot[c] = v;
    const double vs = isnan(v) ? INFINITY : v;  // a failed configuration is never selected first
    if (bi < 0 || vs < bv) {
      bv = vs;
      bi = c;
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    int i = -1;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      if (si[t] < 0) continue;
      if (i < 0 || sv[t] < b || (sv[t] == b && si[t] < i)) {
        b = sv[t];
        i = si[t];
      }
    }
    *best = i;
  }
}

int launch_select(int nconf, int nreal, const double* metrics, double* vtot, int* best,
                  cudaStream_t s) {
  k_select<<<1, 256, 0, s>>>(nconf, nreal, metrics, vtot, best);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

}  // namespace csx
