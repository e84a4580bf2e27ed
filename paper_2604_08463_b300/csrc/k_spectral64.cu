// All-FP64 likelihood and adjoint gradient (Eqs. 3-4, Sec. 3.3.1): the same quantities as the
// streaming kernel, every operation in double precision (the data are read as stored, float32, and
// widened). It exists to check the FP32 kernels' rounding against an FP64 evaluation of the same
// definition on the device (the differentiation check of the nside-128 workload); B300's FP64 rate
// is a small fraction of its FP32 rate, so it is not a production path.
//
// Per pixel: A = [1, A_d, A_s] from FP64 SED tables, M = A^T N A, b_s = A^T N d_s, Cholesky M = L L^T,
// s_hat = M^-1 b_s, r_s = d_s - A s_hat; L_p = chi2_p - d^T N d (residual form);
// dL/dtheta = -2 sum_s (N r_s)^T (dA/dtheta) s_hat_s, added to the owning patch. Grid (pixel blocks,
// problems); FP64 per-thread sums, block reduction, one FP64 atomic per block for L; the gradient
// goes through a shared-memory P-vector (FP64 atomics) flushed once per block.
#include "csx_host.h"

namespace csx {

constexpr int S64_NT = 256;
constexpr int S64_SMEM_P = 4096;  // gradient vectors up to this length accumulate in shared memory

// FP64 SED table rows of one problem (layout of the FP32 tables, in double): P_d, B, dlnB/dT, S.
__device__ double table_entry64(const Bands64& b, int row, int f, int Kd, int KT,
                                const double* __restrict__ x) {
  if (f >= b.nf) return 0.0;
  if (row < Kd) return exp(x[row] * b.lnd[f]);
  row -= Kd;
  if (row < KT) {
    const double T = x[Kd + row];
    if (!(T > 0.0)) return nan("");
    return b.cd[f] * expm1(b.xk0 / T) / expm1(b.xk[f] / T);
  }
  row -= KT;
  if (row < KT) {
    const double T = x[Kd + row];
    if (!(T > 0.0)) return nan("");
    const double xf = b.xk[f] / T, x0 = b.xk0 / T;
    return (xf / -expm1(-xf) - x0 / -expm1(-x0)) / T;
  }
  row -= KT;
  return b.cs[f] * exp(x[Kd + KT + row] * b.lns[f]);
}

__global__ void k_tables64(Bands64 b, int nprob, int Kd, int KT, int Ks, const double* __restrict__ beta,
                           double* __restrict__ tables) {
  const int P = Kd + KT + Ks;
  const int rows = Kd + 2 * KT + Ks;
  const long long total = (long long)nprob * rows * NB;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i % NB);
    const long long rq = i / NB;
    tables[i] = table_entry64(b, (int)(rq % rows), f, Kd, KT, beta + (rq / rows) * P);
  }
}

template <int NOISE, bool GRAD, bool SMEM_GRAD>
__global__ void __launch_bounds__(S64_NT) k_spectral64(const Spec64Args a) {
  extern __shared__ double s64_grad[];
  __shared__ double sred[S64_NT / 32];
  const int q = blockIdx.y;
  const double* tab = a.tables + (long long)q * a.rows * NB;
  const float* d = a.d + (long long)q * a.npix * 2 * NB;
  double* gout = GRAD ? a.grad + (long long)q * a.P : nullptr;
  double* gacc = SMEM_GRAD ? s64_grad : gout;
  if (GRAD && SMEM_GRAD) {
    for (int i = threadIdx.x; i < a.P; i += S64_NT) s64_grad[i] = 0.0;
    __syncthreads();
  }
  double acc = 0.0;
  bool bad = false;
  for (int p = blockIdx.x * S64_NT + threadIdx.x; p < a.npix; p += gridDim.x * S64_NT) {
    const int kd = a.labels[p], kt = a.labels[a.npix + p], ks = a.labels[2 * a.npix + p];
    if ((unsigned)kd >= (unsigned)a.Kd || (unsigned)kt >= (unsigned)a.KT ||
        (unsigned)ks >= (unsigned)a.Ks) {
      bad = true;
      continue;
    }
    const double* pd = tab + (long long)kd * NB;
    const double* bt = tab + (long long)(a.Kd + kt) * NB;
    const double* dt = tab + (long long)(a.Kd + a.KT + kt) * NB;
    const double* ss = tab + (long long)(a.Kd + 2 * a.KT + ks) * NB;
    double n[NB], ad[NB], as[NB], dq[NB], du[NB];
    const double wp = NOISE == CSX_NOISE_SEPARABLE ? (double)a.w[p] : 1.0;
#pragma unroll
    for (int f = 0; f < NB; ++f) {
      n[f] = NOISE == CSX_NOISE_PERPIXEL ? (double)a.ninv_pix[(long long)p * NB + f]
                                          : wp * (double)a.ninv_band[f];
      ad[f] = pd[f] * bt[f];
      as[f] = ss[f];
      dq[f] = (double)d[(long long)p * 2 * NB + f];
      du[f] = (double)d[(long long)p * 2 * NB + NB + f];
    }
    // M = A^T N A (symmetric), b_s = A^T N d_s, d^T N d
    double m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0;
    double bq0 = 0, bq1 = 0, bq2 = 0, bu0 = 0, bu1 = 0, bu2 = 0, dnd = 0;
#pragma unroll
    for (int f = 0; f < NB; ++f) {
      const double na1 = n[f] * ad[f], na2 = n[f] * as[f];
      m00 += n[f];
      m01 += na1;
      m02 += na2;
      m11 += na1 * ad[f];
      m12 += na1 * as[f];
      m22 += na2 * as[f];
      bq0 += n[f] * dq[f];
      bq1 += na1 * dq[f];
      bq2 += na2 * dq[f];
      bu0 += n[f] * du[f];
      bu1 += na1 * du[f];
      bu2 += na2 * du[f];
      dnd += n[f] * (dq[f] * dq[f] + du[f] * du[f]);
    }
    // Cholesky M = L L^T
    if (!(m00 > 0.0)) { bad = true; continue; }
    const double l00 = sqrt(m00), l10 = m01 / l00, l20 = m02 / l00;
    const double t11 = m11 - l10 * l10;
    if (!(t11 > 0.0)) { bad = true; continue; }
    const double l11 = sqrt(t11), l21 = (m12 - l20 * l10) / l11;
    const double t22 = m22 - l20 * l20 - l21 * l21;
    if (!(t22 > 0.0)) { bad = true; continue; }
    const double l22 = sqrt(t22);
    double sq[3], su[3];
    {
      const double yq0 = bq0 / l00, yq1 = (bq1 - l10 * yq0) / l11, yq2 = (bq2 - l20 * yq0 - l21 * yq1) / l22;
      sq[2] = yq2 / l22;
      sq[1] = (yq1 - l21 * sq[2]) / l11;
      sq[0] = (yq0 - l10 * sq[1] - l20 * sq[2]) / l00;
      const double yu0 = bu0 / l00, yu1 = (bu1 - l10 * yu0) / l11, yu2 = (bu2 - l20 * yu0 - l21 * yu1) / l22;
      su[2] = yu2 / l22;
      su[1] = (yu1 - l21 * su[2]) / l11;
      su[0] = (yu0 - l10 * su[1] - l20 * su[2]) / l00;
    }
    double chi = 0, gbd = 0, gtd = 0, gbs = 0;
#pragma unroll
    for (int f = 0; f < NB; ++f) {
      const double rq = dq[f] - (sq[0] + ad[f] * sq[1] + as[f] * sq[2]);
      const double ru = du[f] - (su[0] + ad[f] * su[1] + as[f] * su[2]);
      const double nrq = n[f] * rq, nru = n[f] * ru;
      chi += nrq * rq + nru * ru;
      if (GRAD) {
        const double td = (nrq * sq[1] + nru * su[1]) * ad[f];
        gbd += td * a.bands.lnd[f];
        gtd += td * dt[f];
        gbs += (nrq * sq[2] + nru * su[2]) * as[f] * a.bands.lns[f];
      }
    }
    acc += chi - dnd;
    if (GRAD) {
      atomicAdd(gacc + kd, -2.0 * gbd);
      atomicAdd(gacc + a.Kd + kt, -2.0 * gtd);
      atomicAdd(gacc + a.Kd + a.KT + ks, -2.0 * gbs);
    }
  }
  double v = bad ? nan("") : acc;
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < S64_NT / 32; ++w) t += sred[w];
    atomicAdd(a.L + q, t);
  }
  if (GRAD && SMEM_GRAD) {
    for (int i = threadIdx.x; i < a.P; i += S64_NT) {
      const double g = s64_grad[i];
      if (g != 0.0) atomicAdd(gout + i, g);
    }
  }
}

template <int NOISE>
static int launch64_noise(const Spec64Args& a, bool grad, dim3 grid, cudaStream_t s) {
  if (!grad) {
    k_spectral64<NOISE, false, false><<<grid, S64_NT, 0, s>>>(a);
  } else if (a.P <= S64_SMEM_P) {
    const size_t smem = (size_t)a.P * sizeof(double);
    CSX_CUDA(cudaFuncSetAttribute(k_spectral64<NOISE, true, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(S64_SMEM_P * sizeof(double))));
    k_spectral64<NOISE, true, true><<<grid, S64_NT, smem, s>>>(a);
  } else {
    k_spectral64<NOISE, true, false><<<grid, S64_NT, 0, s>>>(a);
  }
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

int launch_spectral64(const Spec64Args& a, bool grad, cudaStream_t s) {
  if (a.nprob == 0) return CSX_OK;
  const long long total = (long long)a.nprob * a.rows * NB;
  if (total > 0) {
    const long long blocks = (total + 255) / 256;
    k_tables64<<<(int)(blocks < 148 * 32 ? blocks : 148 * 32), 256, 0, s>>>(
        a.bands, a.nprob, a.Kd, a.KT, a.Ks, a.beta, a.tables);
    CSX_CUDA(cudaGetLastError());
  }
  if (a.npix == 0) return CSX_OK;
  for (int q0 = 0; q0 < a.nprob; q0 += 65535) {
    Spec64Args b = a;
    const int nq = (a.nprob - q0 < 65535) ? a.nprob - q0 : 65535;
    b.nprob = nq;
    b.tables = a.tables + (long long)q0 * a.rows * NB;
    b.d = a.d + (long long)q0 * a.npix * 2 * NB;
    b.L = a.L + q0;
    b.grad = a.grad ? a.grad + (long long)q0 * a.P : nullptr;
    // about 8 pixels per thread, at least 2 CTAs per SM over all problems
    long long gx = (a.npix + S64_NT * 8 - 1) / (S64_NT * 8);
    if (gx * nq < 296) gx = (296 + nq - 1) / nq;
    const long long gmax = (a.npix + S64_NT - 1) / S64_NT;
    if (gx > gmax) gx = gmax;
    const dim3 grid((unsigned)gx, (unsigned)nq);
    int rc;
    switch (a.noise_kind) {
      case CSX_NOISE_HOMOGENEOUS: rc = launch64_noise<CSX_NOISE_HOMOGENEOUS>(b, grad, grid, s); break;
      case CSX_NOISE_SEPARABLE: rc = launch64_noise<CSX_NOISE_SEPARABLE>(b, grad, grid, s); break;
      default: rc = launch64_noise<CSX_NOISE_PERPIXEL>(b, grad, grid, s); break;
    }
    if (rc) return rc;
  }
  return CSX_OK;
}

}  // namespace csx
