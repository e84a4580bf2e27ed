// Pseudo-C_ell spectra of polarisation maps on HEALPix rings (the residual spectra of Sec. 2.5).
//
//   plan        ring geometry of the observed pixels (host) and, per ring r and pair (l, m), the
//               spin-2 harmonic combinations F+-(theta_r) = (2lambda_lm +- (-2)lambda_lm) / 2
//               (k_sht_tables: float64 recursion, stored float32);
//   k_ring_dft  per ring and map, the ring coefficients Q_m(r) = sum_j Q_j e^{-i m phi_j} and U_m(r)
//               for m = 0 .. lmax (observed pixels only: the map is zero elsewhere);
//   k_alm_cl    a^E_lm = -w sum_r [F+ Q_m + i F- U_m], a^B_lm = w sum_r [i F- Q_m - F+ U_m]
//               (w = 4 pi / N_pix) and C_l = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1), summed in
//               shared memory, averaged over groups of maps in float64.
// Spin-weighted harmonics follow Goldberg et al. (1967): at l0 = max(m, 2) the closed form has a
// single term, above it the three-term relation of cos(theta) in the orthonormal basis of fixed
// (s, m): cos(theta) y_l = a_l y_{l+1} + b_l y_l + a_{l-1} y_{l-1},
// a_l = sqrt(((l+1)^2 - m^2)((l+1)^2 - s^2) / ((l+1)^2 (2l+1)(2l+3))), b_l = -m s / (l (l+1)).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "csx_host.h"
#include "csx_tma.cuh"

struct csx_sht_plan {
  int nside, lmax, npix, nring, nlm, maxn, device;
  double wpix;               // 4 pi / (12 nside^2): the equal pixel weight of the analysis
  int* ring_start;           // [nring + 1] first observed pixel of each ring (device)
  int* ring_n;               // [nring] pixels in the full ring
  double* ring_phi0;         // [nring] longitude of the ring's pixel j = 0
  int* pix_j;                // [npix] position of each observed pixel in its ring
  int* m_off;                // [lmax + 2] first flattened (l, m) index of each m (m-major)
  float2* F;                 // [nring][nlm] (F+, F-)
};

namespace csx {

// Tuning switches (defaults: the measured best on B300).
#ifndef CSX_DFT_MC
#define CSX_DFT_MC 8      // maps per k_ring_dft block
#endif
#ifndef CSX_DFT_SINCOS
#define CSX_DFT_SINCOS 0  // 1: twiddles re-anchored by sincospif (else from the shared table; measured faster)
#endif
#ifndef CSX_ALM_UNROLL
#define CSX_ALM_UNROLL 4  // ring-loop unroll of k_alm_cl
#endif
#ifndef CSX_ALM_STAGES
#define CSX_ALM_STAGES 1  // staged m groups in flight per k_alm_cl block (1 or 2)
#endif
#ifndef CSX_ALM_MINB
#define CSX_ALM_MINB 1    // k_alm_cl launch-bound blocks of ALM_NT_MAX threads (2: 64 registers)
#endif
#ifndef CSX_ALM_MB_MAX
#define CSX_ALM_MB_MAX 4  // maps per k_alm_cl block (4 or 8; fewer when shared memory is short)
#endif

constexpr int DFT_NT_MAX = 256;  // threads of k_ring_dft: one m per thread, lmax + 1 rounded to 32
constexpr int DFT_MC = CSX_DFT_MC;  // maps per k_ring_dft block (accumulators in registers)
constexpr int kAlmUnroll = CSX_ALM_UNROLL;
constexpr int kAlmStages = CSX_ALM_STAGES;
#ifndef CSX_DFT_REANCHOR
#define CSX_DFT_REANCHOR 16
#endif
constexpr int DFT_REANCHOR = CSX_DFT_REANCHOR;  // twiddles advanced by complex products at most this many pixels
constexpr int ALM_NT_MAX = 512;  // threads of k_alm_cl: one (l, m) pair of an m group each
constexpr size_t ALM_SMEM_MAX = 200 << 10;  // staged ring coefficients + spectra per block
constexpr int SHT_MAX_NSIDE = 256;

// ---- tables ---------------------------------------------------------------------------------------
// log of |s_lambda_lm(theta)| at l0 = max(m, 2) and its sign: the single surviving term of the
// closed form, sqrt[(l0+m)!(l0-m)!(2 l0+1) / (4 pi (l0+s)!(l0-s)!)] C(l0-s, r) C(l0+s, r+s-m)
// (-1)^(l0-r-s+m) sin^(2 l0 - e)(theta/2) cos^e(theta/2), e = 2r + s - m.
__device__ double sht_start(int s, int m, double log_sin, double log_cos) {
  const double log4pi = log(4.0 * 3.141592653589793);
  double lpre, sign = 1.0;
  int pa, pb;
  if (m >= 2) {  // l0 = m, r = m - s: coefficient 1, sign (-1)^m
    lpre = 0.5 * (lgamma(2.0 * m + 1.0) + log(2.0 * m + 1.0) - log4pi - lgamma(m + s + 1.0) -
                  lgamma(m - s + 1.0));
    pa = m + s;
    pb = m - s;
    sign = (m & 1) ? -1.0 : 1.0;
  } else {       // l0 = 2 > m: (2+m)!(2-m)! 5 / (4 pi 4!), coefficient C(4, 2 -+ m) = 6 or 4
    const double f = (m == 0) ? 4.0 : 6.0;
    lpre = 0.5 * (log(f * 5.0 / 24.0) - log4pi) + log(m == 0 ? 6.0 : 4.0);
    if (s > 0) {  // r = 0, sign (-1)^m
      pa = 2 + m;
      pb = 2 - m;
      sign = (m & 1) ? -1.0 : 1.0;
    } else {      // r = m + 2, sign (-1)^m (-1)^m = 1
      pa = 2 - m;
      pb = 2 + m;
    }
  }
  return sign * exp(lpre + pa * log_sin + pb * log_cos);
}

__device__ __forceinline__ double sht_a(int l, int m) {
  const double n = (double)(l + 1) * (l + 1);
  return sqrt((n - (double)m * m) * (n - 4.0) / (n * (2.0 * l + 1.0) * (2.0 * l + 3.0)));
}

// one thread per (ring, m): both spins upward in l, F+- written to the ring's row
__global__ void k_sht_tables(int nring, int lmax, int nlm, const double* z, const double* s2,
                             const double* c2, const int* m_off, float2* F) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nring * (lmax + 1)) return;
  const int r = idx / (lmax + 1), m = idx % (lmax + 1);
  const int l0 = m > 2 ? m : 2;
  if (l0 > lmax) return;
  const double x = z[r], ls = 0.5 * log(s2[r]), lc = 0.5 * log(c2[r]);
  double yp = sht_start(2, m, ls, lc), ym = sht_start(-2, m, ls, lc);
  double pp = 0.0, pm = 0.0;
  float2* out = F + (size_t)r * nlm + m_off[m];
  double a_prev = 0.0;
  for (int l = l0;; ++l) {
    out[l - l0] = make_float2((float)(0.5 * (yp + ym)), (float)(0.5 * (yp - ym)));
    if (l == lmax) break;
    const double a = sht_a(l, m);
    const double b = -2.0 * m / ((double)l * (l + 1));  // b_l for s = +2; s = -2 flips it
    const double np = ((x - b) * yp - a_prev * pp) / a;
    const double nm = ((x + b) * ym - a_prev * pm) / a;
    pp = yp;
    pm = ym;
    yp = np;
    ym = nm;
    a_prev = a;
  }
}

// ---- ring coefficients ------------------------------------------------------------------------------
struct DftArgs {
  const float* maps;         // chunk's first map
  long long map_stride;
  int pix_stride, pol_stride;
  const float* sub_common;   // [npix][2] or NULL
  const float* sub_each;     // chunk's first map's [npix][2] or NULL
  int nmaps, npix, nring, lmax, maxn;
  const int* ring_start;
  const int* ring_n;
  const double* ring_phi0;
  const int* pix_j;
  float4* delta;             // [maps][lmax + 1][nring] (Re Q_m, Im Q_m, Re U_m, Im U_m)
  int out_stride, out_off;   // map b of the chunk is written as map b * out_stride + out_off
};

__global__ void __launch_bounds__(DFT_NT_MAX) k_ring_dft(const DftArgs a) {
  extern __shared__ float2 dft_smem[];
  const int r = blockIdx.x, b0 = blockIdx.y * DFT_MC;
  const int n = a.ring_n[r], p0 = a.ring_start[r], cnt = a.ring_start[r + 1] - p0;
  float2* tw = dft_smem;                                  // [n]   e^{-2 pi i k / n}
  float2* val = dft_smem + a.maxn;                        // [cnt][DFT_MC] (Q, U)
  int* jj = reinterpret_cast<int*>(val + (size_t)a.maxn * DFT_MC);  // [cnt]
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * k / n, &sn, &cs);
    tw[k] = make_float2((float)cs, (float)-sn);
  }
  for (int i = threadIdx.x; i < cnt * DFT_MC; i += blockDim.x) {
    const int pi = i % cnt, bb = i / cnt, b = b0 + bb, p = p0 + pi;
    float q = 0.f, u = 0.f;
    if (b < a.nmaps) {
      const float* mp = a.maps + (long long)b * a.map_stride + (long long)p * a.pix_stride;
      q = mp[0];
      u = mp[a.pol_stride];
      if (a.sub_common) {
        q -= a.sub_common[2 * p];
        u -= a.sub_common[2 * p + 1];
      }
      if (a.sub_each) {
        const float* se = a.sub_each + ((long long)b * a.npix + p) * 2;
        q -= se[0];
        u -= se[1];
      }
    }
    val[pi * DFT_MC + bb] = make_float2(q, u);
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) jj[i] = a.pix_j[p0 + i];
  __syncthreads();
  const int L1 = a.lmax + 1;
  for (int m = threadIdx.x; m < L1; m += blockDim.x) {
    float qr[DFT_MC], qi[DFT_MC], ur[DFT_MC], ui[DFT_MC];
#pragma unroll
    for (int bb = 0; bb < DFT_MC; ++bb) qr[bb] = qi[bb] = ur[bb] = ui[bb] = 0.f;
    const int mm = m % n;
    const float2 step = tw[mm];
    float2 w = make_float2(1.f, 0.f);
    int jprev = -2;
    for (int i = 0; i < cnt; ++i) {
      const int j = jj[i];  // the same for every thread: the branch below is uniform
      if (j == jprev + 1 && (i % DFT_REANCHOR) != 0) {
        w = make_float2(w.x * step.x - w.y * step.y, w.x * step.y + w.y * step.x);
      } else {
        const int k = (mm * j) % n;  // mm, j < n <= 4 SHT_MAX_NSIDE: the product fits in int
        if (CSX_DFT_SINCOS) {  // computed: table reads at k = m j mod n collide across a warp's m
          float sn, cs;
          sincospif(2.f * (float)k / (float)n, &sn, &cs);
          w = make_float2(cs, -sn);
        } else {
          w = tw[k];
        }
      }
      jprev = j;
      const float4* v4 = reinterpret_cast<const float4*>(val + i * DFT_MC);  // two maps a load
#pragma unroll
      for (int h = 0; h < DFT_MC / 2; ++h) {
        const float4 v = v4[h];
        qr[2 * h] = fmaf(v.x, w.x, qr[2 * h]);
        qi[2 * h] = fmaf(v.x, w.y, qi[2 * h]);
        ur[2 * h] = fmaf(v.y, w.x, ur[2 * h]);
        ui[2 * h] = fmaf(v.y, w.y, ui[2 * h]);
        qr[2 * h + 1] = fmaf(v.z, w.x, qr[2 * h + 1]);
        qi[2 * h + 1] = fmaf(v.z, w.y, qi[2 * h + 1]);
        ur[2 * h + 1] = fmaf(v.w, w.x, ur[2 * h + 1]);
        ui[2 * h + 1] = fmaf(v.w, w.y, ui[2 * h + 1]);
      }
    }
    double sn, cs;
    sincos((double)m * a.ring_phi0[r], &sn, &cs);
    const float c = (float)cs, s = (float)-sn;  // e^{-i m phi0}
#pragma unroll
    for (int bb = 0; bb < DFT_MC; ++bb) {
      if (b0 + bb < a.nmaps)
        a.delta[((size_t)((b0 + bb) * a.out_stride + a.out_off) * L1 + m) * a.nring + r] =
            make_float4(qr[bb] * c - qi[bb] * s, qr[bb] * s + qi[bb] * c,
                        ur[bb] * c - ui[bb] * s, ur[bb] * s + ui[bb] * c);
    }
  }
}

// ---- harmonic coefficients and spectra ----------------------------------------------------------
// The (l, m) pairs are taken in m groups of at most lmax pairs: {0}, {1} and {g, lmax + 2 - g}
// for g = 2 .. (lmax + 2) / 2 (the two counts lmax - g + 1 and g - 1 add up to lmax). A block owns
// MB maps and a strided share of the groups; per group it stages the ring coefficients of its
// maps at the group's (one or two) m in shared memory (asynchronous copies, double-buffered),
// each thread sums one (l, m) pair over the rings, and C_l accumulates in shared memory.
struct AlmArgs {
  const float4* delta;  // [nmaps][lmax + 1][nring]
  const float2* F;      // [nring][nlm]
  const int* m_off;     // [lmax + 2] first flattened index of each m
  int nmaps, nring, nlm, lmax, map0, navg, ngroups;
  float w2;             // (4 pi / N_pix)^2
  double* cl;           // [groups of navg maps][2][lmax + 1]
  double* cl_syst;      // residual mode: maps come in pairs (X, Y) of one problem; cl receives
  double* cl_stat;      // <C(X)>, cl_syst <C(Y)>, cl_stat <C(X - Y)> over groups of navg problems
};

__device__ __forceinline__ int sht_l0(int m) { return m > 2 ? m : 2; }

__device__ __forceinline__ void sht_group(int g, int lmax, int& m1, int& m2) {
  m1 = g;
  m2 = (g >= 2 && lmax + 2 - g > g) ? lmax + 2 - g : -1;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}

template <int MB>
__device__ __forceinline__ void alm_stage(const AlmArgs& a, int b0, int nb, int g, float4* dst) {
  int m[2];
  sht_group(g, a.lmax, m[0], m[1]);
  const int L1 = a.lmax + 1, per = MB * a.nring;
  for (int i = threadIdx.x; i < 2 * per; i += blockDim.x) {
    const int mi = i / per, rest = i - mi * per, bb = rest / a.nring, r = rest - bb * a.nring;
    if (m[mi] >= 0 && bb < nb)
      cp_async16(dst + i, a.delta + ((size_t)(b0 + bb) * L1 + m[mi]) * a.nring + r);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int MB, bool RESID>
__global__ void __launch_bounds__(ALM_NT_MAX, CSX_ALM_MINB) k_alm_cl(const AlmArgs a) {
  static_assert(!RESID || MB % 2 == 0, "residual mode takes maps in pairs");
  extern __shared__ __align__(16) float4 alm_smem[];
  const int L1 = a.lmax + 1, nr = a.nring;
  float4* sd = alm_smem;                                      // [stages][2][MB][nring]
  float* cls = reinterpret_cast<float*>(alm_smem + kAlmStages * 2 * MB * nr);
  // plain: [MB][2 (E, B)][L1]; residual: [MB / 2][3 (X, Y, X - Y)][2][L1]
  const int b0 = blockIdx.x * MB;
  const int nb = min(MB, a.nmaps - b0);
  const int ncls = RESID ? (MB / 2) * 3 * 2 * L1 : MB * 2 * L1;
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) cls[i] = 0.f;
  int g = blockIdx.y, stage = 0;
  if (kAlmStages == 2 && g < a.ngroups) alm_stage<MB>(a, b0, nb, g, sd);
  for (; g < a.ngroups; g += gridDim.y) {
    if (kAlmStages == 2) {
      const int gn = g + gridDim.y;
      if (gn < a.ngroups) {
        alm_stage<MB>(a, b0, nb, gn, sd + (stage ^ 1) * 2 * MB * nr);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
    } else {
      alm_stage<MB>(a, b0, nb, g, sd);
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    int m1, m2;
    sht_group(g, a.lmax, m1, m2);
    const int c1 = a.lmax - sht_l0(m1) + 1, c2 = (m2 >= 0) ? a.lmax - sht_l0(m2) + 1 : 0;
    for (int k = threadIdx.x; k < c1 + c2; k += blockDim.x) {
      const int mi = (k < c1) ? 0 : 1;
      const int m = mi ? m2 : m1;
      const int l = sht_l0(m) + (mi ? k - c1 : k);
      const float2* Ft = a.F + a.m_off[m] + (l - sht_l0(m));
      const float4* D = sd + (stage * 2 + mi) * MB * nr;  // [bb][r]
      float eR[MB], eI[MB], bR[MB], bI[MB];
#pragma unroll
      for (int bb = 0; bb < MB; ++bb) eR[bb] = eI[bb] = bR[bb] = bI[bb] = 0.f;
#pragma unroll kAlmUnroll
      for (int r = 0; r < nr; ++r) {
        const float2 f = __ldg(Ft + (size_t)r * a.nlm);  // (F+, F-)
#pragma unroll
        for (int bb = 0; bb < MB; ++bb) {
          const float4 d = D[bb * nr + r];  // one address per m: a broadcast
          eR[bb] -= f.x * d.x - f.y * d.w;
          eI[bb] -= f.x * d.y + f.y * d.z;
          bR[bb] -= f.y * d.y + f.x * d.z;
          bI[bb] += f.y * d.x - f.x * d.w;
        }
      }
      const float wt = (m == 0 ? 1.f : 2.f) * a.w2 / (float)(2 * l + 1);
      if (RESID) {
#pragma unroll
        for (int h = 0; h < MB / 2; ++h) {
          if (2 * h < nb) {
            const int x = 2 * h, y = 2 * h + 1;
            const float dER = eR[x] - eR[y], dEI = eI[x] - eI[y];
            const float dBR = bR[x] - bR[y], dBI = bI[x] - bI[y];
            float* c = cls + (size_t)h * 6 * L1 + l;
            atomicAdd(c, wt * (eR[x] * eR[x] + eI[x] * eI[x]));
            atomicAdd(c + L1, wt * (bR[x] * bR[x] + bI[x] * bI[x]));
            atomicAdd(c + 2 * L1, wt * (eR[y] * eR[y] + eI[y] * eI[y]));
            atomicAdd(c + 3 * L1, wt * (bR[y] * bR[y] + bI[y] * bI[y]));
            atomicAdd(c + 4 * L1, wt * (dER * dER + dEI * dEI));
            atomicAdd(c + 5 * L1, wt * (dBR * dBR + dBI * dBI));
          }
        }
      } else {
#pragma unroll
        for (int bb = 0; bb < MB; ++bb) {
          if (bb < nb) {
            atomicAdd(&cls[(bb * 2) * L1 + l], wt * (eR[bb] * eR[bb] + eI[bb] * eI[bb]));
            atomicAdd(&cls[(bb * 2 + 1) * L1 + l], wt * (bR[bb] * bR[bb] + bI[bb] * bI[bb]));
          }
        }
      }
    }
    __syncthreads();  // the stage just read is the next iteration's copy target
    if (kAlmStages == 2) stage ^= 1;
  }
  const double inv = 1.0 / a.navg;
  if (RESID) {
    for (int i = threadIdx.x; i < (nb / 2) * 6 * L1; i += blockDim.x) {
      const int h = i / (6 * L1), rest = i % (6 * L1), kind = rest / (2 * L1), el = rest % (2 * L1);
      const int gi = ((a.map0 + b0) / 2 + h) / a.navg;
      double* out = kind == 0 ? a.cl : kind == 1 ? a.cl_syst : a.cl_stat;
      if (cls[i] != 0.f) atomicAdd(&out[(size_t)gi * 2 * L1 + el], (double)cls[i] * inv);
    }
  } else {
    for (int i = threadIdx.x; i < nb * 2 * L1; i += blockDim.x) {
      const int bb = i / (2 * L1), rest = i % (2 * L1);
      const int gi = (a.map0 + b0 + bb) / a.navg;
      if (cls[i] != 0.f) atomicAdd(&a.cl[(size_t)gi * 2 * L1 + rest], (double)cls[i] * inv);
    }
  }
}

static size_t alm_smem_bytes(int mb, int nring, int L1, bool resid) {
  return (size_t)kAlmStages * 2 * mb * nring * sizeof(float4) +
         (size_t)mb * (resid ? 3 : 2) * L1 * sizeof(float);
}

static size_t dft_smem_bytes(int maxn) {
  return (size_t)maxn * sizeof(float2) * (1 + DFT_MC) + (size_t)maxn * sizeof(int);
}

}  // namespace csx

using namespace csx;

// ---- C ABI ------------------------------------------------------------------------------------------
extern "C" {

int csx_sht_plan_destroy(csx_sht_plan* p) {
  if (!p) return CSX_OK;
  void* bufs[] = {p->ring_start, p->ring_n, p->ring_phi0, p->pix_j, p->m_off, p->F};
  cudaError_t first = cudaSuccess;
  for (void* b : bufs)
    if (b) {
      const cudaError_t e = cudaFree(b);
      if (first == cudaSuccess) first = e;
    }
  delete p;
  if (first != cudaSuccess) return cuda_fail(first, "cudaFree(plan)");
  return CSX_OK;
}

int csx_sht_plan_create(int32_t nside, int32_t lmax, const int32_t* pix, int32_t npix,
                        csx_sht_plan** out, void* stream) {
  if (!out) return fail(CSX_EINVAL, "plan is NULL");
  *out = nullptr;
  if (nside < 1 || nside > SHT_MAX_NSIDE)
    return fail(CSX_EINVAL, "nside must be in 1 .. " + std::to_string(SHT_MAX_NSIDE));
  if (lmax < 0 || lmax > 4 * nside - 1 || lmax > 1023)
    return fail(CSX_EINVAL, "lmax must be in 0 .. min(4 nside - 1, 1023)");
  const long long ntot = 12LL * nside * nside;
  if (npix < 0 || npix > ntot) return fail(CSX_EINVAL, "npix must be in 0 .. 12 nside^2");
  if (npix > 0 && !pix) return fail(CSX_EINVAL, "pix is NULL");
  for (int q = 0; q < npix; ++q) {
    if (pix[q] < 0 || pix[q] >= ntot) return fail(CSX_EINVAL, "pix out of range");
    if (q > 0 && pix[q] <= pix[q - 1]) return fail(CSX_EINVAL, "pix must be strictly increasing");
  }
  // ring walk (RING scheme, Gorski et al. 2005): first pixel, length, z, 1 - z, 1 + z, phi0
  const double pi = 3.141592653589793, n2 = 3.0 * nside * (double)nside;
  std::vector<int> rs, rn, pj((size_t)npix);
  std::vector<double> rz, rs2, rc2, rphi;
  int q = 0;
  for (int i = 1; i <= 4 * nside - 1 && q < npix; ++i) {
    long long first;
    int n;
    double z, omz, opz, phi0;
    if (i < nside) {
      first = 2LL * i * (i - 1);
      n = 4 * i;
      omz = (double)i * i / n2;
      opz = 2.0 - omz;
      z = 1.0 - omz;
      phi0 = pi / (4.0 * i);
    } else if (i <= 3 * nside) {
      first = 2LL * nside * (nside - 1) + 4LL * nside * (i - nside);
      n = 4 * nside;
      z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside);
      omz = 2.0 * i / (3.0 * nside) - 1.0 / 3.0;
      opz = 7.0 / 3.0 - 2.0 * i / (3.0 * nside);
      phi0 = ((i + nside) % 2 == 0) ? pi / (4.0 * nside) : 0.0;
    } else {
      const int k = 4 * nside - i;
      first = ntot - 2LL * k * (k + 1);
      n = 4 * k;
      opz = (double)k * k / n2;
      omz = 2.0 - opz;
      z = opz - 1.0;
      phi0 = pi / (4.0 * k);
    }
    const int q0 = q;
    while (q < npix && pix[q] < first + n) {
      pj[q] = (int)(pix[q] - first);
      ++q;
    }
    if (q > q0) {
      rs.push_back(q0);
      rn.push_back(n);
      rz.push_back(z);
      rs2.push_back(0.5 * omz);
      rc2.push_back(0.5 * opz);
      rphi.push_back(phi0);
    }
  }
  rs.push_back(npix);
  const int nring = (int)rn.size();
  std::vector<int> m_off((size_t)lmax + 2, 0);
  int nlm = 0;
  for (int m = 0; m <= lmax; ++m) {
    m_off[m] = nlm;
    nlm += std::max(0, lmax - std::max(m, 2) + 1);
  }
  m_off[lmax + 1] = nlm;
  csx_sht_plan* p = new csx_sht_plan();
  p->nside = nside;
  p->lmax = lmax;
  p->npix = npix;
  p->nring = nring;
  p->nlm = nlm;
  p->maxn = 1;
  for (int n : rn) p->maxn = n > p->maxn ? n : p->maxn;
  p->wpix = 4.0 * pi / (double)ntot;
  p->ring_start = p->ring_n = p->pix_j = nullptr;
  p->ring_phi0 = nullptr;
  p->m_off = nullptr;
  p->F = nullptr;
  CSX_CUDA(cudaGetDevice(&p->device));
  cudaStream_t s = (cudaStream_t)stream;
  double* tmp = nullptr;  // z, s2, c2 for the table kernel
  auto cleanup = [&](int rc) {
    if (tmp) cudaFree(tmp);
    csx_sht_plan_destroy(p);
    return rc;
  };
#define SHT_TRY(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, #call)); \
  } while (0)
  SHT_TRY(cudaMalloc(&p->ring_start, sizeof(int) * (nring + 1)));
  SHT_TRY(cudaMalloc(&p->ring_n, sizeof(int) * (nring > 0 ? nring : 1)));
  SHT_TRY(cudaMalloc(&p->ring_phi0, sizeof(double) * (nring > 0 ? nring : 1)));
  SHT_TRY(cudaMalloc(&p->pix_j, sizeof(int) * (npix > 0 ? npix : 1)));
  SHT_TRY(cudaMalloc(&p->m_off, sizeof(int) * (lmax + 2)));
  SHT_TRY(cudaMalloc(&p->F, sizeof(float2) * ((size_t)nring * p->nlm > 0 ? (size_t)nring * p->nlm : 1)));
  SHT_TRY(cudaMalloc(&tmp, sizeof(double) * 3 * (nring > 0 ? nring : 1)));
  SHT_TRY(cudaMemcpyAsync(p->ring_start, rs.data(), sizeof(int) * (nring + 1), cudaMemcpyHostToDevice, s));
  if (nring > 0) {
    SHT_TRY(cudaMemcpyAsync(p->ring_n, rn.data(), sizeof(int) * nring, cudaMemcpyHostToDevice, s));
    SHT_TRY(cudaMemcpyAsync(p->ring_phi0, rphi.data(), sizeof(double) * nring, cudaMemcpyHostToDevice, s));
    SHT_TRY(cudaMemcpyAsync(tmp, rz.data(), sizeof(double) * nring, cudaMemcpyHostToDevice, s));
    SHT_TRY(cudaMemcpyAsync(tmp + nring, rs2.data(), sizeof(double) * nring, cudaMemcpyHostToDevice, s));
    SHT_TRY(cudaMemcpyAsync(tmp + 2 * nring, rc2.data(), sizeof(double) * nring, cudaMemcpyHostToDevice, s));
  }
  if (npix > 0)
    SHT_TRY(cudaMemcpyAsync(p->pix_j, pj.data(), sizeof(int) * npix, cudaMemcpyHostToDevice, s));
  SHT_TRY(cudaMemcpyAsync(p->m_off, m_off.data(), sizeof(int) * (lmax + 2), cudaMemcpyHostToDevice, s));
  const int nthr = nring * (lmax + 1);
  if (nthr > 0 && p->nlm > 0) {
    k_sht_tables<<<(nthr + 127) / 128, 128, 0, s>>>(nring, lmax, p->nlm, tmp, tmp + nring,
                                                    tmp + 2 * nring, p->m_off, p->F);
    SHT_TRY(cudaGetLastError());
  }
  SHT_TRY(cudaStreamSynchronize(s));
#undef SHT_TRY
  cudaFree(tmp);
  *out = p;
  return CSX_OK;
}

}  // extern "C"

namespace csx {

// Spectra of `nunits` units: plain mode, one map per unit (X = maps - sub_common - sub_each);
// residual mode, the pair X = maps - sub_common, Y = r_sys (sub_each unused) per unit, with the
// spectra of X, Y and X - Y. Ring coefficients in chunks of units (about 256 MB of scratch).
static int run_spectra(const csx_sht_plan* p, int nunits, const float* maps, int64_t map_stride,
                       int pix_stride, int pol_stride, const float* sub_common,
                       const float* sub_each, const float* r_sys, int navg, double* cl,
                       double* cl_syst, double* cl_stat, bool resid, cudaStream_t s) {
  int rc, dev = -1;
  CSX_CUDA(cudaGetDevice(&dev));
  if (dev != p->device) return fail(CSX_EINVAL, "the plan belongs to another device");
  const int L1 = p->lmax + 1;
  const size_t out_b = sizeof(double) * (size_t)(nunits / navg) * 2 * L1;
  CSX_CUDA(cudaMemsetAsync(cl, 0, out_b, s));
  if (resid) {
    CSX_CUDA(cudaMemsetAsync(cl_syst, 0, out_b, s));
    CSX_CUDA(cudaMemsetAsync(cl_stat, 0, out_b, s));
  }
  if (p->nring == 0 || p->nlm == 0) return CSX_OK;  // nothing observed, or lmax < 2
  const int per_unit = resid ? 2 : 1;  // maps of ring coefficients per unit
  const size_t per_map = (size_t)p->nring * L1 * sizeof(float4);
  int chunk = (int)std::max<size_t>(DFT_MC, ((size_t)256 << 20) / (per_map * per_unit));
  chunk = std::min(chunk, nunits);
  chunk = (chunk + DFT_MC - 1) / DFT_MC * DFT_MC;
  float4* delta = (float4*)scratch(SCR_SHT, per_map * per_unit * chunk, &rc);
  if (rc) return rc;
  const size_t smA = dft_smem_bytes(p->maxn);
  CSX_CUDA(cudaFuncSetAttribute(k_ring_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA));
  const int ntA = std::min(DFT_NT_MAX, (L1 + 31) / 32 * 32);
  // harmonic sums: maps per block by the shared-memory budget (pairs in residual mode)
  int mb = CSX_ALM_MB_MAX;
  while (mb > (resid ? 2 : 1) && alm_smem_bytes(mb, p->nring, L1, resid) > ALM_SMEM_MAX) mb /= 2;
  const size_t smB = alm_smem_bytes(mb, p->nring, L1, resid);
  if (smB > ALM_SMEM_MAX) return fail(CSX_EINVAL, "too many rings for the harmonic-sum kernel");
  const void* kB = resid ? (mb == 8 ? (const void*)k_alm_cl<8, true>
                            : mb == 4 ? (const void*)k_alm_cl<4, true>
                                      : (const void*)k_alm_cl<2, true>)
                         : (mb == 8 ? (const void*)k_alm_cl<8, false>
                            : mb == 4 ? (const void*)k_alm_cl<4, false>
                            : mb == 2 ? (const void*)k_alm_cl<2, false>
                                      : (const void*)k_alm_cl<1, false>);
  CSX_CUDA(cudaFuncSetAttribute(kB, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smB));
  const int ntB = std::min(ALM_NT_MAX, (p->lmax + 31) / 32 * 32);
  const int ngroups = 1 + (p->lmax + 2) / 2;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  for (int c0 = 0; c0 < nunits; c0 += chunk) {
    const int nb = std::min(chunk, nunits - c0);
    DftArgs da;
    da.maps = maps + (long long)c0 * map_stride;
    da.map_stride = map_stride;
    da.pix_stride = pix_stride;
    da.pol_stride = pol_stride;
    da.sub_common = sub_common;
    da.sub_each = (!resid && sub_each) ? sub_each + (long long)c0 * p->npix * 2 : nullptr;
    da.nmaps = nb;
    da.npix = p->npix;
    da.nring = p->nring;
    da.lmax = p->lmax;
    da.maxn = p->maxn;
    da.ring_start = p->ring_start;
    da.ring_n = p->ring_n;
    da.ring_phi0 = p->ring_phi0;
    da.pix_j = p->pix_j;
    da.delta = delta;
    da.out_stride = per_unit;
    da.out_off = 0;
    const dim3 gA(p->nring, (nb + DFT_MC - 1) / DFT_MC);
    k_ring_dft<<<gA, ntA, smA, s>>>(da);
    CSX_CUDA(cudaGetLastError());
    if (resid) {  // Y = r_sys [units][npix][2]
      da.maps = r_sys + (long long)c0 * p->npix * 2;
      da.map_stride = 2LL * p->npix;
      da.pix_stride = 2;
      da.pol_stride = 1;
      da.sub_common = nullptr;
      da.sub_each = nullptr;
      da.out_off = 1;
      k_ring_dft<<<gA, ntA, smA, s>>>(da);
      CSX_CUDA(cudaGetLastError());
    }
    AlmArgs aa;
    aa.delta = delta;
    aa.F = p->F;
    aa.m_off = p->m_off;
    aa.nmaps = nb * per_unit;
    aa.nring = p->nring;
    aa.nlm = p->nlm;
    aa.lmax = p->lmax;
    aa.map0 = c0 * per_unit;
    aa.navg = navg;
    aa.ngroups = ngroups;
    aa.w2 = (float)(p->wpix * p->wpix);
    aa.cl = cl;
    aa.cl_syst = cl_syst;
    aa.cl_stat = cl_stat;
    const int gx = (nb * per_unit + mb - 1) / mb;
    // slices of the m groups so that the grid covers the SMs a few times
    const int gy = std::max(1, std::min(ngroups, (4 * nsm + gx - 1) / gx));
    const dim3 gB(gx, gy);
    if (resid) {
      if (mb == 8) k_alm_cl<8, true><<<gB, ntB, smB, s>>>(aa);
      else if (mb == 4) k_alm_cl<4, true><<<gB, ntB, smB, s>>>(aa);
      else k_alm_cl<2, true><<<gB, ntB, smB, s>>>(aa);
    } else {
      if (mb == 8) k_alm_cl<8, false><<<gB, ntB, smB, s>>>(aa);
      else if (mb == 4) k_alm_cl<4, false><<<gB, ntB, smB, s>>>(aa);
      else if (mb == 2) k_alm_cl<2, false><<<gB, ntB, smB, s>>>(aa);
      else k_alm_cl<1, false><<<gB, ntB, smB, s>>>(aa);
    }
    CSX_CUDA(cudaGetLastError());
  }
  return CSX_OK;
}

}  // namespace csx

extern "C" {

int csx_pseudo_cl(const csx_sht_plan* p, int32_t nmaps, const float* maps, int64_t map_stride,
                  int32_t pix_stride, int32_t pol_stride, const float* sub_common,
                  const float* sub_each, int32_t navg, double* cl, void* stream) {
  if (!p) return fail(CSX_EINVAL, "plan is NULL");
  if (nmaps < 0 || navg < 1 || nmaps % navg != 0)
    return fail(CSX_EINVAL, "nmaps must be >= 0 and a multiple of navg >= 1");
  if (map_stride < 0 || pix_stride < 0 || pol_stride < 0)
    return fail(CSX_EINVAL, "strides must be >= 0");
  if (nmaps == 0) return CSX_OK;
  if (!cl || (!maps && p->npix > 0)) return fail(CSX_EINVAL, "NULL argument");
  int rc;
  if ((rc = check_align(maps, 4, "maps")) || (rc = check_align(sub_common, 4, "sub_common")) ||
      (rc = check_align(sub_each, 4, "sub_each")) || (rc = check_align(cl, 8, "cl")))
    return rc;
  return run_spectra(p, nmaps, maps, map_stride, pix_stride, pol_stride, sub_common, sub_each,
                     nullptr, navg, cl, nullptr, nullptr, false, (cudaStream_t)stream);
}

int csx_residual_cl(const csx_sht_plan* p, int32_t nprob, const float* s_hat, int64_t map_stride,
                    int32_t pix_stride, int32_t pol_stride, const float* s_true,
                    const float* r_sys, int32_t navg, double* cl_tot, double* cl_syst,
                    double* cl_stat, void* stream) {
  if (!p) return fail(CSX_EINVAL, "plan is NULL");
  if (nprob < 0 || navg < 1 || nprob % navg != 0)
    return fail(CSX_EINVAL, "nprob must be >= 0 and a multiple of navg >= 1");
  if (map_stride < 0 || pix_stride < 0 || pol_stride < 0)
    return fail(CSX_EINVAL, "strides must be >= 0");
  if (nprob == 0) return CSX_OK;
  if (!cl_tot || !cl_syst || !cl_stat || (p->npix > 0 && (!s_hat || !r_sys)))
    return fail(CSX_EINVAL, "NULL argument");
  int rc;
  if ((rc = check_align(s_hat, 4, "s_hat")) || (rc = check_align(s_true, 4, "s_true")) ||
      (rc = check_align(r_sys, 4, "r_sys")) || (rc = check_align(cl_tot, 8, "cl_tot")) ||
      (rc = check_align(cl_syst, 8, "cl_syst")) || (rc = check_align(cl_stat, 8, "cl_stat")))
    return rc;
  return run_spectra(p, nprob, s_hat, map_stride, pix_stride, pol_stride, s_true, nullptr, r_sys,
                     navg, cl_tot, cl_syst, cl_stat, true, (cudaStream_t)stream);
}

}  // extern "C"
