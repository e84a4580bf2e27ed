// Cells of a patch configuration: the pixels sorted stably by (l_d, l_T, l_s) and the start
// offset of every run of equal triples (Sec. 2.2-2.3: three independent labelings whose
// intersections share all spectral parameters).
//
// One CTA per configuration. Stable LSD radix sort on the three labels (l_s first, l_d last),
// 8-bit digits, passes only over the bits a label can use. Each warp owns a contiguous segment of
// the array: per-warp digit histograms, an exclusive scan in (digit, warp) order, then an in-order
// scatter where lanes with equal digits are ranked with __match_any_sync. Labels outside
// [0, K_j) make ncell = -1.
#include "csx_host.h"

namespace csx {

constexpr int CELL_NT = 512;
constexpr int CELL_NW = CELL_NT / 32;

__device__ __forceinline__ int block_excl_scan(int v, int* sbuf, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sbuf[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = (lane < CELL_NW) ? sbuf[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < CELL_NW) sbuf[lane] = t;
  }
  __syncthreads();
  total = sbuf[CELL_NW - 1];
  return x - v + (w > 0 ? sbuf[w - 1] : 0);
}

__global__ void __launch_bounds__(CELL_NT) k_cells(int npix, const int* __restrict__ labels,
                                                   const int* __restrict__ Kdev,
                                                   int* __restrict__ perm, int* __restrict__ cell_off,
                                                   int* __restrict__ ncell) {
  __shared__ int hist[256 * CELL_NW];  // [digit][warp]
  __shared__ int sbuf[32];
  __shared__ int sbad;
  const int c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int* lab = labels + (long long)c * 3 * npix;
  int* out = perm + (long long)c * npix;
  int* tmp = cell_off + (long long)c * (npix + 1);
  const int K0 = Kdev[3 * c], K1 = Kdev[3 * c + 1], K2 = Kdev[3 * c + 2];
  if (tid == 0) sbad = 0;
  __syncthreads();
  for (int i = tid; i < npix; i += CELL_NT) {
    if ((unsigned)lab[i] >= (unsigned)K0 || (unsigned)lab[npix + i] >= (unsigned)K1 ||
        (unsigned)lab[2 * npix + i] >= (unsigned)K2)
      sbad = 1;
    out[i] = i;
  }
  __syncthreads();
  if (sbad) {
    if (tid == 0) ncell[c] = -1;
    return;
  }
  int* src = out;
  int* dst = tmp;
  const int per = (npix + CELL_NW - 1) / CELL_NW;
  const int seg0 = min(npix, w * per), seg1 = min(npix, seg0 + per);
  for (int j = 2; j >= 0; --j) {
    const int Kj = (j == 0) ? K0 : (j == 1) ? K1 : K2;
    if (Kj <= 1) continue;
    const int bits = 32 - __clz(Kj - 1);
    const int* key = lab + (long long)j * npix;
    for (int shift = 0; shift < bits; shift += 8) {
      for (int i = tid; i < 256 * CELL_NW; i += CELL_NT) hist[i] = 0;
      __syncthreads();
      for (int i = seg0 + lane; i < seg1; i += 32)
        atomicAdd(&hist[((key[src[i]] >> shift) & 255) * CELL_NW + w], 1);
      __syncthreads();
      // exclusive scan of hist in (digit, warp) order: 8 consecutive entries per thread
      int loc[8], s = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        loc[k] = hist[tid * 8 + k];
        s += loc[k];
      }
      int total;
      int run = block_excl_scan(s, sbuf, total);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        hist[tid * 8 + k] = run;
        run += loc[k];
      }
      __syncthreads();
      for (int b = seg0; b < seg1; b += 32) {
        const int i = b + lane;
        const bool valid = i < seg1;
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        int v = 0, dg = 0, rank = 0;
        unsigned peers = 0;
        if (valid) {
          v = src[i];
          dg = (key[v] >> shift) & 255;
          peers = __match_any_sync(act, dg);
          rank = __popc(peers & ((1u << lane) - 1u));
          dst[hist[dg * CELL_NW + w] + rank] = v;
        }
        __syncwarp();
        if (valid && rank == 0) hist[dg * CELL_NW + w] += __popc(peers);
        __syncwarp();
      }
      __syncthreads();
      int* t = src;
      src = dst;
      dst = t;
    }
  }
  if (src != out) {
    for (int i = tid; i < npix; i += CELL_NT) out[i] = src[i];
    __syncthreads();
  }
  // cell starts: positions where the (l_d, l_T, l_s) triple changes
  int running = 0;
  for (int b = 0; b < npix; b += CELL_NT) {
    const int i = b + tid;
    int flag = 0;
    if (i < npix) {
      if (i == 0) {
        flag = 1;
      } else {
        const int u = out[i], v = out[i - 1];
        flag = (lab[u] != lab[v]) || (lab[npix + u] != lab[npix + v]) ||
               (lab[2 * npix + u] != lab[2 * npix + v]);
      }
    }
    int total;
    const int ex = block_excl_scan(flag, sbuf, total);
    if (flag) tmp[running + ex] = i;
    running += total;
  }
  if (tid == 0) {
    tmp[running] = npix;
    ncell[c] = running;
  }
}

// Work-queue order of the persistent fit, longest first: configurations sorted by the cost
// estimate ncell + 8 P (descending; ties by configuration index; a configuration with a bad label,
// ncell < 0, costs 0 and goes last), each expanded to its nreal problems c * nreal + n. One CTA,
// bitonic sort of (cost, index) keys in shared memory, nconf <= FIT_ORDER_MAX.
constexpr int ORDER_NT = 1024;

__global__ void __launch_bounds__(ORDER_NT) k_fit_order(int nconf, int nreal,
                                                        const int* __restrict__ Kdev,
                                                        const int* __restrict__ ncell,
                                                        int* __restrict__ order) {
  extern __shared__ unsigned long long okey[];
  int n2 = 1;
  while (n2 < nconf) n2 <<= 1;
  for (int i = threadIdx.x; i < n2; i += ORDER_NT) {
    unsigned long long k = ~0ULL;  // padding sorts last
    if (i < nconf) {
      const long long cost = (ncell ? (long long)max(ncell[i], 0) : 0LL) +
                             8LL * ((long long)Kdev[3 * i] + Kdev[3 * i + 1] + Kdev[3 * i + 2]);
      const unsigned inv = 0x7fffffffu - (unsigned)min(cost, 0x7fffffffLL);
      k = ((unsigned long long)inv << 32) | (unsigned)i;
    }
    okey[i] = k;
  }
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n2; i += ORDER_NT) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned long long a = okey[i], b = okey[j];
          if ((a > b) == up) {
            okey[i] = b;
            okey[j] = a;
          }
        }
      }
      __syncthreads();
    }
  for (long long t = threadIdx.x; t < (long long)nconf * nreal; t += ORDER_NT) {
    const int rank = (int)(t / nreal), r = (int)(t % nreal);
    const int c = (int)(okey[rank] & 0xffffffffu);
    order[t] = c * nreal + r;
  }
}

// Problem descriptors of the fit and the reconstruction: problem q = c * nreal + n; its parameters
// start at nreal * coff[c] + n * P_c (coff the exclusive prefix sum of P_c) and its SED tables at
// row nreal * roff[c] + n * rows_c (roff that of rows_c = K_d + 2 K_T + K_s). One CTA.
constexpr int DESC_NT = 1024;

__global__ void __launch_bounds__(DESC_NT) k_fit_desc(int nconf, int nreal, const int* __restrict__ Kdev,
                                                      ProbDesc* __restrict__ probs) {
  __shared__ long long part[DESC_NT], rpart[DESC_NT];
  const int chunk = (nconf + DESC_NT - 1) / DESC_NT;
  const int c0 = min(nconf, (int)threadIdx.x * chunk), c1 = min(nconf, c0 + chunk);
  long long sum = 0, rsum = 0;
  for (int c = c0; c < c1; ++c) {
    sum += (long long)Kdev[3 * c] + Kdev[3 * c + 1] + Kdev[3 * c + 2];
    rsum += (long long)Kdev[3 * c] + 2LL * Kdev[3 * c + 1] + Kdev[3 * c + 2];
  }
  part[threadIdx.x] = sum;
  rpart[threadIdx.x] = rsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0, rrun = 0;
    for (int t = 0; t < DESC_NT; ++t) {
      const long long v = part[t], rv = rpart[t];
      part[t] = run;
      rpart[t] = rrun;
      run += v;
      rrun += rv;
    }
  }
  __syncthreads();
  long long coff = part[threadIdx.x], roff = rpart[threadIdx.x];
  for (int c = c0; c < c1; ++c) {
    const int kd = Kdev[3 * c], kt = Kdev[3 * c + 1], ks = Kdev[3 * c + 2];
    const int P = kd + kt + ks, rows = kd + 2 * kt + ks;
    for (int n = 0; n < nreal; ++n) {
      ProbDesc d;
      d.conf = c;
      d.real = n;
      d.Kd = kd;
      d.KT = kt;
      d.Ks = ks;
      d.P = P;
      d.poff = (long long)nreal * coff + (long long)n * P;
      d.toff = (long long)nreal * roff + (long long)n * rows;
      probs[(long long)c * nreal + n] = d;
    }
    coff += P;
    roff += rows;
  }
}

int launch_fit_desc(int nconf, int nreal, const int* K_dev, ProbDesc* probs, cudaStream_t s) {
  if (nconf == 0 || nreal == 0) return CSX_OK;
  k_fit_desc<<<1, DESC_NT, 0, s>>>(nconf, nreal, K_dev, probs);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

int launch_fit_order(int nconf, int nreal, const int* K_dev, const int* ncell, int* order,
                     cudaStream_t s) {
  if (nconf == 0 || nreal == 0) return CSX_OK;
  if (nconf > FIT_ORDER_MAX) return fail(CSX_EINVAL, "too many configurations for the device order");
  int n2 = 1;
  while (n2 < nconf) n2 <<= 1;
  const size_t smem = (size_t)n2 * sizeof(unsigned long long);
  CSX_CUDA(cudaFuncSetAttribute(k_fit_order, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(FIT_ORDER_MAX * sizeof(unsigned long long))));
  k_fit_order<<<1, ORDER_NT, smem, s>>>(nconf, nreal, K_dev, ncell, order);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

int launch_cells(int npix, int nconf, const int* labels, const int* K_dev, int* perm, int* cell_off,
                 int* ncell, cudaStream_t s) {
  if (nconf == 0) return CSX_OK;
  k_cells<<<nconf, CELL_NT, 0, s>>>(npix, labels, K_dev, perm, cell_off, ncell);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

}  // namespace csx
