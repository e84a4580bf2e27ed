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

int launch_cells(int npix, int nconf, const int* labels, const int* K_dev, int* perm, int* cell_off,
                 int* ncell, cudaStream_t s) {
  if (nconf == 0) return CSX_OK;
  k_cells<<<nconf, CELL_NT, 0, s>>>(npix, labels, K_dev, perm, cell_off, ncell);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

}  // namespace csx
