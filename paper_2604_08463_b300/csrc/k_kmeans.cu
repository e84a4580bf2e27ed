// Seeded spherical K-means patches (Sec. 2.2) on the device: the Lloyd iterations that turn the
// pixel-centre unit vectors into patch labels, for many cluster counts at once (one CTA per
// labeling). The arithmetic is the input generator's, operation by operation in float64 and in
// the same order, so the labels are bit-exact with it:
//   assignment: the largest dot product (x cx + y cy) + z cz (each product and sum rounded once,
//               no fused multiply-add), the first cluster on ties;
//   stop:       when an assignment repeats the previous one, or after max_iter assignments;
//   centroids:  member sums accumulated in increasing pixel order (the pixels are placed in a
//               list grouped by cluster, in pixel order within a cluster, by one warp walking
//               them in order; the thread owning a cluster then adds its members), an emptied
//               cluster re-seeded at the pixel with the
//               smallest best dot product (stable order: the i-th emptied cluster takes the i-th),
//               renormalised by sqrt((x x + y y) + z z) (a zero norm counts as 1);
//   labels:     renumbered 0..K_eff-1 in order of first appearance.
// The assignment screens the clusters in FP32 first (B300's FP64 rate is a small fraction of its
// FP32 rate): with unit vectors the FP32 dot product is within 3e-7 of the FP64 one, so every
// cluster whose FP32 value is within KM_SCREEN of the FP32 maximum is evaluated in FP64 as above
// (in index order, the first of equal maxima kept), which contains the FP64 maximum: the labels
// stay bit-exact.
// K >= n gives one pixel per patch and K <= 1 a single patch, as in the generator.
#include <cmath>

#include "csx_host.h"

namespace csx {

constexpr int KM_NT = 256;
constexpr int KM_KMAX = KMEANS_KMAX;  // clusters per labeling (centroids, sums in shared memory)
constexpr float KM_SCREEN = 2e-6f;    // twice a bound of |FP32 - FP64| dot product (1e-6 > 3e-7)

// float4 copies of the centroids follow the double arrays, 16-byte aligned
__host__ __device__ constexpr size_t km_f4_offset(int kmax) {
  return ((size_t)kmax * (6 * sizeof(double) + 2 * sizeof(int)) + 15) & ~size_t(15);
}

__device__ __forceinline__ double km_dot(double x, double y, double z, double cx, double cy,
                                         double cz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, cx), __dmul_rn(y, cy)), __dmul_rn(z, cz));
}

struct KmArgs {
  const double* vec;     // [n][3]
  int n, nlab, max_iter;
  const int* K;          // [nlab] (device)
  const long long* ioff; // [nlab] offsets into init (device)
  const int* init;       // concatenated starting pixels
  int* labels;           // [nlab][n] (output; also the working assignment)
  double* best;          // [nlab][n] scratch
  int* members;          // [nlab][n] scratch: pixels grouped by cluster
  int* iters;            // [nlab] or NULL
};

__global__ void __launch_bounds__(KM_NT) k_kmeans(const KmArgs a) {
  extern __shared__ double km_smem[];
  __shared__ double s_bb[KM_NT / 32];
  __shared__ long long s_bp[KM_NT / 32];
  __shared__ long long s_pick;
  const int L = blockIdx.x, tid = threadIdx.x, n = a.n;
  const int K = a.K[L];
  int* lab = a.labels + (long long)L * n;
  double* best = a.best + (long long)L * n;
  int* members = a.members + (long long)L * n;
  if (K <= 1 || K >= n) {
    for (int p = tid; p < n; p += KM_NT) lab[p] = (K <= 1) ? 0 : p;
    if (a.iters && tid == 0) a.iters[L] = 0;
    return;
  }
  double* cent = km_smem;             // [K][3]
  double* sums = km_smem + 3 * K;     // [K][3]
  int* cnt = reinterpret_cast<int*>(km_smem + 6 * K);  // [K]
  float4* cf = reinterpret_cast<float4*>(reinterpret_cast<char*>(km_smem) + km_f4_offset(K));
  const int* init = a.init + a.ioff[L];
  for (int k = tid; k < K; k += KM_NT) {
    const int p = init[k];
    cent[3 * k] = a.vec[3 * p];
    cent[3 * k + 1] = a.vec[3 * p + 1];
    cent[3 * k + 2] = a.vec[3 * p + 2];
    cf[k] = make_float4((float)cent[3 * k], (float)cent[3 * k + 1], (float)cent[3 * k + 2], 0.f);
  }
  __syncthreads();
  int it = 0;
  for (; it < a.max_iter; ++it) {
    // ---- assignment --------------------------------------------------------------------
    int changed = 0;
    for (int p = tid; p < n; p += KM_NT) {
      const double x = a.vec[3 * p], y = a.vec[3 * p + 1], z = a.vec[3 * p + 2];
      const float xf = (float)x, yf = (float)y, zf = (float)z;
      // FP32 maximum and runner-up (the first index of the maximum kept)
      float b32 = -INFINITY, r32 = -INFINITY;
      int k32 = 0;
      for (int k = 0; k < K; ++k) {
        const float4 c = cf[k];
        const float v = fmaf(zf, c.z, fmaf(yf, c.y, xf * c.x));
        if (v > b32) {
          r32 = b32;
          b32 = v;
          k32 = k;
        } else {
          r32 = fmaxf(r32, v);
        }
      }
      const float thr = b32 - KM_SCREEN;
      double bv = -INFINITY;
      int bk = 0;
      if (r32 < thr) {
        // a single candidate: it is the FP64 maximum
        bk = k32;
        bv = km_dot(x, y, z, cent[3 * k32], cent[3 * k32 + 1], cent[3 * k32 + 2]);
      } else {
        for (int k = 0; k < K; ++k) {
          const float4 c = cf[k];
          if (fmaf(zf, c.z, fmaf(yf, c.y, xf * c.x)) >= thr) {
            const double v = km_dot(x, y, z, cent[3 * k], cent[3 * k + 1], cent[3 * k + 2]);
            if (v > bv) {
              bv = v;
              bk = k;
            }
          }
        }
      }
      if (it == 0 || lab[p] != bk) changed = 1;
      lab[p] = bk;
      best[p] = bv;
    }
    changed = __syncthreads_or(changed);
    if (!changed) break;
    // ---- member sums, in pixel order, by the thread owning the cluster ------------------------
    // counts, then each cluster's start in the member list (warp 0: an exclusive scan over K)
    int* cur = cnt + K;  // [K] placement cursor
    for (int k = tid; k < K; k += KM_NT) cnt[k] = 0;
    __syncthreads();
    for (int p = tid; p < n; p += KM_NT) atomicAdd(&cnt[lab[p]], 1);
    __syncthreads();
    if (tid < 32) {
      const int per = (K + 31) / 32, k0 = min(K, tid * per), k1 = min(K, k0 + per);
      int tot = 0;
      for (int k = k0; k < k1; ++k) tot += cnt[k];
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += y;
      }
      int run = incl - tot;
      for (int k = k0; k < k1; ++k) {
        cur[k] = run;
        run += cnt[k];
      }
      __syncwarp();
      // placement in pixel order: lanes with equal labels take consecutive slots, lowest lane first
      for (int base = 0; base < n; base += 32) {
        const int p = base + tid;
        const int l = p < n ? lab[p] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, l);
        const int rank = __popc(grp & ((1u << tid) - 1u));
        const int c0 = (l >= 0) ? cur[l] : 0;
        __syncwarp();
        if (l >= 0) {
          members[c0 + rank] = p;
          if (rank == 0) cur[l] = c0 + __popc(grp);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int k = tid; k < K; k += KM_NT) {
      const int e = cur[k], b = e - cnt[k];
      double sx = 0.0, sy = 0.0, sz = 0.0;
      for (int i = b; i < e; ++i) {
        const int p = members[i];
        sx = __dadd_rn(sx, a.vec[3 * p]);
        sy = __dadd_rn(sy, a.vec[3 * p + 1]);
        sz = __dadd_rn(sz, a.vec[3 * p + 2]);
      }
      sums[3 * k] = sx;
      sums[3 * k + 1] = sy;
      sums[3 * k + 2] = sz;
    }
    __syncthreads();
    // ---- emptied clusters, in index order, take the pixels of smallest best value ---------------
    long long prev = -1;  // previous pick: pixels are taken in (best, index) order
    double prev_b = -INFINITY;
    for (int e = 0; e < K; ++e) {
      if (cnt[e] != 0) continue;  // uniform: every thread reads the same shared value
      double bb = INFINITY;
      long long bp = (long long)n;
      for (int p = tid; p < n; p += KM_NT) {
        const double b = best[p];
        const bool after = (b > prev_b) || (b == prev_b && p > prev);
        if (after && (b < bb || (b == bb && p < bp))) {
          bb = b;
          bp = p;
        }
      }
      // block-wide minimum of (bb, bp)
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, bb, o);
        const long long op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (ob < bb || (ob == bb && op < bp)) {
          bb = ob;
          bp = op;
        }
      }
      __syncthreads();
      if ((tid & 31) == 0) {
        s_bb[tid >> 5] = bb;
        s_bp[tid >> 5] = bp;
      }
      __syncthreads();
      if (tid == 0) {
        double b0 = s_bb[0];
        long long p0 = s_bp[0];
        for (int w = 1; w < KM_NT / 32; ++w)
          if (s_bb[w] < b0 || (s_bb[w] == b0 && s_bp[w] < p0)) {
            b0 = s_bb[w];
            p0 = s_bp[w];
          }
        if (p0 >= n) p0 = n - 1;  // unreachable: fewer clusters than pixels can be emptied
        s_pick = p0;
        sums[3 * e] = a.vec[3 * p0];
        sums[3 * e + 1] = a.vec[3 * p0 + 1];
        sums[3 * e + 2] = a.vec[3 * p0 + 2];
      }
      __syncthreads();
      prev = s_pick;
      prev_b = best[prev];
    }
    // ---- renormalised centroids ---------------------------------------------------------
    for (int k = tid; k < K; k += KM_NT) {
      const double x = sums[3 * k], y = sums[3 * k + 1], z = sums[3 * k + 2];
      double nr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
      if (nr == 0.0) nr = 1.0;
      cent[3 * k] = __ddiv_rn(x, nr);
      cent[3 * k + 1] = __ddiv_rn(y, nr);
      cent[3 * k + 2] = __ddiv_rn(z, nr);
      cf[k] = make_float4((float)cent[3 * k], (float)cent[3 * k + 1], (float)cent[3 * k + 2], 0.f);
    }
    __syncthreads();
  }
  if (a.iters && tid == 0) a.iters[L] = it;
  // ---- renumber by first appearance -------------------------------------------------------------
  int* first = cnt;  // reuse: first pixel of each cluster
  for (int k = tid; k < K; k += KM_NT) first[k] = n;
  __syncthreads();
  for (int p = tid; p < n; p += KM_NT) atomicMin(first + lab[p], p);
  __syncthreads();
  int* remap = reinterpret_cast<int*>(sums);  // reuse: new number of each cluster
  for (int k = tid; k < K; k += KM_NT) {
    int r = 0;
    const int fk = first[k];
    for (int j = 0; j < K; ++j) r += (first[j] < fk) ? 1 : 0;
    remap[k] = (fk < n) ? r : -1;
  }
  __syncthreads();
  for (int p = tid; p < n; p += KM_NT) lab[p] = remap[lab[p]];
}

size_t kmeans_smem(int kmax) { return km_f4_offset(kmax) + (size_t)kmax * sizeof(float4); }

int launch_kmeans(const double* vec, int n, int nlab, const int* K_dev, const long long* ioff_dev,
                  const int* init, int max_iter, int kmax, int* labels, double* best, int* members,
                  int* iters, cudaStream_t s) {
  if (nlab == 0) return CSX_OK;
  KmArgs a;
  a.vec = vec;
  a.n = n;
  a.nlab = nlab;
  a.max_iter = max_iter;
  a.K = K_dev;
  a.ioff = ioff_dev;
  a.init = init;
  a.labels = labels;
  a.best = best;
  a.members = members;
  a.iters = iters;
  const size_t smem = kmeans_smem(kmax < 1 ? 1 : kmax);
  CSX_CUDA(cudaFuncSetAttribute(k_kmeans, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kmeans_smem(KM_KMAX)));
  k_kmeans<<<nlab, KM_NT, smem, s>>>(a);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

}  // namespace csx
