// SED tables, the mixing matrix (Eq. 5) and the streaming likelihood / adjoint-gradient kernel
// (Eqs. 3-4 over the patches of Sec. 2.2; gradient of Sec. 3.3.1).
#include "csx_host.h"
#include "csx_tma.cuh"

#include <atomic>

namespace csx {

// Count of bounded waits that gave up (a tensor copy that did not arrive within the bound) since the
// last device_timeouts() on this device; the affected problem's L is also set to NaN.
__device__ unsigned int g_wait_timeouts;

int device_timeouts(cudaStream_t s, unsigned* count) {
  CSX_CUDA(cudaStreamSynchronize(s));
  unsigned v = 0;
  CSX_CUDA(cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)));
  if (v) {
    const unsigned zero = 0;
    CSX_CUDA(cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(zero)));
  }
  *count = v;
  return CSX_OK;
}

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
// Cell plan. Every pixel of a cell (equal (l_d, l_T, l_s)) shares its Gram-Schmidt scalars and band
// vectors (see run_scalars), so they are formed once per (problem, cell) by one thread each, before
// the streaming kernel, instead of once per run of equal labels inside it.
template <bool GRAD>
__global__ void k_cell_tables(const SpecArgs a, float* __restrict__ ctab) {
  float n0 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) n0 += a.ninv_band[f];
  const long long total = (long long)a.nprob * a.ncell;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / a.ncell), c = (int)(i % a.ncell);
    const int4 t = a.cell_lab[c];
    const float* tab = a.tables + (long long)q * a.rows * NB;
    float* out = ctab + i * CELL_TAB;
    run_scalars<GRAD>(tab + (long long)t.x * NB, tab + (long long)(a.Kd + t.y) * NB,
                      tab + (long long)(a.Kd + a.KT + t.y) * NB,
                      tab + (long long)(a.Kd + 2 * a.KT + t.z) * NB, a.ninv_band, a.bands, n0, out,
                      out + 16);
  }
}

int launch_cell_tables(const SpecArgs& a, bool grad, float* ctab, cudaStream_t s) {
  const long long total = (long long)a.nprob * a.ncell;
  if (total == 0) return CSX_OK;
  const long long blocks = (total + 127) / 128;
  const int g = (int)(blocks < 148 * 16 ? blocks : 148 * 16);
  if (grad) k_cell_tables<true><<<g, 128, 0, s>>>(a, ctab);
  else k_cell_tables<false><<<g, 128, 0, s>>>(a, ctab);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

// Each pixel's cell and each cell's labels from the sorted cell structure of launch_cells: sorted
// position i belongs to the cell c with cell_off[c] <= i < cell_off[c + 1] (binary search).
__global__ void k_plan_cells(int npix, int ncell, const int* __restrict__ labels,
                             const int* __restrict__ perm, const int* __restrict__ cell_off,
                             int* __restrict__ pcell, int4* __restrict__ cell_lab) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = ncell - 1;  // largest c with cell_off[c] <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cell_off[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const int px = perm[i];
    pcell[px] = lo;
    if (cell_off[lo] == i)
      cell_lab[lo] = make_int4(labels[px], labels[npix + px], labels[2 * npix + px], 0);
  }
}

int launch_plan_cells(int npix, int ncell, const int* labels, const int* perm, const int* cell_off,
                      int* pcell, int4* cell_lab, cudaStream_t s) {
  if (npix == 0 || ncell <= 0) return CSX_OK;
  const int blocks = (npix + 255) / 256;
  k_plan_cells<<<blocks < 148 * 8 ? blocks : 148 * 8, 256, 0, s>>>(npix, ncell, labels, perm,
                                                                   cell_off, pcell, cell_lab);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

// ---------------------------------------------------------------------------------------------
// Streaming likelihood (+ gradient) of Eqs. 3-4 and Sec. 3.3.1, TMA-staged. Grid (pixel blocks,
// problems); a CTA takes a contiguous range of tiles of TS_NT consecutive pixels of its problem
// (CSX_TS_CONTIG; else tiles strided by the grid). One thread keeps up to TS_S tiles of d (and of N^-1 for per-pixel
// noise) in flight with bulk-tensor copies into a ring of shared-memory stages (128-byte swizzled
// rows, so the per-pixel 16-byte reads are free of bank conflicts); every thread then reads its
// pixel from shared memory. Labels and hit weights of the next tile are fetched into registers one
// tile ahead; a stage is refilled after the barrier that follows its last read.
//
// Separable / homogeneous noise: the pixels of a tile are split into runs of consecutive pixels
// with equal labels (within a warp); the Gram-Schmidt scalars of each run -- and, for L alone and
// the first TS_RUNVEC / (warps) runs of a warp, its band vectors -- are formed by the run's head
// lane into its warp's part of the run table (run_scalars; CSX_TS_WARPRUNS, while the tile's data is
// still in flight; else by one thread per run of the tile into a block-wide table behind two more
// barriers), and every pixel is then evaluated in its run's basis
// (cell_pixel_vec from the stored vectors; cell_pixel from the SED table rows otherwise: with the
// gradient, the stored-vector form measured slower, its three extra vectors costing registers). Per-pixel noise: each pixel's own Gram-Schmidt solve (pixel_eval).
//
// L_p is accumulated in FP32 per thread (a few pixels) and in FP64 across the block, then added to
// L[problem] with one FP64 atomic per block; gradients go to a shared-memory copy of the problem's
// P-vector (one atomic per run of equal labels in a warp), flushed with one global atomic per
// touched parameter and block. A label outside [0, K_j) or a non-positive-definite A^T N A poisons
// L with NaN. Waits are bounded (about 2 s): on time-out the CTA waits (bounded) for its copies
// still in flight, poisons L with NaN and returns.
// ---------------------------------------------------------------------------------------------
// Tile schedule: pixels (= threads) per tile NT and pipeline stages S are template parameters; the
// schedule of a launch is the one selected with set_stream_schedule (csx_stream_schedule), default
// (128, 2), the measured best on the full-sky nside-64 case; resident CTAs per SM asked of ptxas:
// 512 / NT. Build-time switches of the algorithm (the defaults are the measured best on B300):
#ifndef CSX_TS_WARPRUNS
#define CSX_TS_WARPRUNS 1  // 1: each warp forms the scalars of its own runs (no block-wide table)
#endif
#ifndef CSX_TS_CONTIG
#define CSX_TS_CONTIG 1  // 1: each CTA streams a contiguous range of tiles (else tiles strided by the grid)
#endif
#ifndef CSX_TS_RUNCACHE
#define CSX_TS_RUNCACHE 0  // 1: a warp keeps its runs' scalars across tiles (with CSX_TS_WARPRUNS)
#endif
#ifndef CSX_TS_GRADVEC
#define CSX_TS_GRADVEC 0  // 1: the gradient kernel also evaluates pixels from the run vectors
#endif
constexpr long long TS_WAIT_CYCLES = 4000000000LL;  // bound of one wait, in SM clock cycles
constexpr int TS_RUNVEC = 32;  // runs per tile whose band vectors are kept in the run table
constexpr bool TS_GRADVEC = CSX_TS_GRADVEC != 0;
constexpr bool TS_WARPRUNS = CSX_TS_WARPRUNS != 0;
constexpr bool TS_CONTIG = CSX_TS_CONTIG != 0;
constexpr bool TS_RUNCACHE = CSX_TS_RUNCACHE != 0;

template <int NOISE, int TS_NT, int TS_S, bool CELLS = false>
struct TsShape {
  static constexpr bool PIXNOISE = NOISE == CSX_NOISE_PERPIXEL;         // N^-1 staged per pixel
  static constexpr bool RUNS = !PIXNOISE && !CELLS;                      // in-kernel run table
  static constexpr int DB = TS_NT * 128;                                 // d: [TS_NT][2][16] floats
  static constexpr int NBY = PIXNOISE ? TS_NT * 64 : 0;                  // N^-1: [TS_NT][16] floats
  static constexpr int SB = DB + NBY;                                    // bytes per stage
  static constexpr int RB = RUNS ? TS_NT * (16 * 4 + 16) + TS_RUNVEC * 80 * 4 : 0;  // run table
  static constexpr size_t smem(int P, bool smem_grad) {
    return 1024 + (size_t)TS_S * SB + RB + (smem_grad ? (size_t)P * sizeof(float) : 0);
  }
};

template <int NOISE, bool GRAD, bool SMEM_GRAD, int TS_NT, int TS_S, bool CELLS>
__global__ void __launch_bounds__(TS_NT, 512 / TS_NT)
    k_spectral_tma(const __grid_constant__ CUtensorMap md, const __grid_constant__ CUtensorMap mn,
                   const SpecArgs a) {
  constexpr int TS_NW = TS_NT / 32;
  constexpr int TS_RUNVEC_W = TS_RUNVEC / TS_NW;  // run vectors per warp
  using Sh = TsShape<NOISE, TS_NT, TS_S, CELLS>;
  extern __shared__ __align__(16) unsigned char ts_smem[];
  __shared__ __align__(8) uint64_t full[TS_S];
  __shared__ double sred[TS_NW];
  __shared__ int s_cnt[2][TS_NW];
  const unsigned off = smem_addr(ts_smem);
  unsigned char* stage0 = ts_smem + (((off + 1023u) & ~1023u) - off);  // 1024-byte aligned ring
  float* s_sc = reinterpret_cast<float*>(stage0 + TS_S * Sh::SB);      // [TS_NT][16] run scalars
  int4* s_trip = reinterpret_cast<int4*>(s_sc + (Sh::RUNS ? TS_NT * 16 : 0));  // [TS_NT] labels
  float* s_vec = reinterpret_cast<float*>(s_trip + (Sh::RUNS ? TS_NT : 0));    // [TS_RUNVEC][80]
  float* sgrad = reinterpret_cast<float*>(stage0 + TS_S * Sh::SB + Sh::RB);
  const int q = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntile = (a.npix + TS_NT - 1) / TS_NT;
  // tiles of this CTA: tile(j) = t0 + j (a contiguous range) or blockIdx.x + j gridDim.x (strided)
  const int t0 = TS_CONTIG ? (int)(((long long)blockIdx.x * ntile) / gridDim.x) : (int)blockIdx.x;
  const int tstep = TS_CONTIG ? 1 : (int)gridDim.x;
  const int my = TS_CONTIG ? (int)((((long long)blockIdx.x + 1) * ntile) / gridDim.x) - t0
                           : (((int)blockIdx.x < ntile) ? (ntile - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0);
  const float* tab = a.tables + (long long)q * a.rows * NB;
  float* ggl = GRAD ? a.grad + (long long)q * a.P : nullptr;
  float* gacc = SMEM_GRAD ? sgrad : ggl;
  if (tid == 0) {
    for (int s = 0; s < TS_S; ++s) mbar_init(&full[s], 1);
    mbar_init_fence();
    tma_prefetch_map(&md);
  }
  if (GRAD && SMEM_GRAD)
    for (int i = tid; i < a.P; i += TS_NT) sgrad[i] = 0.f;
  __syncthreads();
  auto issue = [&](int j) {
    const int s = j % TS_S;
    const int p0 = (t0 + j * tstep) * TS_NT;
    unsigned char* st = stage0 + s * Sh::SB;
    mbar_expect_tx(&full[s], Sh::SB);
    tma_load_3d(st, &md, 0, p0, q, &full[s]);
    if (NOISE == CSX_NOISE_PERPIXEL) tma_load_2d(st + Sh::DB, &mn, 0, p0, &full[s]);
  };
  if (tid == 0)
    for (int j = 0; j < TS_S && j < my; ++j) issue(j);
  const int* ld = a.labels;
  const int* lt = a.labels + a.npix;
  const int* ls = a.labels + 2 * a.npix;
  int nkd = 0, nkt = 0, nks = 0, ncl = 0;
  float nw = 1.f;
  auto fetch = [&](int j) {
    const int p = (t0 + j * tstep) * TS_NT + tid;
    if (j < my && p < a.npix) {
      if (CELLS) {
        ncl = __ldg(a.pcell + p);
      } else {
        nkd = __ldg(ld + p);
        nkt = __ldg(lt + p);
        nks = __ldg(ls + p);
      }
      if (NOISE == CSX_NOISE_SEPARABLE) nw = __ldg(a.w + p);
    }
  };
  fetch(0);
  float n0 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) n0 += a.ninv_band[f];
  float acc = 0.f;
  bool bad = false;
  int j = 0;
  bool timed_out = false;
  constexpr bool WR = Sh::RUNS && TS_WARPRUNS && !CELLS;
  int wnent = 0;  // entries of this warp's run cache
  for (; j < my; ++j) {
    const int s = j % TS_S;
    // per-warp run table: the labels of this tile are already in registers, so the head lane of
    // each run of equal labels in a warp forms the run's scalars while the tile's data is in flight
    int wkd = nkd, wkt = nkt, wks = nks, wslot = 0;
    bool wvalid = false;
    if (WR) {
      const int pw = (t0 + j * tstep) * TS_NT + tid;
      wvalid = pw < a.npix && (unsigned)wkd < (unsigned)a.Kd && (unsigned)wkt < (unsigned)a.KT &&
               (unsigned)wks < (unsigned)a.Ks;
      const int pkd = __shfl_up_sync(0xffffffffu, wkd, 1), pkt = __shfl_up_sync(0xffffffffu, wkt, 1),
                pks = __shfl_up_sync(0xffffffffu, wks, 1);
      const bool pv = __shfl_up_sync(0xffffffffu, wvalid, 1);
      const bool whead = wvalid && (lane == 0 || !pv || wkd != pkd || wkt != pkt || wks != pks);
      const unsigned whb = __ballot_sync(0xffffffffu, whead);
      __syncwarp();  // the warp's reads of the previous tile's table are done
      bool miss = whead;
      if (TS_RUNCACHE) {
        // runs seen by this warp in earlier tiles keep their slot: look the label triple up
        int found = -1;
        for (int e = 0; e < wnent; ++e) {  // wnent is the same in every lane
          const int4 t = s_trip[warp * 32 + e];
          if (t.x == wkd && t.y == wkt && t.z == wks) found = e;
        }
        const unsigned mm = __ballot_sync(0xffffffffu, whead && found < 0);
        if (wnent + __popc(mm) > 32) {  // table full: start it again with this tile's runs
          wnent = 0;
          found = -1;
        }
        miss = whead && found < 0;
        const unsigned mb = __ballot_sync(0xffffffffu, miss);
        wslot = miss ? wnent + __popc(mb & ((1u << lane) - 1u)) : found;
        wnent += __popc(mb);
      } else {
        wslot = __popc(whb & ((2u << lane) - 1u)) - 1;
      }
      if (miss) {
        if (TS_RUNCACHE) s_trip[warp * 32 + wslot] = make_int4(wkd, wkt, wks, 0);
        run_scalars<GRAD>(tab + (long long)wkd * NB, tab + (long long)(a.Kd + wkt) * NB,
                          tab + (long long)(a.Kd + a.KT + wkt) * NB,
                          tab + (long long)(a.Kd + 2 * a.KT + wks) * NB, a.ninv_band, a.bands,
                          n0, s_sc + 16 * (warp * 32 + wslot),
                          ((!GRAD || TS_GRADVEC) && wslot < TS_RUNVEC_W)
                              ? s_vec + 80 * (warp * TS_RUNVEC_W + wslot) : nullptr);
      }
      if (TS_RUNCACHE) {  // every pixel takes its run head's slot
        const unsigned upto = whb & ((2u << lane) - 1u);
        const int hl = upto ? 31 - __clz(upto) : lane;
        wslot = __shfl_sync(0xffffffffu, wslot, hl);
      }
    }
    const bool ok = mbar_wait_bounded(&full[s], (unsigned)(j / TS_S) & 1u, TS_WAIT_CYCLES);
    const float4* row = reinterpret_cast<const float4*>(stage0 + s * Sh::SB);
    float dq[NB], du[NB], nn[NB];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 v = row[swz128(tid, k)];
      const float4 u = row[swz128(tid, 4 + k)];
      dq[4 * k] = v.x; dq[4 * k + 1] = v.y; dq[4 * k + 2] = v.z; dq[4 * k + 3] = v.w;
      du[4 * k] = u.x; du[4 * k + 1] = u.y; du[4 * k + 2] = u.z; du[4 * k + 3] = u.w;
    }
    if (NOISE == CSX_NOISE_PERPIXEL) {
      const float4* nr = reinterpret_cast<const float4*>(stage0 + s * Sh::SB + Sh::DB);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 v = nr[swz64(tid, k)];
        nn[4 * k] = v.x; nn[4 * k + 1] = v.y; nn[4 * k + 2] = v.z; nn[4 * k + 3] = v.w;
      }
    }
    int kd = nkd, kt = nkt, ks = nks;
    const int cl = ncl;
    const float wp = nw;
    fetch(j + 1);
    const int p = (t0 + j * tstep) * TS_NT + tid;
    bool valid = p < a.npix;
    if (CELLS) {
      if (valid && (unsigned)cl >= (unsigned)a.ncell) {
        bad = true;
        valid = false;
      }
    } else if (valid && ((unsigned)kd >= (unsigned)a.Kd || (unsigned)kt >= (unsigned)a.KT ||
                         (unsigned)ks >= (unsigned)a.Ks)) {
      bad = true;
      valid = false;
    }
    // runs of equal labels within the warp: a valid pixel starts one at lane 0, after an invalid
    // pixel or where a label changes
    bool head = false;
    unsigned hb = 0u;
    if (Sh::RUNS && !WR && !CELLS) {
      const int pkd = __shfl_up_sync(0xffffffffu, kd, 1), pkt = __shfl_up_sync(0xffffffffu, kt, 1),
                pks = __shfl_up_sync(0xffffffffu, ks, 1);
      const bool pv = __shfl_up_sync(0xffffffffu, valid, 1);
      head = valid && (lane == 0 || !pv || kd != pkd || kt != pkt || ks != pks);
      hb = __ballot_sync(0xffffffffu, head);
      if (lane == 0) s_cnt[j & 1][warp] = __popc(hb);
    }
    if (__syncthreads_or(!ok)) {  // every thread holds its pixel: the stage may be refilled
      timed_out = true;
      break;
    }
    if (tid == 0 && j + TS_S < my) issue(j + TS_S);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (CELLS) {
      // the cell's scalars and band vectors were formed for this problem before the launch
      if (valid) {
        const float* ct = a.ctab + ((long long)q * a.ncell + cl) * CELL_TAB;
        float sc[NSC];
        load_scalars(ct, sc);
        const float wpx = NOISE == CSX_NOISE_SEPARABLE ? wp : 1.f;
        acc += cell_pixel_vec<GRAD>(dq, du, a.ninv_band, ct + 16, sc, wpx, g0, g1, g2);
        if (GRAD) {
          const int4 t = __ldg(a.cell_lab + cl);
          kd = t.x;
          kt = t.y;
          ks = t.z;
        }
      }
    } else if (WR) {
      if (valid) {  // the block barrier above published the warp's run table
        float sc[NSC];
        load_scalars(s_sc + 16 * (warp * 32 + wslot), sc);
        const float wpx = NOISE == CSX_NOISE_SEPARABLE ? wp : 1.f;
        if ((!GRAD || TS_GRADVEC) && wslot < TS_RUNVEC_W)
          acc += cell_pixel_vec<GRAD>(dq, du, a.ninv_band, s_vec + 80 * (warp * TS_RUNVEC_W + wslot),
                                      sc, wpx, g0, g1, g2);
        else
          acc += cell_pixel<GRAD>(dq, du, tab + (long long)kd * NB,
                                  tab + (long long)(a.Kd + kt) * NB,
                                  tab + (long long)(a.Kd + a.KT + kt) * NB,
                                  tab + (long long)(a.Kd + 2 * a.KT + ks) * NB, a.ninv_band,
                                  a.bands, sc, wpx, g0, g1, g2);
      }
    } else if (Sh::RUNS) {
      int roff = 0, nruns = 0;
#pragma unroll
      for (int w = 0; w < TS_NW; ++w) {
        const int c = s_cnt[j & 1][w];
        roff += (w < warp) ? c : 0;
        nruns += c;
      }
      const int rid = roff + __popc(hb & ((2u << lane) - 1u)) - 1;  // this pixel's run
      if (head) s_trip[rid] = make_int4(kd, kt, ks, 0);
      __syncthreads();
      for (int r = tid; r < nruns; r += TS_NT) {
        const int4 t = s_trip[r];
        run_scalars<GRAD>(tab + (long long)t.x * NB, tab + (long long)(a.Kd + t.y) * NB,
                          tab + (long long)(a.Kd + a.KT + t.y) * NB,
                          tab + (long long)(a.Kd + 2 * a.KT + t.z) * NB, a.ninv_band, a.bands,
                          n0, s_sc + 16 * r, ((!GRAD || TS_GRADVEC) && r < TS_RUNVEC) ? s_vec + 80 * r : nullptr);
      }
      __syncthreads();
      if (valid) {
        float sc[NSC];
        load_scalars(s_sc + 16 * rid, sc);
        const float wpx = NOISE == CSX_NOISE_SEPARABLE ? wp : 1.f;
        if ((!GRAD || TS_GRADVEC) && rid < TS_RUNVEC)
          acc += cell_pixel_vec<GRAD>(dq, du, a.ninv_band, s_vec + 80 * rid, sc, wpx, g0, g1, g2);
        else
          acc += cell_pixel<GRAD>(dq, du, tab + (long long)kd * NB,
                                  tab + (long long)(a.Kd + kt) * NB,
                                  tab + (long long)(a.Kd + a.KT + kt) * NB,
                                  tab + (long long)(a.Kd + 2 * a.KT + ks) * NB, a.ninv_band,
                                  a.bands, sc, wpx, g0, g1, g2);
      }
    } else if (valid) {
      PixOut o;
      if (pixel_eval<GRAD, false>(dq, du, nn, tab + (long long)kd * NB,
                                  tab + (long long)(a.Kd + kt) * NB,
                                  tab + (long long)(a.Kd + a.KT + kt) * NB,
                                  tab + (long long)(a.Kd + 2 * a.KT + ks) * NB, a.bands, o)) {
        acc += o.chi2 - o.dnd;
        if (GRAD) {
          g0 = o.gbd;
          g1 = o.gtd;
          g2 = o.gbs;
        }
      } else {
        bad = true;
      }
    }
    if (GRAD) {
      if (!valid) kd = kt = ks = -1;
      warp_run_add3(gacc, kd, g0, gacc + a.Kd, kt, g1, gacc + a.Kd + a.KT, ks, g2);
    }
    if (CELLS && j + 1 < my) {
      // the next tile's cells (their indices arrived during this tile): the first lane of each run
      // of equal cells asks L1 for the cell's table entry (3 lines) and labels
      const int pc = __shfl_up_sync(0xffffffffu, ncl, 1);
      if (lane == 0 || ncl != pc) {
        const char* e = reinterpret_cast<const char*>(a.ctab + ((long long)q * a.ncell + ncl) * CELL_TAB);
        prefetch_l1(e);
        prefetch_l1(e + 128);
        prefetch_l1(e + 256);
        if (GRAD) prefetch_l1(a.cell_lab + ncl);
      }
    }
  }
  if (timed_out) {
    if (tid == 0) {
      for (int jj = j; jj < my && jj < j + TS_S; ++jj)
        (void)mbar_wait_bounded(&full[jj % TS_S], (unsigned)(jj / TS_S) & 1u, TS_WAIT_CYCLES);
      atomicAdd(a.L + q, (double)nan_f());
      atomicAdd(&g_wait_timeouts, 1u);
    }
    return;
  }
  const double tot = block_sum<TS_NT>(bad ? (double)nan_f() : (double)acc, sred);
  if (tid == 0) atomicAdd(a.L + q, tot);
  if (GRAD && SMEM_GRAD) {
    __syncthreads();
    for (int i = tid; i < a.P; i += TS_NT) {
      const float v = sgrad[i];
      if (v != 0.f) atomicAdd(ggl + i, v);
    }
  }
}

template <int NOISE, bool GRAD, bool SMEM_GRAD, int NT, int S, bool CELLS>
static int launch_tma_one(const CUtensorMap& md, const CUtensorMap& mn, const SpecArgs& a, dim3 grid,
                          cudaStream_t s) {
  using Sh = TsShape<NOISE, NT, S, CELLS>;
  const size_t smem = Sh::smem(a.P, GRAD && SMEM_GRAD);
  // the attribute covers the ring plus a P-vector of up to 16384 floats
  CSX_CUDA(cudaFuncSetAttribute(k_spectral_tma<NOISE, GRAD, SMEM_GRAD, NT, S, CELLS>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem(16384, true)));
  k_spectral_tma<NOISE, GRAD, SMEM_GRAD, NT, S, CELLS><<<grid, NT, smem, s>>>(md, mn, a);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

template <int NOISE, int NT, int S, bool CELLS>
static int launch_tma(const CUtensorMap& md, const CUtensorMap& mn, const SpecArgs& a, bool grad,
                      dim3 grid, cudaStream_t s) {
  if (!grad) return launch_tma_one<NOISE, false, false, NT, S, CELLS>(md, mn, a, grid, s);
  if (a.P <= 16384) return launch_tma_one<NOISE, true, true, NT, S, CELLS>(md, mn, a, grid, s);
  return launch_tma_one<NOISE, true, false, NT, S, CELLS>(md, mn, a, grid, s);
}

// Tensor maps of one launch: d as [problems][npix][32 floats] (box 32 x 256 x 1, 128-byte
// swizzle) and, for per-pixel noise, N^-1 as [npix][16 floats] (box 16 x 256, 64-byte swizzle).
// Returns false if the encoder is unavailable or refuses (the entry points have already checked
// that d and N^-1 are 16-byte aligned).
static bool make_maps(const SpecArgs& a, CUtensorMap* md, CUtensorMap* mn, int TS_NT) {
  if ((reinterpret_cast<uintptr_t>(a.d) & 15) != 0) return false;
  {
    const cuuint64_t dims[3] = {2 * NB, (cuuint64_t)a.npix, (cuuint64_t)a.nprob};
    const cuuint64_t str[2] = {2 * NB * sizeof(float), (cuuint64_t)a.npix * 2 * NB * sizeof(float)};
    const cuuint32_t box[3] = {2 * NB, TS_NT, 1};
    if (encode_tiled(md, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.d, dims, str, box,
                     CU_TENSOR_MAP_SWIZZLE_128B))
      return false;
  }
  if (a.noise_kind == CSX_NOISE_PERPIXEL) {
    if ((reinterpret_cast<uintptr_t>(a.ninv_pix) & 15) != 0) return false;
    const cuuint64_t dims[2] = {NB, (cuuint64_t)a.npix};
    const cuuint64_t str[1] = {NB * sizeof(float)};
    const cuuint32_t box[2] = {NB, TS_NT};
    if (encode_tiled(mn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.ninv_pix, dims, str, box,
                     CU_TENSOR_MAP_SWIZZLE_64B))
      return false;
  } else {
    *mn = *md;  // unused
  }
  return true;
}

// Tiles per CTA of the TMA kernel: up to 2048 pixels' worth, fewer when that would leave under
// 4 CTAs per resident CTA slot.
static int tma_grid_x(int npix, int nprob, int TS_NT) {
  const long long ntile = (npix + TS_NT - 1) / TS_NT;
  long long tpc = ntile * nprob / (148LL * (512 / TS_NT) * 4);
  const long long tmax = 2048 / TS_NT;
  tpc = tpc < 1 ? 1 : (tpc > tmax ? tmax : tpc);
  return (int)((ntile + tpc - 1) / tpc);
}

// The schedules the streaming kernel is built for: (pixels per tile, stages).
constexpr int TS_SCHED[][2] = {{128, 2}, {64, 2}, {64, 3}, {128, 3}, {128, 4}, {256, 2}};
constexpr int TS_NSCHED = sizeof(TS_SCHED) / sizeof(TS_SCHED[0]);
static std::atomic<int> g_sched{0};

int set_stream_schedule(int tile, int stages) {
  if (tile == 0 && stages == 0) {
    g_sched.store(0);
    return CSX_OK;
  }
  for (int i = 0; i < TS_NSCHED; ++i)
    if (TS_SCHED[i][0] == tile && TS_SCHED[i][1] == stages) {
      g_sched.store(i);
      return CSX_OK;
    }
  return fail(CSX_EINVAL, "unsupported streaming schedule (tile, stages)");
}

void get_stream_schedule(int* tile, int* stages) {
  const int i = g_sched.load();
  *tile = TS_SCHED[i][0];
  *stages = TS_SCHED[i][1];
}

template <int NT, int S>
static int launch_sched(const SpecArgs& b, bool grad, cudaStream_t s) {
  CUtensorMap md, mn;
  if (!make_maps(b, &md, &mn, NT)) return fail(CSX_ECUDA, "tensor-map encoding failed (cuTensorMapEncodeTiled)");
  const dim3 grid(tma_grid_x(b.npix, b.nprob, NT), b.nprob);
  if (b.pcell) {  // cell plan: separable or homogeneous noise only (checked by the entry point)
    if (b.noise_kind == CSX_NOISE_HOMOGENEOUS)
      return launch_tma<CSX_NOISE_HOMOGENEOUS, NT, S, true>(md, mn, b, grad, grid, s);
    return launch_tma<CSX_NOISE_SEPARABLE, NT, S, true>(md, mn, b, grad, grid, s);
  }
  switch (b.noise_kind) {
    case CSX_NOISE_HOMOGENEOUS: return launch_tma<CSX_NOISE_HOMOGENEOUS, NT, S, false>(md, mn, b, grad, grid, s);
    case CSX_NOISE_SEPARABLE: return launch_tma<CSX_NOISE_SEPARABLE, NT, S, false>(md, mn, b, grad, grid, s);
    default: return launch_tma<CSX_NOISE_PERPIXEL, NT, S, false>(md, mn, b, grad, grid, s);
  }
}

int launch_spectral(const SpecArgs& a, bool grad, cudaStream_t s) {
  if (a.nprob == 0 || a.npix == 0) return CSX_OK;
  const int sched = g_sched.load();
  // at most 65535 problems per launch (grid.y limit)
  for (int q0 = 0; q0 < a.nprob; q0 += 65535) {
    SpecArgs b = a;
    const int nq = (a.nprob - q0 < 65535) ? a.nprob - q0 : 65535;
    b.nprob = nq;
    b.tables = a.tables + (long long)q0 * a.rows * NB;
    b.d = a.d + (long long)q0 * a.npix * 2 * NB;
    b.beta = a.beta + (long long)q0 * a.P;
    b.L = a.L + q0;
    b.grad = a.grad ? a.grad + (long long)q0 * a.P : nullptr;
    b.ctab = a.ctab ? a.ctab + (long long)q0 * a.ncell * CELL_TAB : nullptr;
    int rc;
    switch (sched) {
      case 1: rc = launch_sched<64, 2>(b, grad, s); break;
      case 2: rc = launch_sched<64, 3>(b, grad, s); break;
      case 3: rc = launch_sched<128, 3>(b, grad, s); break;
      case 4: rc = launch_sched<128, 4>(b, grad, s); break;
      case 5: rc = launch_sched<256, 2>(b, grad, s); break;
      default: rc = launch_sched<128, 2>(b, grad, s); break;
    }
    if (rc) return rc;
  }
  return CSX_OK;
}

}  // namespace csx
