// Persistent batched fit beta* = argmin L(beta) (Eq. 7) over (configuration x realization)
// problems: one CTA per problem at a time, problems taken from an atomic work queue (the
// single-GPU analogue of the contiguous chunking of Sec. 3.1). Each CTA runs the whole fit:
//
//   likelihood + adjoint gradient (Eq. 4, Sec. 3.3.1), by one of two exact evaluations
//     MOMENT: separable noise N_p^-1 = w_p diag(n): every pixel of a cell (equal (l_d,l_T,l_s))
//             has the same A, so chi2 and its gradient need only the cell's weighted second
//             moments, kept as residual moments about a reference point (see build_moments and
//             eval_moment): one pass over the pixels per reference point, then each evaluation
//             costs O(cells), not O(pixels). The reference point is moved to the current point
//             (at most 6 times) when the fit converges far from it or a line search fails
//             there.
//     STREAM: per pixel, residual form (any diagonal noise).
//   the optimiser: L-BFGS (memory m) in variables scaled by the square root of the Gauss-Newton
//     diagonal at the start point; box bounds handled as in App. A: parameters at a bound whose
//     gradient points outward are held (active set), the step is limited by the distance to the
//     nearest bound and the limiting parameter is clamped; line search on the approximate Wolfe
//     conditions (sufficient decrease tested through the directional derivative when function
//     differences are below rounding).
//   stop: every free parameter's quasi-Newton step and last step below xtol (physical units).
//
// Plain form (CSX_GRAD_FD): same optimiser, gradient by central differences of the forward
// likelihood (2P extra evaluations per gradient), STREAM evaluation only.
//
// No CTA waits on another: the only shared state is the queue counter (one atomicAdd per problem).
#include "csx_host.h"

namespace csx {

// Build-time tuning switches (the defaults are the measured best on B300):
//   CSX_FIT_MIN_BLOCKS     minimum resident 128-thread moment-path CTAs per SM asked of ptxas.
//   CSX_FIT_NEAR           step size (in xtol) below which the reference point first moves to
//                          the current point (0: only at convergence).
#ifndef CSX_FIT_NEAR
#define CSX_FIT_NEAR 0.f
#endif
#ifndef CSX_FIT_MIN_BLOCKS
#define CSX_FIT_MIN_BLOCKS 3
#endif

constexpr int SMEM_P = 1024;   // parameter vectors up to this length accumulate in shared memory
constexpr int MAXM = 16;       // maximum L-BFGS memory

struct Ctx {
  int P, Kd, KT, Ks, rows, ncell, npix;
  const int* lab;     // [3][npix] of the configuration
  const int* perm;    // sorted pixels
  const int* coff;    // cell offsets
  const float* d;     // [npix][2][16] of the realization
  float *z, *g, *p, *zt, *gt, *hs, *x, *gacc, *hacc, *S, *Y, *tab, *mom;
  float *tabr, *xr;   // moment path: SED tables and parameters of the reference point
  float *gw, *hw;     // warp-private partial gradients / Gauss-Newton diagonals [warps][P]
  int* trip;
  float* smem;        // moment path: dynamic shared memory (build staging, then per-thread rows)
};

struct Shared {
  double red[16];
  double rho[MAXM], alpha[MAXM];
  float gacc[SMEM_P], hacc[SMEM_P];
  float stage[8][32];  // per-warp staging of warp_run_accum3
};

// Gradient (and Gauss-Newton diagonal) accumulation without float atomics: each warp adds its
// run totals to its own partial P-vector in program order (warp_run_accum3), and the vectors are
// summed in warp order at the end of the evaluation, so every evaluation of the same point gives
// the same bits.
template <int NT>
__device__ __forceinline__ void partials_zero(const Ctx& c, bool want_h) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* gw = c.gw + (long long)warp * c.P;
  float* hw = c.hw + (long long)warp * c.P;
  for (int i = lane; i < c.P; i += 32) {
    gw[i] = 0.f;
    if (want_h) hw[i] = 0.f;
  }
  __syncwarp();
}

template <int NT>
__device__ __forceinline__ void partials_reduce(const Ctx& c, bool want_h) {
  __syncthreads();
  for (int i = threadIdx.x; i < c.P; i += NT) {
    float g = c.gw[i], h = want_h ? c.hw[i] : 0.f;
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) {
      g += c.gw[(long long)w * c.P + i];
      if (want_h) h += c.hw[(long long)w * c.P + i];
    }
    c.gacc[i] = g;
    if (want_h) c.hacc[i] = h;
  }
  __syncthreads();
}

__device__ __forceinline__ int ptype(const Ctx& c, int i) {
  return i < c.Kd ? 0 : (i < c.Kd + c.KT ? 1 : 2);
}

// ------------------------------------------------------------------------------ tables ----------
// The rows of table_entry; a dust-temperature patch's B and dlnB/dT entries of a band are formed by
// one thread from the same two expm1 values: with E = e^x - 1, x / (1 - e^-x) = x (1 + E) / E.
// STAGE (moment path): the parameters are first copied, coalesced, into the shared memory of the
// evaluation rows or the build staging (free until the tables are formed), so that each entry's
// read of its parameter is a shared-memory load rather than a dependent global one.
template <int NT, bool STAGE = false>
__device__ void fill_tables(const FitArgs& a, const Ctx& c, const float* x, float* tab) {
  if (STAGE && c.P <= 90 * NT) {
    for (int i = threadIdx.x; i < c.P; i += NT) c.smem[i] = x[i];
    __syncthreads();
    x = c.smem;
  }
  const int nd = c.Kd * NB, nt = c.KT * NB, n = nd + nt + c.Ks * NB;
  const Bands& b = a.bands;
  for (int i = threadIdx.x; i < n; i += NT) {
    const int f = i & 15;
    if (i < nd) {
      tab[i] = table_entry(b, i >> 4, f, c.Kd, c.KT, x);
    } else if (i < nd + nt) {
      const int j = (i - nd) >> 4;
      const float T = x[c.Kd + j];
      float vb = 0.f, vd = 0.f;
      if (f < b.nf) {
        if (T > 0.f) {
          const float x0 = b.xk0 / T, xf = b.xk[f] / T;
          const float E0 = expm1f(x0), Ef = expm1f(xf);
          vb = b.cd[f] * E0 / Ef;
          vd = (xf * (1.f + Ef) / Ef - x0 * (1.f + E0) / E0) / T;
        } else {
          vb = vd = nan_f();
        }
      }
      tab[(c.Kd + j) * NB + f] = vb;
      tab[(c.Kd + c.KT + j) * NB + f] = vd;
    } else {
      const int r = c.Kd + 2 * c.KT + ((i - nd - nt) >> 4);
      tab[r * NB + f] = table_entry(b, r, f, c.Kd, c.KT, x);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------ moments ---------
// Residual moments of a cell about a reference point beta_ref (tables c.tabr). Per pixel and Stokes,
// with A_r the cell's mixing matrix at beta_ref:
//   s = (A_r^T N A_r)^-1 A_r^T N d,   r = d - A_r s,   v = [r_0 .. r_14, s_0, s_1, s_2]
// and per cell M_c = sum_p w_p sum_s v v^T (18 x 18): its blocks are R = sum w r r^T,
// C = sum w r s^T and Q = sum w s s^T. Stored as the upper triangle, entry-major within groups of
// 32 consecutive cells (one 128-byte row per entry and group, so the warp that evaluates a group
// reads one line per entry at a compile-time offset):
//   mom[((cell / 32) * 171 + e(i,j)) * 32 + cell % 32],  e(i,j) = i (35 - i) / 2 + j,
//   0 <= i <= j < 18   (171 entries).
// Since d = A_r s + r (to the rounding of r), S_c = sum w d d^T = A_r Q A_r^T + A_r C^T + C A_r^T + R, but every stored
// block is small where it has to be: R and C carry residuals, not the foreground signal.
//
// One warp per cell. Phase 1, lane = pixel: the cell's Gram-Schmidt basis of A_r (computed once per
// cell, the noise weight w_p scales out of s and r), then s by back-substitution and r = d - A_r s
// (ORDERED: FMAs in order of decreasing foreground, resid_fma; else in the Gram-Schmidt basis) of up
// to 32 pixels into shared memory. Phase 2: lanes = 15 upper 4x4 blocks of the 20x20 (zero-padded)
// v v^T x 2 pixel groups;
// partial sums are flushed every 16 pixels to bound FP32 rounding growth. Also sum w d^T n d.
constexpr int NM = 171;          // stored moment entries per cell
constexpr int VROW = 44;         // shared floats per pixel: v_Q[20], v_U[20], w (16-byte rows)
constexpr int BUILD_SMEM_PER_WARP = 32 * VROW + 64;  // pixel rows + the cell's basis and columns

// d - (s0 + a1 s1 + a2 s2) with FMAs: the larger of the two foreground products first, then the
// smaller, then s0. Each step rounds once, at the scale of what is left (s0, the smaller
// foreground and r after the first; s0 and r after the second; r after the last), so the error is
// about u (|s0| + min(|a1 s1|, |a2 s2|) + |r|) instead of the plain form's u |d|: the moments'
// decomposition d = A_r s + r then holds to rounding at the scale of the CMB and the fainter
// foreground, not of the brightest foreground, and so does the gradient formed from the moments
// at the reference point.
__device__ __forceinline__ float resid_fma(float d, float s0, float s1, float s2, float a1,
                                           float a2) {
  const bool dust_first = fabsf(a1 * s1) >= fabsf(a2 * s2);
  const float ab = dust_first ? a1 : a2, sb = dust_first ? s1 : s2;
  const float ac = dust_first ? a2 : a1, sc = dust_first ? s2 : s1;
  return fmaf(-ac, sc, fmaf(-ab, sb, d)) - s0;
}

__device__ __forceinline__ int mom_index(int i, int j) { return (i * (35 - i)) / 2 + j; }
// first entry of the group of 32 cells that holds `cell` (entry e of the cell: [e * 32 + cell % 32])
__device__ __forceinline__ long long mom_group(int cell) { return (long long)(cell >> 5) * NM * 32; }
// cells of the moment scratch, rounded up to whole groups
__host__ __device__ __forceinline__ long long mom_cells(long long ncell) { return (ncell + 31) & ~31LL; }

// Floats of the per-thread evaluation rows at the start of the dynamic shared memory (moment path:
// N A_1, N A_2, A_1, A_2, dA_1 and dA_2 per thread); the warp partials of the gradient follow them.
template <int NT, int PATH>
constexpr int fit_rows_floats() {
  return PATH == CSX_PATH_MOMENT ? 90 * NT : 0;
}

template <int NT, bool SEP, bool ORDERED>
__device__ double build_moments(const FitArgs& a, Ctx& c, float* smem, Shared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* sv = smem + warp * BUILD_SMEM_PER_WARP;  // 32 pixel rows
  float* sb = sv + 32 * VROW;  // the cell's basis c1[16], c2[16] and columns A_d[16], A_s[16]
  const int grp = lane / 15, blk = lane % 15;
  // upper-triangle 4x4 blocks of a 5x5 block grid: (ba, bb), ba <= bb
  int ba = 0, rem = blk;
  while (rem >= 5 - ba) {
    rem -= 5 - ba;
    ++ba;
  }
  const int bb = ba + rem;
  const float* nb = a.ninv_band;
  double dnd = 0.0;
  for (int cell = warp; cell < c.ncell; cell += NT / 32) {
    const int i0 = c.coff[cell], i1 = c.coff[cell + 1];
    const int px0 = c.perm[i0];
    const int kd = c.lab[px0], kt = c.lab[c.npix + px0], ks = c.lab[2 * c.npix + px0];
    // The cell's N-weighted Gram-Schmidt basis (the steps of mgs3), one band per lane; lanes
    // 16..31 carry zero weight. c1, c2 go to the warp's basis slot for the pixel phase.
    Mgs3 g;
    bool okb;
    {
      const int f = lane & 15;
      const float nf = (lane < 16) ? nb[f] : 0.f;
      const float adf = c.tabr[kd * NB + f] * c.tabr[(c.Kd + kt) * NB + f];
      const float asf = c.tabr[(c.Kd + 2 * c.KT + ks) * NB + f];
      const float n0 = warp_sum(nf), s1 = warp_sum(nf * adf), s2 = warp_sum(nf * asf);
      g.i0 = 1.f / n0;
      g.mu1 = s1 * g.i0;
      g.mu2 = s2 * g.i0;
      const float c1f = adf - g.mu1;
      const float n1 = warp_sum(nf * c1f * c1f), x12 = warp_sum(nf * c1f * asf);
      g.i1 = 1.f / n1;
      g.nu = x12 * g.i1;
      const float c2f = fmaf(-g.nu, c1f, asf - g.mu2);
      const float n2 = warp_sum(nf * c2f * c2f);
      g.i2 = 1.f / n2;
      okb = (n0 > 0.f) && (n1 > 0.f) && (n2 > 0.f);
      if (lane < 16) {
        sb[f] = c1f;
        sb[16 + f] = c2f;
        sb[32 + f] = adf;
        sb[48 + f] = asf;
      }
      __syncwarp();
    }
    float acc[16], tot[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = tot[k] = 0.f;
    int cnt = 0;
    for (int base = i0; base < i1; base += 32) {
      const int i = base + lane;
      float* row = sv + lane * VROW;
      if (i < i1) {
        const int px = c.perm[i];
        const float wp = SEP ? __ldg(a.w + px) : 1.f;
        float dq[NB], du[NB];
        load_pixel(c.d + (long long)px * 2 * NB, dq, du);
        float tq0 = 0.f, tq1 = 0.f, tq2 = 0.f, tu0 = 0.f, tu1 = 0.f, tu2 = 0.f, pd = 0.f;
#pragma unroll
        for (int f = 0; f < NB; ++f) {
          const float nq = nb[f] * dq[f], nu = nb[f] * du[f];
          const float c1 = sb[f], c2 = sb[16 + f];
          tq0 += nq;
          tq1 = fmaf(nq, c1, tq1);
          tq2 = fmaf(nq, c2, tq2);
          tu0 += nu;
          tu1 = fmaf(nu, c1, tu1);
          tu2 = fmaf(nu, c2, tu2);
          pd = fmaf(nq, dq[f], fmaf(nu, du[f], pd));
        }
        dnd += (double)(wp * pd);
        tq0 *= g.i0; tq1 *= g.i1; tq2 *= g.i2;
        tu0 *= g.i0; tu1 *= g.i1; tu2 *= g.i2;
        // s = R^-1 t (Gram-Schmidt back-substitution), then r = d - A_r s for this s
        const float sq1 = fmaf(-g.nu, tq2, tq1), su1 = fmaf(-g.nu, tu2, tu1);
        const float sq0 = tq0 - g.mu1 * sq1 - g.mu2 * tq2;
        const float su0 = tu0 - g.mu1 * su1 - g.mu2 * tu2;
#pragma unroll
        for (int f = 0; f < NB; ++f) {
          if (ORDERED) {
            const float a1 = sb[32 + f], a2 = sb[48 + f];
            row[f] = (f < 15) ? resid_fma(dq[f], sq0, sq1, tq2, a1, a2) : 0.f;
            row[20 + f] = (f < 15) ? resid_fma(du[f], su0, su1, tu2, a1, a2) : 0.f;
          } else {  // in the Gram-Schmidt basis, rounded at the data's scale
            const float c1 = sb[f], c2 = sb[16 + f];
            row[f] = (f < 15) ? dq[f] - fmaf(tq2, c2, fmaf(tq1, c1, tq0)) : 0.f;
            row[20 + f] = (f < 15) ? du[f] - fmaf(tu2, c2, fmaf(tu1, c1, tu0)) : 0.f;
          }
        }
        row[15] = sq0;
        row[16] = sq1;
        row[17] = tq2;
        row[18] = row[19] = 0.f;
        row[35] = su0;
        row[36] = su1;
        row[37] = tu2;
        row[38] = row[39] = 0.f;
        row[40] = okb ? wp : nan_f();
      } else {
#pragma unroll
        for (int k = 0; k < VROW; ++k) row[k] = 0.f;
      }
      __syncwarp();
      const int np = min(32, i1 - base);
      if (grp < 2) {
        for (int p = grp; p < np; p += 2) {
          const float* r = sv + p * VROW;
          const float wp = r[40];
          const float4 xq = *reinterpret_cast<const float4*>(r + 4 * ba);
          const float4 yq = *reinterpret_cast<const float4*>(r + 4 * bb);
          const float4 xu = *reinterpret_cast<const float4*>(r + 20 + 4 * ba);
          const float4 yu = *reinterpret_cast<const float4*>(r + 20 + 4 * bb);
          const float x[8] = {xq.x * wp, xq.y * wp, xq.z * wp, xq.w * wp,
                              xu.x * wp, xu.y * wp, xu.z * wp, xu.w * wp};
          const float y[8] = {yq.x, yq.y, yq.z, yq.w, yu.x, yu.y, yu.z, yu.w};
#pragma unroll
          for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
              acc[ii * 4 + jj] = fmaf(x[ii], y[jj], fmaf(x[4 + ii], y[4 + jj], acc[ii * 4 + jj]));
          if (++cnt == 16) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              tot[k] += acc[k];
              acc[k] = 0.f;
            }
            cnt = 0;
          }
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      tot[k] += acc[k];
      tot[k] += __shfl_down_sync(0xffffffffu, tot[k], 15);
    }
    if (lane < 15) {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int i = 4 * ba + ii, j = 4 * bb + jj;
          if (i <= j && j < 18) c.mom[mom_group(cell) + mom_index(i, j) * 32 + (cell & 31)] = tot[ii * 4 + jj];
        }
    }
    if (lane == 0) {
      c.trip[cell] = kd;
      c.trip[c.ncell + cell] = kt;
      c.trip[2 * c.ncell + cell] = ks;
    }
  }
  return block_sum<NT>(dnd, sh.red);
}

// -------------------------------------------------------------------- moment evaluation --------
// chi2 of every cell in the residual-moment form, and the adjoint gradient. With A = A(beta),
// A_r = A(beta_ref), M = A^T N A, the N-orthogonal projector P = I - A M^-1 A^T N, D = P A_r and
// Z = A_r^T N A:
//   chi2_c = tr(D^T N D Q) + 2 tr(D^T N C) + tr(N R) - tr(M^-1 A^T N R N A)
//   dL/dA  = -2 N [ D (Q Z + C^T N A) + P (C Z + R N A) ] M^-1       (Sec. 3.3.1, moment form)
// D vanishes at beta_ref, so the rounding of the foreground-sized terms shrinks with |beta-beta_ref|.
// Returns the sum of chi2_c; adds dL/dbeta into gacc (and the projected Gauss-Newton diagonal
// into hacc). Per-thread rows in shared memory (stride NT), formed in the first pass over the
// bands: N A_1, N A_2, A_1, A_2 and dA_1, dA_2 (90 floats).
// Each warp takes groups of 32 cells (NT / 32 groups apart) and asks L2 for its next group while
// it evaluates the current one (the first while the tables are formed): the moments of the CTAs'
// problems together exceed L2, so without it every entry would wait on DRAM.
template <int NT, bool WANT_H>
__device__ double eval_moment(const FitArgs& a, Ctx& c, Shared& sh) {
  constexpr unsigned GROUP_BYTES = NM * 32 * sizeof(float);
  if ((threadIdx.x & 31) == 0 && (threadIdx.x & ~31) < c.ncell)
    prefetch_l2(c.mom + mom_group(threadIdx.x & ~31), GROUP_BYTES);
  partials_zero<NT>(c, WANT_H);
  fill_tables<NT, true>(a, c, c.x, c.tab);  // ends with a barrier
  const float* nb = a.ninv_band;
  float nsum = 0.f;
#pragma unroll
  for (int f = 0; f < 15; ++f) nsum += nb[f];
  float* row = c.smem + threadIdx.x;  // row[k * NT]: N A_1 (k = 0..14), N A_2, A_1, A_2, dA_1, dA_2
  float acc = 0.f;  // per-thread sum over its few cells in FP32, FP64 across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* gwv = c.gw + (long long)warp * c.P;
  float* hwv = c.hw + (long long)warp * c.P;
  // warp-uniform trip count: lane l of a warp takes cell base + l (consecutive cells, so the
  // warp's run scan combines the cells of one patch)
  for (int base = threadIdx.x & ~31; base < c.ncell; base += NT) {
    const int cell = base + lane;
    if (lane == 0 && base + NT < c.ncell) prefetch_l2(c.mom + mom_group(base + NT), GROUP_BYTES);
    int kd = -1, kt = -1, ks = -1;
    float gbd = 0.f, gtd = 0.f, gbs = 0.f, h0 = 0.f, h1 = 0.f, h2 = 0.f;
    if (cell < c.ncell) do {
    kd = c.trip[cell];
    kt = c.trip[c.ncell + cell];
    ks = c.trip[2 * c.ncell + cell];
    const float* pd = c.tab + kd * NB;
    const float* bt = c.tab + (c.Kd + kt) * NB;
    const float* dt = c.tab + (c.Kd + c.KT + kt) * NB;
    const float* ss = c.tab + (c.Kd + 2 * c.KT + ks) * NB;
    const float* pdr = c.tabr + kd * NB;
    const float* btr = c.tabr + (c.Kd + kt) * NB;
    const float* ssr = c.tabr + (c.Kd + 2 * c.KT + ks) * NB;
    const float* ms = c.mom + mom_group(cell) + lane;
    // M = A^T N A, Z = A_r^T N A and G = A^T N dA with dA = A - A_r (its first column is 0)
    float m01 = 0.f, m02 = 0.f, m11 = 0.f, m12 = 0.f, m22 = 0.f;
    float z10 = 0.f, z11 = 0.f, z12 = 0.f, z20 = 0.f, z21 = 0.f, z22 = 0.f;
    float g01 = 0.f, g02 = 0.f, g11 = 0.f, g12 = 0.f, g21 = 0.f, g22 = 0.f;
#pragma unroll 3
    for (int f = 0; f < 15; ++f) {
      const float a1 = pd[f] * bt[f], a2 = ss[f];
      const float r1 = pdr[f] * btr[f], r2 = ssr[f];
      const float n = nb[f];
      const float t1 = n * a1, t2 = n * a2;
      row[f * NT] = t1;
      row[(15 + f) * NT] = t2;
      row[(30 + f) * NT] = a1;
      row[(45 + f) * NT] = a2;
      row[(60 + f) * NT] = a1 - r1;
      row[(75 + f) * NT] = a2 - r2;
      m01 += t1;
      m02 += t2;
      m11 = fmaf(t1, a1, m11);
      m12 = fmaf(t1, a2, m12);
      m22 = fmaf(t2, a2, m22);
      z10 = fmaf(r1, n, z10);
      z11 = fmaf(r1, t1, z11);
      z12 = fmaf(r1, t2, z12);
      z20 = fmaf(r2, n, z20);
      z21 = fmaf(r2, t1, z21);
      z22 = fmaf(r2, t2, z22);
      const float e1 = a1 - r1, e2 = a2 - r2;
      g01 = fmaf(n, e1, g01);
      g02 = fmaf(n, e2, g02);
      g11 = fmaf(t1, e1, g11);
      g12 = fmaf(t1, e2, g12);
      g21 = fmaf(t2, e1, g21);
      g22 = fmaf(t2, e2, g22);
    }
    Chol3 ch;
    if (!chol3(nsum, m01, m02, m11, m12, m22, ch)) {
      acc += nan_f();
      kd = kt = ks = -1;
      break;
    }
    float v[3][3];
    chol3_inverse(ch, v[0][0], v[0][1], v[0][2], v[1][1], v[1][2], v[2][2]);
    v[1][0] = v[0][1];
    v[2][0] = v[0][2];
    v[2][1] = v[1][2];
    const float Z[3][3] = {{nsum, m01, m02}, {z10, z11, z12}, {z20, z21, z22}};
    // D = P A_r = -P dA = A M^-1 A^T N dA - dA (P the N-orthogonal projector off the columns of A):
    // its first column vanishes (the constant column lies in span A) and D is formed from dA, so it
    // is exactly zero at the reference point and as accurate as dA near it (forming it as
    // A_r - A M^-1 A^T N A_r would leave the FP32 inverse's error, eps cond M, on the signal-sized
    // moments). Yd[k][j] = (M^-1 A^T N dA)[k][j + 1], j = 0, 1.
    float Yd[3][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Yd[k][0] = v[k][0] * g01 + v[k][1] * g11 + v[k][2] * g21;
      Yd[k][1] = v[k][0] * g02 + v[k][1] * g12 + v[k][2] * g22;
    }
    // pass 1 over bands: G1 = D^T N D, t2 = tr(D^T N C), CtA = C^T N A
    float G1[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float CtA[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float tdc = 0.f;
#pragma unroll 3
    for (int f = 0; f < 15; ++f) {
      const float a1 = row[(30 + f) * NT], a2 = row[(45 + f) * NT];
      const float e1 = row[(60 + f) * NT], e2 = row[(75 + f) * NT];
      const float na[3] = {nb[f], row[f * NT], row[(15 + f) * NT]};
      float D[3], C[3];
      D[0] = 0.f;
      D[1] = fmaf(a2, Yd[2][0], fmaf(a1, Yd[1][0], Yd[0][0])) - e1;
      D[2] = fmaf(a2, Yd[2][1], fmaf(a1, Yd[1][1], Yd[0][1])) - e2;
      row[(60 + f) * NT] = D[1];  // dA is not needed again: the gradient pass reads D back
      row[(75 + f) * NT] = D[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) C[k] = ms[mom_index(f, 15 + k) * 32];
#pragma unroll
      for (int k = 1; k < 3; ++k) {
        const float nd = nb[f] * D[k];
        tdc = fmaf(nd, C[k], tdc);
#pragma unroll
        for (int l = 1; l < 3; ++l) G1[k][l] = fmaf(nd, D[l], G1[k][l]);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) CtA[k][l] = fmaf(C[k], na[l], CtA[k][l]);
    }
    // B = R N A: every stored entry of R's upper triangle is read once and serves (i, j) and
    // (j, i); N A_1, N A_2 held in registers. Then A^T N R N A, tr(N R), and the gradient part
    // carried by B: with E = U + C Z + B - A Psi, the B term of E M^-1 in band i is
    // sum_l B[i][l] M^-1[l][k]
    float x1[15], x2[15], B[15][3];
#pragma unroll
    for (int j = 0; j < 15; ++j) {
      x1[j] = row[j * NT];
      x2[j] = row[(15 + j) * NT];
      B[j][0] = B[j][1] = B[j][2] = 0.f;
    }
    float trNR = 0.f;
#pragma unroll
    for (int i = 0; i < 15; ++i) {
#pragma unroll
      for (int j = i; j < 15; ++j) {
        const float r = ms[mom_index(i, j) * 32];
        B[i][0] = fmaf(r, nb[j], B[i][0]);
        B[i][1] = fmaf(r, x1[j], B[i][1]);
        B[i][2] = fmaf(r, x2[j], B[i][2]);
        if (j == i) {
          trNR = fmaf(nb[i], r, trNR);
        } else {
          B[j][0] = fmaf(r, nb[i], B[j][0]);
          B[j][1] = fmaf(r, x1[i], B[j][1]);
          B[j][2] = fmaf(r, x2[i], B[j][2]);
        }
      }
    }
    float AtRA[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int i = 0; i < 15; ++i) {
      const float na[3] = {nb[i], x1[i], x2[i]};
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) AtRA[k][l] = fmaf(na[k], B[i][l], AtRA[k][l]);
      const float fb1 = B[i][0] * v[0][1] + B[i][1] * v[1][1] + B[i][2] * v[2][1];
      const float fb2 = B[i][0] * v[0][2] + B[i][1] * v[1][2] + B[i][2] * v[2][2];
      const float t1 = fb1 * na[1];
      gbd = fmaf(t1, a.bands.lnd[i], gbd);
      gtd = fmaf(t1, dt[i], gtd);
      gbs = fmaf(fb2 * na[2], a.bands.lns[i], gbs);
    }
    float Q[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) Q[k][l] = Q[l][k] = ms[mom_index(15 + k, 15 + l) * 32];
    float chi = 2.f * tdc + trNR;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l) chi += G1[k][l] * Q[l][k] - v[k][l] * AtRA[l][k];
    acc += chi;
    // W1 = Q Z + C^T N A ;  Psi = M^-1 A^T N (C Z + R N A) = M^-1 (CtA^T Z + AtRA)
    float W1[3][3], Psi[3][3];
    {
      float H[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          W1[k][l] = Q[k][0] * Z[0][l] + Q[k][1] * Z[1][l] + Q[k][2] * Z[2][l] + CtA[k][l];
          H[k][l] = CtA[0][k] * Z[0][l] + CtA[1][k] * Z[1][l] + CtA[2][k] * Z[2][l] + AtRA[k][l];
        }
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int l = 0; l < 3; ++l) Psi[m][l] = v[m][0] * H[0][l] + v[m][1] * H[1][l] + v[m][2] * H[2][l];
    }
#pragma unroll 3
    for (int f = 0; f < 15; ++f) {
      const float a1 = row[(30 + f) * NT], a2 = row[(45 + f) * NT];
      float D[3], C[3];
      D[0] = 0.f;
      D[1] = row[(60 + f) * NT];
      D[2] = row[(75 + f) * NT];
#pragma unroll
      for (int k = 0; k < 3; ++k) C[k] = ms[mom_index(f, 15 + k) * 32];
      float E[3];
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const float U = D[0] * W1[0][l] + D[1] * W1[1][l] + D[2] * W1[2][l];
        const float X = C[0] * Z[0][l] + C[1] * Z[1][l] + C[2] * Z[2][l];  // + B: added above
        E[l] = U + X - fmaf(a2, Psi[2][l], fmaf(a1, Psi[1][l], Psi[0][l]));
      }
      const float F1 = E[0] * v[0][1] + E[1] * v[1][1] + E[2] * v[2][1];
      const float F2 = E[0] * v[0][2] + E[1] * v[1][2] + E[2] * v[2][2];
      const float t1 = F1 * row[f * NT];
      gbd = fmaf(t1, a.bands.lnd[f], gbd);
      gtd = fmaf(t1, dt[f], gtd);
      gbs = fmaf(F2 * row[(15 + f) * NT], a.bands.lns[f], gbs);
    }
    gbd *= -2.f;
    gtd *= -2.f;
    gbs *= -2.f;
    if (WANT_H) {
      // Gauss-Newton diagonal 2 (sum w s_k^2) da^T N da (the scaling of the optimiser's variables;
      // the same quantity as the streaming path's), with sum w s s^T at the reference point (Q)
      float n2[3] = {0.f, 0.f, 0.f};
#pragma unroll 3
      for (int f = 0; f < 15; ++f) {
        const float a1 = row[(30 + f) * NT], a2 = row[(45 + f) * NT];
        const float da[3] = {a1 * a.bands.lnd[f], a1 * dt[f], a2 * a.bands.lns[f]};
#pragma unroll
        for (int k = 0; k < 3; ++k) n2[k] = fmaf(nb[f] * da[k], da[k], n2[k]);
      }
      h0 = 2.f * Q[1][1] * n2[0];
      h1 = 2.f * Q[1][1] * n2[1];
      h2 = 2.f * Q[2][2] * n2[2];
    }
    } while (0);
    const int j1 = kt < 0 ? -1 : c.Kd + kt, j2 = ks < 0 ? -1 : c.Kd + c.KT + ks;
    warp_run_accum3(gwv, kd, gbd, j1, gtd, j2, gbs, sh.stage[warp]);
    if (WANT_H) warp_run_accum3(hwv, kd, h0, j1, h1, j2, h2, sh.stage[warp]);
  }
  // the optimiser's vectors and L-BFGS history (the slot's head, read next) were likely pushed
  // out of L2 by the moments: ask for them back
  if (threadIdx.x < 32) {
    const unsigned long long bytes = (unsigned long long)(9 + 2 * a.history) * a.Pmax * sizeof(float);
    for (unsigned long long off = (unsigned long long)threadIdx.x * 8192; off < bytes; off += 32 * 8192)
      prefetch_l2(reinterpret_cast<const char*>(c.z) + off, (unsigned)min(8192ull, bytes - off));
  }
  partials_reduce<NT>(c, WANT_H);
  return block_sum<NT>((double)acc, sh.red);
}

// -------------------------------------------------------------------- stream evaluation --------
// Returns chi2 (sum of residual norms) and, through dnd, sum d^T N d.
template <int NT, int NOISE, bool GRAD, bool WANT_H>
__device__ double eval_stream(const FitArgs& a, Ctx& c, Shared& sh, double& dnd_out) {
  if (GRAD || WANT_H) partials_zero<NT>(c, WANT_H);
  fill_tables<NT>(a, c, c.x, c.tab);
  float nb[NB];
#pragma unroll
  for (int f = 0; f < NB; ++f) nb[f] = a.ninv_band[f];
  double chi = 0.0, dn = 0.0;
  const int* ld = c.lab;
  const int* lt = c.lab + c.npix;
  const int* ls = c.lab + 2 * c.npix;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* gwv = c.gw + (long long)warp * c.P;
  float* hwv = c.hw + (long long)warp * c.P;
  // warp-uniform trip count: every lane reaches the warp-wide gradient scatter
  for (int base = threadIdx.x & ~31; base < c.npix; base += NT) {
    const int p = base + lane;
    int kd = -1, kt = -1, ks = -1;
    PixOut o;
    o.gbd = o.gtd = o.gbs = o.hbd = o.htd = o.hbs = 0.f;
    if (p < c.npix) {
      kd = ld[p];
      kt = lt[p];
      ks = ls[p];
      if ((unsigned)kd >= (unsigned)c.Kd || (unsigned)kt >= (unsigned)c.KT ||
          (unsigned)ks >= (unsigned)c.Ks) {
        chi += (double)nan_f();
        kd = kt = ks = -1;
      } else {
        float dq[NB], du[NB], nn[NB];
        load_pixel(c.d + (long long)p * 2 * NB, dq, du);
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
        if (pixel_eval<GRAD, WANT_H>(dq, du, nn, c.tab + kd * NB, c.tab + (c.Kd + kt) * NB,
                                     c.tab + (c.Kd + c.KT + kt) * NB,
                                     c.tab + (c.Kd + 2 * c.KT + ks) * NB, a.bands, o)) {
          chi += (double)o.chi2;
          dn += (double)o.dnd;
        } else {
          chi += (double)nan_f();
          o.gbd = o.gtd = o.gbs = o.hbd = o.htd = o.hbs = 0.f;
        }
      }
    }
    const int j1 = kt < 0 ? -1 : c.Kd + kt, j2 = ks < 0 ? -1 : c.Kd + c.KT + ks;
    if (GRAD) warp_run_accum3(gwv, kd, o.gbd, j1, o.gtd, j2, o.gbs, sh.stage[warp]);
    if (WANT_H) warp_run_accum3(hwv, kd, o.hbd, j1, o.htd, j2, o.hbs, sh.stage[warp]);
  }
  if (GRAD || WANT_H) partials_reduce<NT>(c, WANT_H);
  block_sum2<NT>(chi, dn, sh.red);
  dnd_out = dn;
  return chi;
}

// -------------------------------------------------------------------- objective ---------------
// f(x) at the physical parameters in c.x; gradient (physical units) in c.gacc.
template <int NT, int PATH, int GMODE, int NOISE, bool WANT_H>
__device__ double objective(const FitArgs& a, Ctx& c, Shared& sh, double& dnd) {
  if (PATH == CSX_PATH_MOMENT) {
    return eval_moment<NT, WANT_H>(a, c, sh);  // chi2; dnd comes from the moment build
  } else {
    return eval_stream<NT, NOISE, GMODE == CSX_GRAD_ADJOINT, WANT_H>(a, c, sh, dnd);
  }
}

// z -> g (scaled units) by central differences of the forward objective (plain form).
template <int NT, int NOISE>
__device__ void fd_gradient(const FitArgs& a, Ctx& c, Shared& sh, const float* z, float* g) {
  const float h = a.fd_step;
  for (int i = threadIdx.x; i < c.P; i += NT) c.x[i] = z[i] / c.hs[i];
  __syncthreads();
  for (int i = 0; i < c.P; ++i) {
    double dn;
    if (threadIdx.x == 0) c.x[i] = (z[i] + h) / c.hs[i];
    __syncthreads();
    const double fp = eval_stream<NT, NOISE, false, false>(a, c, sh, dn);
    if (threadIdx.x == 0) c.x[i] = (z[i] - h) / c.hs[i];
    __syncthreads();
    const double fm = eval_stream<NT, NOISE, false, false>(a, c, sh, dn);
    if (threadIdx.x == 0) {
      g[i] = (float)((fp - fm) / (2.0 * h));
      c.x[i] = z[i] / c.hs[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------ the fit --------------
// Moment path: make the current point c.x the reference point and rebuild the cell moments. The
// first build of a fit (at the start point, far from the optimum) forms the residuals in the
// Gram-Schmidt basis; every later one (a move of the reference point near convergence) forms them
// with the ordered FMAs of resid_fma, which the precision of the last iterations' gradients rests on.
template <int NT, int NOISE>
__device__ double recentre(const FitArgs& a, Ctx& c, Shared& sh, float* smem, bool ordered = true) {
  for (int i = threadIdx.x; i < c.P; i += NT) c.xr[i] = c.x[i];
  __syncthreads();
  fill_tables<NT, true>(a, c, c.xr, c.tabr);
  constexpr bool SEP = NOISE == CSX_NOISE_SEPARABLE;
  return ordered ? build_moments<NT, SEP, true>(a, c, smem, sh)
               : build_moments<NT, SEP, false>(a, c, smem, sh);
}

// The two-loop recursion of L-BFGS with this thread's elements of p in registers (P <= TL_E NT)
// and the next pair of history vectors loaded while the current dot product is being reduced:
// the operations and their order are those of the loops over the slot vectors in fit_problem
// (elements beyond P are zeros and add exact zeros), so the direction has the same bits.
constexpr int TL_E = 12;
template <int NT>
__device__ __forceinline__ void two_loop_reg(const FitArgs& a, Ctx& c, Shared& sh, int P, int m,
                                             int head, int count, float gamma) {
  const int tid = threadIdx.x;
  const long long Pm = a.Pmax;
  float pr[TL_E], u[TL_E], v[TL_E];  // p; the next dot-product and update operands
#pragma unroll
  for (int e = 0; e < TL_E; ++e) {
    const int i = tid + e * NT;
    pr[e] = i < P ? c.p[i] : 0.f;
  }
  auto load = [&](const float* dv, const float* av) {
#pragma unroll
    for (int e = 0; e < TL_E; ++e) {
      const int i = tid + e * NT;
      u[e] = i < P ? dv[i] : 0.f;
      v[e] = i < P ? av[i] : 0.f;
    }
  };
  if (count > 0) {
    const int k = (head - 1 + m) % m;
    load(c.S + k * Pm, c.Y + k * Pm);
  }
  for (int j = 0; j < count; ++j) {
    const int k = (head - 1 - j + m) % m;
    float sv[TL_E], yv[TL_E];
#pragma unroll
    for (int e = 0; e < TL_E; ++e) {
      sv[e] = u[e];
      yv[e] = v[e];
    }
    if (j + 1 < count) {
      const int kn = (head - 2 - j + m) % m;
      load(c.S + kn * Pm, c.Y + kn * Pm);
    }
    float dotf = 0.f;
#pragma unroll
    for (int e = 0; e < TL_E; ++e) dotf = fmaf(sv[e], pr[e], dotf);
    const double dot = block_sum_f<NT>(dotf, sh.red);
    const double al = sh.rho[k] * dot;
    if (tid == 0) sh.alpha[k] = al;
#pragma unroll
    for (int e = 0; e < TL_E; ++e) pr[e] -= (float)al * yv[e];
  }
#pragma unroll
  for (int e = 0; e < TL_E; ++e) pr[e] *= gamma;
  if (count > 0) {
    const int k = (head - count + m) % m;  // j = count - 1
    load(c.Y + k * Pm, c.S + k * Pm);
  }
  for (int j = count - 1; j >= 0; --j) {
    const int k = (head - 1 - j + m) % m;
    float yv[TL_E], sv[TL_E];
#pragma unroll
    for (int e = 0; e < TL_E; ++e) {
      yv[e] = u[e];
      sv[e] = v[e];
    }
    if (j > 0) {
      const int kn = (head - j + m) % m;  // j - 1
      load(c.Y + kn * Pm, c.S + kn * Pm);
    }
    float dotf = 0.f;
#pragma unroll
    for (int e = 0; e < TL_E; ++e) dotf = fmaf(yv[e], pr[e], dotf);
    const double dot = block_sum_f<NT>(dotf, sh.red);
    const double be = sh.rho[k] * dot;
    const float coef = (float)(sh.alpha[k] - be);
#pragma unroll
    for (int e = 0; e < TL_E; ++e) pr[e] += coef * sv[e];
  }
#pragma unroll
  for (int e = 0; e < TL_E; ++e) {
    const int i = tid + e * NT;
    if (i < P) c.p[i] = pr[e];
  }
}

template <int NT, int PATH, int GMODE, int NOISE>
__device__ void fit_problem(const FitArgs& a, Ctx& c, Shared& sh, float* smem, int q,
                            long long poff) {
  const int P = c.P;
  const int tid = threadIdx.x;
  const int m = a.history;
  // start point, clamped into the box
  for (int i = tid; i < P; i += NT) {
    const int t = ptype(c, i);
    c.x[i] = fminf(fmaxf(a.beta0[poff + i], a.lower[t]), a.upper[t]);
  }
  __syncthreads();
  double dnd = 0.0;
  int recentres = 0;
  if (PATH == CSX_PATH_MOMENT) dnd = recentre<NT, NOISE>(a, c, sh, smem, false);
  double f = objective<NT, PATH, GMODE, NOISE, true>(a, c, sh, dnd);
  int nev = 1;  // likelihood evaluations (each forward pass of a finite difference counts once)
  int status = CSX_FIT_MAXITER, it = 0;
  if (!isfinite(f)) {
    for (int i = tid; i < P; i += NT) a.beta_out[poff + i] = c.x[i];
    if (tid == 0) {
      a.L_out[q] = (double)nan_f();
      a.status[q] = CSX_FIT_NONPHYSICAL;
      a.iters[q] = 0;
      if (a.nevals) a.nevals[q] = nev;
    }
    __syncthreads();
    return;
  }
  // scaling by sqrt of the Gauss-Newton diagonal
  float hm = 0.f;
  for (int i = tid; i < P; i += NT) hm = fmaxf(hm, isfinite(c.hacc[i]) ? c.hacc[i] : 0.f);
  hm = block_max<NT>(hm, reinterpret_cast<float*>(sh.red));
  const float hfloor = fmaxf(1e-12f * hm, 1e-30f);
  for (int i = tid; i < P; i += NT) {
    const float h = c.hacc[i];
    c.hs[i] = sqrtf((isfinite(h) && h > hfloor) ? h : hfloor);
    c.z[i] = c.hs[i] * c.x[i];
    if (GMODE == CSX_GRAD_ADJOINT) c.g[i] = c.gacc[i] / c.hs[i];
  }
  __syncthreads();
  if (GMODE == CSX_GRAD_FD) {
    fd_gradient<NT, NOISE>(a, c, sh, c.z, c.g);
    nev += 2 * P;
  }

  int count = 0, head = 0;
  double gamma = 1.0;
  float last_step = 1e30f;
  const double delta = 0.1, sigma = 0.9;
  for (it = 0; it < a.max_iter; ++it) {
    // ---- direction: two-loop recursion on the free-set gradient --------------------------
    for (int i = tid; i < P; i += NT) {
      const int t = ptype(c, i);
      const float zl = c.hs[i] * a.lower[t], zu = c.hs[i] * a.upper[t];
      const float gi = c.g[i];
      const bool act = (c.z[i] <= zl && gi > 0.f) || (c.z[i] >= zu && gi < 0.f);
      c.p[i] = act ? 0.f : gi;
    }
    if (P <= TL_E * NT) {
      two_loop_reg<NT>(a, c, sh, P, m, head, count, (float)gamma);
    } else {
      for (int j = 0; j < count; ++j) {
        const int k = (head - 1 - j + m) % m;
        const float* Sk = c.S + (long long)k * a.Pmax;
        float dotf = 0.f;  // per-thread partial in FP32 (a few terms), FP64 across the block
        for (int i = tid; i < P; i += NT) dotf = fmaf(Sk[i], c.p[i], dotf);
        const double dot = block_sum_f<NT>(dotf, sh.red);
        const double al = sh.rho[k] * dot;
        if (tid == 0) sh.alpha[k] = al;
        const float* Yk = c.Y + (long long)k * a.Pmax;
        for (int i = tid; i < P; i += NT) c.p[i] -= (float)al * Yk[i];
      }
      for (int i = tid; i < P; i += NT) c.p[i] *= (float)gamma;
      for (int j = count - 1; j >= 0; --j) {
        const int k = (head - 1 - j + m) % m;
        const float* Yk = c.Y + (long long)k * a.Pmax;
        float dotf = 0.f;
        for (int i = tid; i < P; i += NT) dotf = fmaf(Yk[i], c.p[i], dotf);
        const double dot = block_sum_f<NT>(dotf, sh.red);
        const double be = sh.rho[k] * dot;
        const float* Sk = c.S + (long long)k * a.Pmax;
        const float coef = (float)(sh.alpha[k] - be);
        for (int i = tid; i < P; i += NT) c.p[i] += coef * Sk[i];
      }
    }
    // negate, mask the active set and outward steps at a bound, directional derivative, QN step
    float gpf = 0.f;
    float stepn = 0.f;
    for (int i = tid; i < P; i += NT) {
      const int t = ptype(c, i);
      const float zl = c.hs[i] * a.lower[t], zu = c.hs[i] * a.upper[t];
      const float gi = c.g[i];
      const bool act = (c.z[i] <= zl && gi > 0.f) || (c.z[i] >= zu && gi < 0.f);
      float pi = act ? 0.f : -c.p[i];
      if ((c.z[i] <= zl && pi < 0.f) || (c.z[i] >= zu && pi > 0.f)) pi = 0.f;
      c.p[i] = pi;
      gpf = fmaf(gi, pi, gpf);
      stepn = fmaxf(stepn, fabsf(pi) / c.hs[i] / a.xtol[t]);
    }
    double gp = block_sum_f<NT>(gpf, sh.red);
    stepn = block_max<NT>(stepn, reinterpret_cast<float*>(sh.red));
    if (!(gp < 0.0)) {
      // not a descent direction: restart from the projected steepest descent
      count = 0;
      gamma = 1.0;
      gpf = 0.f;
      stepn = 0.f;
      for (int i = tid; i < P; i += NT) {
        const int t = ptype(c, i);
        const float zl = c.hs[i] * a.lower[t], zu = c.hs[i] * a.upper[t];
        const float gi = c.g[i];
        const bool act = (c.z[i] <= zl && gi > 0.f) || (c.z[i] >= zu && gi < 0.f);
        float pi = act ? 0.f : -gi;
        if ((c.z[i] <= zl && pi < 0.f) || (c.z[i] >= zu && pi > 0.f)) pi = 0.f;
        c.p[i] = pi;
        gpf = fmaf(gi, pi, gpf);
        stepn = fmaxf(stepn, fabsf(pi) / c.hs[i] / a.xtol[t]);
      }
      gp = block_sum_f<NT>(gpf, sh.red);
      stepn = block_max<NT>(stepn, reinterpret_cast<float*>(sh.red));
      if (!(gp < 0.0)) {
        status = CSX_FIT_CONVERGED;  // projected gradient vanishes
        break;
      }
    }
    const bool near_opt = CSX_FIT_NEAR > 0.f && recentres == 0 && stepn <= CSX_FIT_NEAR &&
                          last_step <= CSX_FIT_NEAR;
    const bool at_opt = recentres < 6 && stepn <= 1.f && last_step <= 1.f;
    if (PATH == CSX_PATH_MOMENT && it > 0 && (near_opt || at_opt)) {
      {
        // The moment form rounds in proportion to the distance from the reference point: at
        // convergence (and, with CSX_FIT_NEAR > 0, also once the steps first fall within that many
        // tolerances), move the reference here unless it is already close, so that the last
        // iterations run on precise values. Each move costs one pass over the pixels.
        float dref = 0.f;
        for (int i = tid; i < P; i += NT)
          dref = fmaxf(dref, fabsf(c.z[i] / c.hs[i] - c.xr[i]) / a.xtol[ptype(c, i)]);
        dref = block_max<NT>(dref, reinterpret_cast<float*>(sh.red));
        if (dref > 30.f) {
          for (int i = tid; i < P; i += NT) c.x[i] = c.z[i] / c.hs[i];
          __syncthreads();
          dnd = recentre<NT, NOISE>(a, c, sh, smem);
          f = objective<NT, PATH, GMODE, NOISE, false>(a, c, sh, dnd);
          ++nev;
          for (int i = tid; i < P; i += NT) c.g[i] = c.gacc[i] / c.hs[i];
          ++recentres;
          --it;  // a move of the reference point is not a quasi-Newton iteration
          __syncthreads();
          continue;
        }
      }
    }
    if (it > 0 && stepn <= 1.f && last_step <= 1.f) {
      status = CSX_FIT_CONVERGED;
      break;
    }
    // ---- largest step inside the box --------------------------------------------------
    float amax = 1e30f;
    for (int i = tid; i < P; i += NT) {
      const int t = ptype(c, i);
      const float pi = c.p[i];
      if (pi < 0.f) amax = fminf(amax, (c.hs[i] * a.lower[t] - c.z[i]) / pi);
      else if (pi > 0.f) amax = fminf(amax, (c.hs[i] * a.upper[t] - c.z[i]) / pi);
    }
    amax = fmaxf(block_min<NT>(amax, reinterpret_cast<float*>(sh.red)), 0.f);
    // ---- line search (approximate Wolfe) ------------------------------------------------
    const double eps_f = 1e-6 * fabs(f);
    double alpha = fmin(1.0, (double)amax);
    double a_lo = 0.0, d_lo = gp, a_hi = -1.0, d_hi = 0.0;
    double ft = 0.0, dnd_t = 0.0;
    bool ok = false;
    for (int ls = 0; ls < a.max_ls && alpha > 0.0; ++ls) {
      for (int i = tid; i < P; i += NT) {
        const int t = ptype(c, i);
        const float zl = c.hs[i] * a.lower[t], zu = c.hs[i] * a.upper[t];
        const float zi = fminf(fmaxf(c.z[i] + (float)alpha * c.p[i], zl), zu);
        c.zt[i] = zi;
        c.x[i] = zi / c.hs[i];
      }
      __syncthreads();
      ft = objective<NT, PATH, GMODE, NOISE, false>(a, c, sh, dnd_t);
      ++nev;
      if (GMODE == CSX_GRAD_FD) {
        fd_gradient<NT, NOISE>(a, c, sh, c.zt, c.gt);
        nev += 2 * P;
      } else {
        for (int i = tid; i < P; i += NT) c.gt[i] = c.gacc[i] / c.hs[i];
      }
      float dphif = 0.f;
      for (int i = tid; i < P; i += NT) dphif = fmaf(c.gt[i], c.p[i], dphif);
      const double dphi = block_sum_f<NT>(dphif, sh.red);
      if (!isfinite(ft) || !isfinite(dphi)) {
        a_hi = alpha;
        d_hi = 1.0;
        alpha = a_lo + 0.25 * (alpha - a_lo);
        continue;
      }
      const bool wolfe = (ft <= f + delta * alpha * gp) && (dphi >= sigma * gp);
      const bool approx = (ft <= f + eps_f) && (dphi <= (2.0 * delta - 1.0) * gp) && (dphi >= sigma * gp);
      const bool at_bound = (alpha >= (double)amax * (1.0 - 1e-7)) && (dphi < 0.0) && (ft <= f + eps_f);
      if (wolfe || approx || at_bound) {
        ok = true;
        break;
      }
      if (dphi >= 0.0 || ft > f + eps_f) {
        a_hi = alpha;
        d_hi = dphi;
      } else {
        a_lo = alpha;
        d_lo = dphi;
      }
      if (a_hi < 0.0) {
        if (alpha >= (double)amax) break;
        alpha = fmin(4.0 * alpha, (double)amax);
      } else {
        double an = (d_hi > 0.0) ? a_lo - d_lo * (a_hi - a_lo) / (d_hi - d_lo) : 0.5 * (a_lo + a_hi);
        const double w = a_hi - a_lo;
        an = fmin(fmax(an, a_lo + 0.1 * w), a_hi - 0.1 * w);
        if (w <= 1e-12 * fmax(1.0, a_hi)) break;
        alpha = an;
      }
    }
    if (!ok) {
      if (PATH == CSX_PATH_MOMENT && recentres < 6) {
        // Far from the reference point the moment form's rounding can hide the decrease the
        // line search looks for: move the reference here and try again.
        float dref = 0.f;
        for (int i = tid; i < P; i += NT)
          dref = fmaxf(dref, fabsf(c.z[i] / c.hs[i] - c.xr[i]) / a.xtol[ptype(c, i)]);
        dref = block_max<NT>(dref, reinterpret_cast<float*>(sh.red));
        if (dref > 1.f) {
          for (int i = tid; i < P; i += NT) c.x[i] = c.z[i] / c.hs[i];
          __syncthreads();
          dnd = recentre<NT, NOISE>(a, c, sh, smem);
          f = objective<NT, PATH, GMODE, NOISE, false>(a, c, sh, dnd);
          ++nev;
          for (int i = tid; i < P; i += NT) c.g[i] = c.gacc[i] / c.hs[i];
          ++recentres;
          --it;
          __syncthreads();
          continue;
        }
      }
      if (count > 0) {  // drop the curvature history and retry from steepest descent
        count = 0;
        gamma = 1.0;
        continue;
      }
      status = CSX_FIT_LINESEARCH;
      break;
    }
    // ---- accept: curvature pair and update --------------------------------------------
    float syf = 0.f, yyf = 0.f;
    float sn = 0.f;
    float* Sn = c.S + (long long)head * a.Pmax;
    float* Yn = c.Y + (long long)head * a.Pmax;
    for (int i = tid; i < P; i += NT) {
      const int t = ptype(c, i);
      const float si = c.zt[i] - c.z[i], yi = c.gt[i] - c.g[i];
      Sn[i] = si;
      Yn[i] = yi;
      syf = fmaf(si, yi, syf);
      yyf = fmaf(yi, yi, yyf);
      sn = fmaxf(sn, fabsf(si) / c.hs[i] / a.xtol[t]);
      c.z[i] = c.zt[i];
      c.g[i] = c.gt[i];
    }
    double sy, yy;
    block_sum2_f<NT>(syf, yyf, sh.red, sy, yy);
    sn = block_max<NT>(sn, reinterpret_cast<float*>(sh.red));
    last_step = sn;
    f = ft;
    if (PATH != CSX_PATH_MOMENT) dnd = dnd_t;
    if (sy > 1e-12 * yy && yy > 0.0) {
      if (tid == 0) sh.rho[head] = 1.0 / sy;
      head = (head + 1) % m;
      count = min(count + 1, m);
      gamma = sy / yy;
    }
    __syncthreads();
  }
  for (int i = tid; i < P; i += NT) a.beta_out[poff + i] = c.z[i] / c.hs[i];
  if (tid == 0) {
    a.L_out[q] = f - dnd;  // L = chi2_min - sum d^T N d
    a.status[q] = status;
    a.iters[q] = it;
    if (a.nevals) a.nevals[q] = nev;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------- AdaTopK --------------
// App. A: internal space y = (x - l) / (u - l); pivots p in {-1, 0, 1} (lower bound, free, upper
// bound); per iteration: release the bound constraints whose score p_i g_i is positive (Top-K:
// max(1, floor(topk n)) of the n candidates, highest first, ties to the lowest index; the printed
// score has the opposite sign of its stated intent, the alignment of -g with the way into the box,
// which is followed here), project the gradient onto the free set, rescale the objective and the
// AdaBelief moments by 1 / |g_proj| when |g_proj| leaves [1e-15, 1e15], AdaBelief direction
// (beta1 0.9, beta2 0.999, eps 1e-16, bias-corrected) masked to the free set, step limit at the
// nearest bound, backtracking line search from min(eta, alpha_max) (Armijo 1e-4; accepted also when
// the value change is below 1e-5 |f| and the slope at the trial point is still downhill, as the FP32
// likelihood -- residual moments included -- cannot resolve smaller changes), clamp and pin the limiting parameter when the step
// reaches the bound. A non-descent direction or a failed search resets the AdaBelief state and
// retries with the normalised projected steepest descent. The direction is zeroed where a free
// parameter sits on a bound and points out of the box. Stop: no positive release score, the last
// two steps of every parameter below 0.003 xtol, and every free parameter's Newton-step estimate
// |dL/dx_i| / H_ii below xtol_i (H: the Gauss-Newton diagonal, evaluated at the candidate point);
// a candidate that fails the last test restarts the AdaBelief moments. eta: 0.1 at the start, min(1, 2 alpha) after
// an accepted step of nonzero length. Moment path: the reference point moves to the current point when the fit is
// 1000 xtol away from it or converging more than 0.09 xtol away (at most 24 times). Slot vectors: z = y, g = scaled internal gradient, p = direction, zt/gt = trial,
// hs = pivots, first rows of S/Y = AdaBelief m/s.
constexpr float ADA_B1 = 0.9f, ADA_B2 = 0.999f, ADA_EPS = 1e-16f;
constexpr float ADA_STEP_FACTOR = 0.003f;
constexpr int ADA_MAX_RECENTRES = 24;
constexpr double ADA_EPS_REL = 1e-5;  // value changes below this fraction of |f| are unresolved

template <int NT, int PATH, int NOISE>
__device__ void fit_problem_adatopk(const FitArgs& a, Ctx& c, Shared& sh, float* smem, int q,
                                    long long poff) {
  const int P = c.P;
  const int tid = threadIdx.x;
  float* y = c.z;
  float* g = c.g;
  float* dv = c.p;
  float* yt = c.zt;
  float* gt = c.gt;
  float* piv = c.hs;
  float* mm = c.S;
  float* ssq = c.Y;
  auto rng = [&](int i) { const int t = ptype(c, i); return a.upper[t] - a.lower[t]; };
  auto low = [&](int i) { return a.lower[ptype(c, i)]; };
  auto thr = [&](int i) { return ADA_STEP_FACTOR * a.xtol[ptype(c, i)] / rng(i); };
  for (int i = tid; i < P; i += NT) {
    const int t = ptype(c, i);
    const float x0 = fminf(fmaxf(a.beta0[poff + i], a.lower[t]), a.upper[t]);
    const float yi = fminf(fmaxf((x0 - a.lower[t]) / (a.upper[t] - a.lower[t]), 0.f), 1.f);
    y[i] = yi;
    piv[i] = yi <= 0.f ? -1.f : (yi >= 1.f ? 1.f : 0.f);
    mm[i] = 0.f;
    ssq[i] = 0.f;
    c.x[i] = x0;
  }
  __syncthreads();
  double dnd = 0.0;
  int recentres = 0;
  if (PATH == CSX_PATH_MOMENT) dnd = recentre<NT, NOISE>(a, c, sh, smem, false);
  double f = objective<NT, PATH, CSX_GRAD_ADJOINT, NOISE, false>(a, c, sh, dnd);
  int nev = 1, status = CSX_FIT_MAXITER, it = 0;
  if (!isfinite(f)) {
    for (int i = tid; i < P; i += NT) a.beta_out[poff + i] = c.x[i];
    if (tid == 0) {
      a.L_out[q] = (double)nan_f();
      a.status[q] = CSX_FIT_NONPHYSICAL;
      a.iters[q] = 0;
      if (a.nevals) a.nevals[q] = nev;
    }
    __syncthreads();
    return;
  }
  double scale = 1.0;
  for (int i = tid; i < P; i += NT) g[i] = c.gacc[i] * rng(i);
  __syncthreads();
  float eta = 0.1f;
  int tb = 0, small = 0;
  float b1t = 1.f, b2t = 1.f;  // beta1^t, beta2^t
  for (it = 0; it < a.max_iter; ++it) {
    // ---- release (Top-K) ----------------------------------------------------------------
    int ncand = 0;
    for (int i = tid; i < P; i += NT) ncand += (piv[i] != 0.f && piv[i] * g[i] > 0.f) ? 1 : 0;
    ncand = block_sum<NT>(ncand, reinterpret_cast<int*>(sh.red));
    const int nrel = ncand > 0 ? max(1, (int)floorf(a.topk * (float)ncand)) : 0;
    for (int r = 0; r < nrel; ++r) {
      float bv = -INFINITY;
      int bi = 0x7fffffff;
      for (int i = tid; i < P; i += NT) {
        const float sc = piv[i] * g[i];
        if (piv[i] != 0.f && sc > 0.f && sc > bv) {
          bv = sc;
          bi = i;
        }
      }
      const float best = block_max<NT>(bv, reinterpret_cast<float*>(sh.red));
      int mine = (bv == best && best > -INFINITY) ? bi : 0x7fffffff;
      mine = block_min<NT>(mine, reinterpret_cast<int*>(sh.red));
      if (tid == 0 && mine < P) piv[mine] = 0.f;
      __syncthreads();
    }
    // ---- project, rescale -----------------------------------------------------------------
    double gn2 = 0.0;
    for (int i = tid; i < P; i += NT) {
      const float gi = (piv[i] == 0.f) ? g[i] : 0.f;
      gn2 += (double)gi * (double)gi;
    }
    gn2 = block_sum<NT>(gn2, sh.red);
    const double gn = sqrt(gn2);
    if (gn > 0.0 && (gn < 1e-15 || gn > 1e15)) {
      const double fs = 1.0 / gn;
      scale *= fs;
      f *= fs;
      for (int i = tid; i < P; i += NT) {
        g[i] = (float)(g[i] * fs);
        mm[i] = (float)(mm[i] * fs);
        ssq[i] = (float)(ssq[i] * fs * fs);
      }
      __syncthreads();
    }
    if (nrel == 0 && gn == 0.0) {
      status = CSX_FIT_CONVERGED;
      break;
    }
    // ---- AdaBelief direction --------------------------------------------------------------
    ++tb;
    b1t *= ADA_B1;
    b2t *= ADA_B2;
    double slope = 0.0;
    for (int i = tid; i < P; i += NT) {
      const bool fr = piv[i] == 0.f;
      const float gi = fr ? g[i] : 0.f;
      const float m = ADA_B1 * mm[i] + (1.f - ADA_B1) * gi;
      const float dg = gi - m;
      const float s2 = ADA_B2 * ssq[i] + (1.f - ADA_B2) * dg * dg + ADA_EPS;
      mm[i] = m;
      ssq[i] = s2;
      float di = fr ? -(m / (1.f - b1t)) / (sqrtf(s2 / (1.f - b2t)) + ADA_EPS) : 0.f;
      if ((y[i] <= 0.f && di < 0.f) || (y[i] >= 1.f && di > 0.f)) di = 0.f;  // out of the box
      dv[i] = di;
      slope += (double)gi * (double)di;
    }
    slope = block_sum<NT>(slope, sh.red);
    const double eps_f = ADA_EPS_REL * fabs(f);
    bool accepted = false;
    float alpha = 0.f, amax = 0.f;
    int jlim = 0x7fffffff;
    double ft = 0.0, dnd_t = 0.0;
    for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
      if (attempt == 1 || !(slope < 0.0)) {
        // reset the AdaBelief state; normalised projected steepest descent
        tb = 0;
        b1t = b2t = 1.f;
        float gmax = 0.f;
        for (int i = tid; i < P; i += NT) {
          mm[i] = 0.f;
          ssq[i] = 0.f;
          if (piv[i] == 0.f) gmax = fmaxf(gmax, fabsf(g[i]));
        }
        gmax = block_max<NT>(gmax, reinterpret_cast<float*>(sh.red));
        if (!(gmax > 0.f)) break;
        slope = 0.0;
        for (int i = tid; i < P; i += NT) {
          const float gi = (piv[i] == 0.f) ? g[i] : 0.f;
          float di = -gi / gmax;
          if ((y[i] <= 0.f && di < 0.f) || (y[i] >= 1.f && di > 0.f)) di = 0.f;
          dv[i] = di;
          slope += (double)gi * (double)di;
        }
        slope = block_sum<NT>(slope, sh.red);
      }
      // step limit: nearest bound along d (lowest index on ties)
      float lv = INFINITY;
      int li = 0x7fffffff;
      for (int i = tid; i < P; i += NT) {
        const float di = dv[i];
        const float lim = di < 0.f ? -y[i] / di : (di > 0.f ? (1.f - y[i]) / di : INFINITY);
        if (lim < lv) {
          lv = lim;
          li = i;
        }
      }
      amax = block_min<NT>(lv, reinterpret_cast<float*>(sh.red));
      int mine = (lv == amax) ? li : 0x7fffffff;
      jlim = block_min<NT>(mine, reinterpret_cast<int*>(sh.red));
      alpha = fminf(eta, amax);
      for (int ls = 0; ls < a.max_ls; ++ls) {
        for (int i = tid; i < P; i += NT) {
          float v = fminf(fmaxf(y[i] + alpha * dv[i], 0.f), 1.f);
          if (alpha == amax && i == jlim) v = dv[i] < 0.f ? 0.f : 1.f;
          yt[i] = v;
          c.x[i] = low(i) + rng(i) * v;
        }
        __syncthreads();
        ft = objective<NT, PATH, CSX_GRAD_ADJOINT, NOISE, false>(a, c, sh, dnd_t) * scale;
        ++nev;
        double st = 0.0;
        for (int i = tid; i < P; i += NT) {
          const float gi = (float)(c.gacc[i] * rng(i) * scale);
          gt[i] = gi;
          st += (double)gi * (double)dv[i];
        }
        st = block_sum<NT>(st, sh.red);
        if (isfinite(ft) && isfinite(st) &&
            ((ft <= f + 1e-4 * alpha * slope) || (ft <= f + eps_f && st <= 0.0))) {
          accepted = true;
          break;
        }
        alpha *= 0.5f;
      }
    }
    if (!accepted) {
      if (PATH == CSX_PATH_MOMENT && recentres < ADA_MAX_RECENTRES) {
        // the moment form rounds in proportion to the distance from the reference point
        float dref = 0.f;
        for (int i = tid; i < P; i += NT)
          dref = fmaxf(dref, fabsf(low(i) + rng(i) * y[i] - c.xr[i]) / (ADA_STEP_FACTOR * a.xtol[ptype(c, i)]));
        dref = block_max<NT>(dref, reinterpret_cast<float*>(sh.red));
        if (dref > 1.f) {
          for (int i = tid; i < P; i += NT) c.x[i] = low(i) + rng(i) * y[i];
          __syncthreads();
          dnd = recentre<NT, NOISE>(a, c, sh, smem);
          f = objective<NT, PATH, CSX_GRAD_ADJOINT, NOISE, false>(a, c, sh, dnd) * scale;
          ++nev;
          for (int i = tid; i < P; i += NT) g[i] = (float)(c.gacc[i] * rng(i) * scale);
          ++recentres;
          --it;
          __syncthreads();
          continue;
        }
      }
      status = CSX_FIT_LINESEARCH;
      break;
    }
    // ---- accept ----------------------------------------------------------------------------
    float stepr = 0.f, newt = 0.f;
    int pos = 0;
    for (int i = tid; i < P; i += NT) {
      stepr = fmaxf(stepr, fabsf(yt[i] - y[i]) / thr(i));
      y[i] = yt[i];
      g[i] = gt[i];
      if (alpha == amax && i == jlim) piv[i] = dv[i] < 0.f ? -1.f : 1.f;
    }
    __syncthreads();
    for (int i = tid; i < P; i += NT) pos += (piv[i] != 0.f && piv[i] * g[i] > 0.f) ? 1 : 0;
    stepr = block_max<NT>(stepr, reinterpret_cast<float*>(sh.red));
    pos = block_sum<NT>(pos, reinterpret_cast<int*>(sh.red));
    f = ft;
    if (PATH != CSX_PATH_MOMENT) dnd = dnd_t;
    if (alpha > 0.f) eta = fminf(1.f, 2.f * alpha);
    small = (stepr <= 1.f) ? small + 1 : 0;
    if (PATH == CSX_PATH_MOMENT && recentres < ADA_MAX_RECENTRES) {
      // move the reference point here when the fit has gone far from it (the moment form rounds in
      // proportion to that distance; first-order steps are short, so the path is long) or, near
      // convergence, unless it is already close
      float dref = 0.f;
      for (int i = tid; i < P; i += NT)
        dref = fmaxf(dref, fabsf(low(i) + rng(i) * y[i] - c.xr[i]) / a.xtol[ptype(c, i)]);
      dref = block_max<NT>(dref, reinterpret_cast<float*>(sh.red));
      if (dref > 1000.f || (small >= 2 && dref > 30.f * ADA_STEP_FACTOR)) {
        for (int i = tid; i < P; i += NT) c.x[i] = low(i) + rng(i) * y[i];
        __syncthreads();
        dnd = recentre<NT, NOISE>(a, c, sh, smem);
        f = objective<NT, PATH, CSX_GRAD_ADJOINT, NOISE, false>(a, c, sh, dnd) * scale;
        ++nev;
        for (int i = tid; i < P; i += NT) g[i] = (float)(c.gacc[i] * rng(i) * scale);
        ++recentres;
        small = 0;
        __syncthreads();
        continue;
      }
    }
    if (small >= 2 && pos == 0) {
      // candidate stop: the Gauss-Newton diagonal at this point (one more evaluation, same
      // gradient) gives each free parameter's Newton-step estimate |dL/dx_i| / H_ii
      for (int i = tid; i < P; i += NT) c.x[i] = low(i) + rng(i) * y[i];
      __syncthreads();
      double dn2 = dnd;
      (void)objective<NT, PATH, CSX_GRAD_ADJOINT, NOISE, true>(a, c, sh, dn2);
      ++nev;
      for (int i = tid; i < P; i += NT)
        if (piv[i] == 0.f && c.hacc[i] > 0.f)
          newt = fmaxf(newt, fabsf(c.gacc[i]) / (c.hacc[i] * a.xtol[ptype(c, i)]));
      newt = block_max<NT>(newt, reinterpret_cast<float*>(sh.red));
      if (newt <= 1.f) {
        status = CSX_FIT_CONVERGED;
        break;
      }
      // still far along some parameter while the steps are short: restart the AdaBelief moments
      small = 0;
      tb = 0;
      b1t = b2t = 1.f;
      for (int i = tid; i < P; i += NT) {
        mm[i] = 0.f;
        ssq[i] = 0.f;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < P; i += NT) a.beta_out[poff + i] = low(i) + rng(i) * y[i];
  if (tid == 0) {
    a.L_out[q] = f / scale - dnd;  // L = chi2_min - sum d^T N d
    a.status[q] = status;
    a.iters[q] = min(it + 1, a.max_iter);
    if (a.nevals) a.nevals[q] = nev;
  }
  __syncthreads();
}

// The problem's view of its CTA slot (layout sized by fit_slot_floats): optimiser vectors, L-BFGS
// history, SED tables of the current and reference points, warp partials, cell moments.
template <int NT, int PATH>
__device__ __forceinline__ void setup_ctx(const FitArgs& a, const ProbDesc& pd, float* base,
                                          Shared& sh, float* build_smem, Ctx& c) {
  const long long Pm = a.Pmax;
  c.P = pd.P;
  c.Kd = pd.Kd;
  c.KT = pd.KT;
  c.Ks = pd.Ks;
  c.rows = pd.Kd + 2 * pd.KT + pd.Ks;
  c.npix = a.npix;
  c.lab = a.labels + (long long)pd.conf * 3 * a.npix;
  c.perm = a.perm ? a.perm + (long long)pd.conf * a.npix : nullptr;
  c.coff = a.cell_off ? a.cell_off + (long long)pd.conf * (a.npix + 1) : nullptr;
  c.ncell = a.ncell ? a.ncell[pd.conf] : 0;
  c.d = a.d + (long long)pd.real * a.npix * 2 * NB;
  c.z = base;
  c.g = base + Pm;
  c.p = base + 2 * Pm;
  c.zt = base + 3 * Pm;
  c.gt = base + 4 * Pm;
  c.hs = base + 5 * Pm;
  c.x = base + 6 * Pm;
  const bool sm = pd.P <= SMEM_P;
  c.gacc = sm ? sh.gacc : base + 7 * Pm;
  c.hacc = sm ? sh.hacc : base + 8 * Pm;
  c.S = base + 9 * Pm;
  c.Y = c.S + (long long)a.history * Pm;
  c.tab = c.Y + (long long)a.history * Pm;
  c.tabr = c.tab + (long long)a.rows_max * NB;
  c.xr = c.tabr + (long long)a.rows_max * NB;
  float* gwg = c.xr + Pm;  // warp partials in global memory: [8][Pmax] gradient, then GN diagonal
  c.gw = sm ? build_smem + fit_rows_floats<NT, PATH>() : gwg;
  c.hw = gwg + 8 * Pm;
  c.mom = base + ((gwg + 16 * Pm - base + 31) & ~31LL);  // 128-byte aligned groups
  c.trip = reinterpret_cast<int*>(c.mom + (long long)NM * mom_cells(a.ncell_max));
  c.smem = build_smem;
}

template <int NT, int PATH, int GMODE, int NOISE, int SOLVER>
__global__ void __launch_bounds__(NT, (PATH == CSX_PATH_MOMENT && NT <= 128)
                                         ? CSX_FIT_MIN_BLOCKS * (128 / NT) : 1)
k_fit(const __grid_constant__ FitArgs a) {
  __shared__ Shared sh;
  __shared__ int s_q;
  extern __shared__ float4 build_smem4[];  // moment build staging (moment path only)
  float* build_smem = reinterpret_cast<float*>(build_smem4);
  float* base = a.slots + (long long)blockIdx.x * a.slot_floats;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(a.head, 1);
    __syncthreads();
    const int qi = s_q;
    __syncthreads();
    if (qi >= a.nprob) break;
    const int q = a.order[qi];
    const ProbDesc pd = a.probs[q];
    Ctx c;
    setup_ctx<NT, PATH>(a, pd, base, sh, build_smem, c);
    if (PATH == CSX_PATH_MOMENT && c.ncell < 0) {
      // the configuration has a label outside [0, K_j) (found when its cells were built)
      for (int i = threadIdx.x; i < c.P; i += NT) {
        const int t = ptype(c, i);
        a.beta_out[pd.poff + i] = fminf(fmaxf(a.beta0[pd.poff + i], a.lower[t]), a.upper[t]);
      }
      if (threadIdx.x == 0) {
        a.L_out[q] = (double)nan_f();
        a.status[q] = CSX_FIT_BADLABEL;
        a.iters[q] = 0;
        if (a.nevals) a.nevals[q] = 0;
      }
      __syncthreads();
      continue;
    }
    if (SOLVER == CSX_SOLVER_ADATOPK)
      fit_problem_adatopk<NT, PATH, NOISE>(a, c, sh, build_smem, q, pd.poff);
    else
      fit_problem<NT, PATH, GMODE, NOISE>(a, c, sh, build_smem, q, pd.poff);
  }
}

// ---------------------------------------------------------------------------- launcher --------
int fit_slot_floats(int Pmax, int rows_max, int ncell_max, int history, int path, long long* out) {
  long long n = (long long)(9 + 2 * history) * Pmax + (long long)rows_max * NB;
  n += (long long)rows_max * NB + Pmax;  // reference tables and parameters (moment path)
  n += 16LL * Pmax;                      // warp partials (gradient, Gauss-Newton diagonal)
  if (path == CSX_PATH_MOMENT) n += 32 + (long long)NM * mom_cells(ncell_max) + 3LL * ncell_max;
  n = (n + 63) & ~63LL;
  *out = n;
  return CSX_OK;
}

template <int NT, int PATH>
constexpr size_t fit_dyn_smem() {
  // moment path: build staging (32 pixel rows per warp) or, during evaluations, 90 floats per
  // thread followed by the warp partials; streaming path: the warp partials
  constexpr size_t build = (size_t)(NT / 32) * BUILD_SMEM_PER_WARP;
  constexpr size_t eval = (size_t)fit_rows_floats<NT, PATH>() + (size_t)(NT / 32) * SMEM_P;
  if (PATH != CSX_PATH_MOMENT) return eval * sizeof(float);
  return (build > eval ? build : eval) * sizeof(float);
}

// ------------------------------------------------------------------ fixed-point evaluation ------
// L and dL/dbeta of nprob problems of one configuration by the fit's own cell-moment evaluation:
// per problem q (realization q), the residual moments of its cells about beta0[q] (one pass over
// the pixels, build_moments), then L = chi2 - sum d^T N d and the gradient at beta_eval[q] from the
// moments alone (eval_moment). CTA b takes problems b, b + grid, ...; slot layout as the fit's.
template <int NT, int NOISE>
__global__ void __launch_bounds__(NT, CSX_FIT_MIN_BLOCKS) k_cell_eval(const __grid_constant__ FitArgs a) {
  __shared__ Shared sh;
  extern __shared__ float4 ce_smem4[];
  float* build_smem = reinterpret_cast<float*>(ce_smem4);
  float* base = a.slots + (long long)blockIdx.x * a.slot_floats;
  for (int q = blockIdx.x; q < a.nprob; q += gridDim.x) {
    const ProbDesc pd = a.probs[q];
    Ctx c;
    setup_ctx<NT, CSX_PATH_MOMENT>(a, pd, base, sh, build_smem, c);
    if (c.ncell < 0) {  // a label outside [0, K_j)
      for (int i = threadIdx.x; i < c.P; i += NT) a.grad_out[pd.poff + i] = nan_f();
      if (threadIdx.x == 0) a.L_out[q] = (double)nan_f();
      continue;
    }
    for (int i = threadIdx.x; i < c.P; i += NT) c.x[i] = a.beta0[pd.poff + i];
    __syncthreads();
    const double dnd = recentre<NT, NOISE>(a, c, sh, build_smem);
    for (int i = threadIdx.x; i < c.P; i += NT) c.x[i] = a.beta_eval[pd.poff + i];
    __syncthreads();
    const double chi = eval_moment<NT, false>(a, c, sh);
    for (int i = threadIdx.x; i < c.P; i += NT) a.grad_out[pd.poff + i] = c.gacc[i];
    if (threadIdx.x == 0) a.L_out[q] = chi - dnd;
    __syncthreads();
  }
}

template <int NOISE>
static int launch_cell_eval_t(const FitArgs& a, int grid, cudaStream_t s) {
  constexpr size_t dyn = fit_dyn_smem<128, CSX_PATH_MOMENT>();
  CSX_CUDA(cudaFuncSetAttribute(k_cell_eval<128, NOISE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dyn));
  k_cell_eval<128, NOISE><<<grid, 128, dyn, s>>>(a);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

int launch_cell_eval(const FitArgs& a, int grid, cudaStream_t s) {
  if (a.nprob == 0) return CSX_OK;
  return a.noise_kind == CSX_NOISE_SEPARABLE ? launch_cell_eval_t<CSX_NOISE_SEPARABLE>(a, grid, s)
                                             : launch_cell_eval_t<CSX_NOISE_HOMOGENEOUS>(a, grid, s);
}

template <int NT, int PATH, int GMODE, int NOISE, int SOLVER>
static int prepare_kernel() {
  const size_t dyn = fit_dyn_smem<NT, PATH>();
  if (dyn > 0)
    CSX_CUDA(cudaFuncSetAttribute(k_fit<NT, PATH, GMODE, NOISE, SOLVER>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  return CSX_OK;
}

template <int NT, int PATH, int GMODE, int NOISE, int SOLVER>
static int occupancy_grid(int* grid) {
  int dev = 0, sms = 0, per = 0;
  int rc = prepare_kernel<NT, PATH, GMODE, NOISE, SOLVER>();
  if (rc) return rc;
  CSX_CUDA(cudaGetDevice(&dev));
  CSX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CSX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fit<NT, PATH, GMODE, NOISE, SOLVER>, NT,
                                                         fit_dyn_smem<NT, PATH>()));
  if (per < 1) per = 1;
  *grid = sms * per;
  return CSX_OK;
}

template <int NT, int PATH, int GMODE, int NOISE, int SOLVER>
static int launch_one(const FitArgs& a, int grid, cudaStream_t s) {
  int rc = prepare_kernel<NT, PATH, GMODE, NOISE, SOLVER>();
  if (rc) return rc;
  k_fit<NT, PATH, GMODE, NOISE, SOLVER><<<grid, NT, fit_dyn_smem<NT, PATH>(), s>>>(a);
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

// CTA size: the moment path runs 128-thread CTAs by default (four problems per SM overlap their
// barriers), the streaming path 256; `threads` (64, 128 or 256) overrides it for the moment path
// (64 with L-BFGS only).
static int fit_threads(int threads, int path) {
  if (path != CSX_PATH_MOMENT) return 256;
  return (threads == 256 || threads == 64) ? threads : 128;
}

int fit_grid(int threads, int path, int grad_mode, int solver, int* grid) {
  constexpr int M = CSX_PATH_MOMENT, ST = CSX_PATH_STREAM, AD = CSX_GRAD_ADJOINT, FD = CSX_GRAD_FD;
  constexpr int SE = CSX_NOISE_SEPARABLE, LB = CSX_SOLVER_LBFGS, AT = CSX_SOLVER_ADATOPK;
  const bool ada = solver == AT;
  if (path == M) {
    const int nt = fit_threads(threads, path);
    if (nt == 64 && !ada) return occupancy_grid<64, M, AD, SE, LB>(grid);
    if (nt == 128 || nt == 64)
      return ada ? occupancy_grid<128, M, AD, SE, AT>(grid) : occupancy_grid<128, M, AD, SE, LB>(grid);
    return ada ? occupancy_grid<256, M, AD, SE, AT>(grid) : occupancy_grid<256, M, AD, SE, LB>(grid);
  }
  if (grad_mode == FD) return occupancy_grid<256, ST, FD, SE, LB>(grid);
  return ada ? occupancy_grid<256, ST, AD, SE, AT>(grid) : occupancy_grid<256, ST, AD, SE, LB>(grid);
}

template <int SOLVER>
static int launch_adjoint(const FitArgs& a, int threads, int grid, cudaStream_t s) {
  constexpr int M = CSX_PATH_MOMENT, ST = CSX_PATH_STREAM, AD = CSX_GRAD_ADJOINT;
  constexpr int HO = CSX_NOISE_HOMOGENEOUS, SE = CSX_NOISE_SEPARABLE, PP = CSX_NOISE_PERPIXEL;
  if (a.path == M) {
    const bool sep = a.noise_kind == SE;
    const int nt = fit_threads(threads, M);
    if (nt == 64 && SOLVER == CSX_SOLVER_LBFGS)
      return sep ? launch_one<64, M, AD, SE, SOLVER>(a, grid, s)
                 : launch_one<64, M, AD, HO, SOLVER>(a, grid, s);
    if (nt == 128 || nt == 64)
      return sep ? launch_one<128, M, AD, SE, SOLVER>(a, grid, s)
                 : launch_one<128, M, AD, HO, SOLVER>(a, grid, s);
    return sep ? launch_one<256, M, AD, SE, SOLVER>(a, grid, s)
               : launch_one<256, M, AD, HO, SOLVER>(a, grid, s);
  }
  if (a.noise_kind == SE) return launch_one<256, ST, AD, SE, SOLVER>(a, grid, s);
  if (a.noise_kind == HO) return launch_one<256, ST, AD, HO, SOLVER>(a, grid, s);
  return launch_one<256, ST, AD, PP, SOLVER>(a, grid, s);
}

int launch_fit(const FitArgs& a, int threads, int grid, cudaStream_t s) {
  if (a.nprob == 0) return CSX_OK;
  CSX_CUDA(cudaMemsetAsync(a.head, 0, sizeof(int), s));
  constexpr int ST = CSX_PATH_STREAM, FD = CSX_GRAD_FD, LB = CSX_SOLVER_LBFGS;
  constexpr int HO = CSX_NOISE_HOMOGENEOUS, SE = CSX_NOISE_SEPARABLE, PP = CSX_NOISE_PERPIXEL;
  if (a.grad_mode == FD) {
    if (a.noise_kind == SE) return launch_one<256, ST, FD, SE, LB>(a, grid, s);
    if (a.noise_kind == HO) return launch_one<256, ST, FD, HO, LB>(a, grid, s);
    return launch_one<256, ST, FD, PP, LB>(a, grid, s);
  }
  if (a.solver == CSX_SOLVER_ADATOPK) return launch_adjoint<CSX_SOLVER_ADATOPK>(a, threads, grid, s);
  return launch_adjoint<LB>(a, threads, grid, s);
}

}  // namespace csx
