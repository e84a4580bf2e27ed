// Persistent batched fit beta* = argmin L(beta) (Eq. 7) over (configuration x realization)
// problems: one CTA per problem at a time, problems taken from an atomic work queue (the
// single-GPU analogue of the contiguous chunking of Sec. 3.1). Each CTA runs the whole fit:
//
//   likelihood + adjoint gradient (Eq. 4, Sec. 3.3.1), by one of two exact evaluations
//     MOMENT: separable noise N_p^-1 = w_p diag(n): every pixel of a cell (equal (l_d,l_T,l_s))
//             has the same A, so L = -sum_c tr[M_c^-1 A^T n S_c n A],  S_c = sum_{p in c} w_p
//             sum_s d d^T is built once per problem (one pass over the pixels) and each evaluation
//             costs O(cells), not O(pixels):
//               dL/dA = -2 (n S n A - n A M^-1 G) M^-1,  G = A^T n S n A,  M = A^T n A.
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

constexpr int SMEM_P = 2048;   // parameter vectors up to this length accumulate in shared memory
constexpr int MAXM = 16;       // maximum L-BFGS memory

struct Ctx {
  int P, Kd, KT, Ks, rows, ncell, npix;
  const int* lab;     // [3][npix] of the configuration
  const int* perm;    // sorted pixels
  const int* coff;    // cell offsets
  const float* d;     // [npix][2][16] of the realization
  float *z, *g, *p, *zt, *gt, *hs, *x, *gacc, *hacc, *S, *Y, *tab, *mom;
  int* trip;
};

struct Shared {
  double red[16];
  double rho[MAXM], alpha[MAXM];
  float gacc[SMEM_P], hacc[SMEM_P];
};

__device__ __forceinline__ int ptype(const Ctx& c, int i) {
  return i < c.Kd ? 0 : (i < c.Kd + c.KT ? 1 : 2);
}

// ------------------------------------------------------------------------------ tables ----------
template <int NT>
__device__ void fill_tables(const FitArgs& a, Ctx& c) {
  const int n = c.rows * NB;
  for (int i = threadIdx.x; i < n; i += NT) c.tab[i] = table_entry(a.bands, i >> 4, i & 15, c.Kd, c.KT, c.x);
  __syncthreads();
}

// ------------------------------------------------------------------------------ moments ---------
// S_c[e(i,j)] for i <= j < 15, e = i(29-i)/2 + j, stored entry-major: mom[e * ncell + cell].
// One warp per cell; lanes 0..29 = 10 upper-triangle 4x4 blocks x 3 pixel groups; partial sums
// are flushed to a second accumulator every 16 pixels to bound FP32 rounding growth.
template <int NT, bool SEP>
__device__ void build_moments(const FitArgs& a, Ctx& c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / 10, blk = lane % 10;
  const int ba = blk < 4 ? 0 : (blk < 7 ? 1 : (blk < 9 ? 2 : 3));
  const int bb = ba + blk - (ba == 0 ? 0 : (ba == 1 ? 4 : (ba == 2 ? 7 : 9)));
  for (int cell = warp; cell < c.ncell; cell += NT / 32) {
    const int i0 = c.coff[cell], i1 = c.coff[cell + 1];
    float acc[16], tot[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = tot[k] = 0.f;
    if (grp < 3) {
      int cnt = 0;
      for (int i = i0 + grp; i < i1; i += 3) {
        const int px = c.perm[i];
        const float wp = SEP ? __ldg(a.w + px) : 1.f;
        const float4* base = reinterpret_cast<const float4*>(c.d + (long long)px * 2 * NB);
        float4 rq = __ldg(base + ba), cq = __ldg(base + bb);
        float4 ru = __ldg(base + 4 + ba), cu = __ldg(base + 4 + bb);
        const float r[8] = {rq.x * wp, rq.y * wp, rq.z * wp, rq.w * wp,
                            ru.x * wp, ru.y * wp, ru.z * wp, ru.w * wp};
        const float cc[8] = {cq.x, cq.y, cq.z, cq.w, cu.x, cu.y, cu.z, cu.w};
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            acc[ii * 4 + jj] = fmaf(r[ii], cc[jj], fmaf(r[4 + ii], cc[4 + jj], acc[ii * 4 + jj]));
        if (++cnt == 16) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            tot[k] += acc[k];
            acc[k] = 0.f;
          }
          cnt = 0;
        }
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) tot[k] += acc[k];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float t1 = __shfl_down_sync(0xffffffffu, tot[k], 10);
      const float t2 = __shfl_down_sync(0xffffffffu, tot[k], 20);
      tot[k] = tot[k] + t1 + t2;
    }
    if (lane < 10) {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int i = 4 * ba + ii, j = 4 * bb + jj;
          if (i <= j && j < 15) c.mom[(long long)((i * (29 - i)) / 2 + j) * c.ncell + cell] = tot[ii * 4 + jj];
        }
    }
    if (lane == 0) {
      const int px0 = c.perm[i0];
      c.trip[cell] = c.lab[px0];
      c.trip[c.ncell + cell] = c.lab[c.npix + px0];
      c.trip[2 * c.ncell + cell] = c.lab[2 * c.npix + px0];
    }
  }
  __syncthreads();
}

// -------------------------------------------------------------------- moment evaluation --------
// Returns L; adds dL/dbeta into gacc (and the projected Gauss-Newton diagonal into hacc).
template <int NT, bool WANT_H>
__device__ double eval_moment(const FitArgs& a, Ctx& c, Shared& sh) {
  for (int i = threadIdx.x; i < c.P; i += NT) {
    c.gacc[i] = 0.f;
    if (WANT_H) c.hacc[i] = 0.f;
  }
  fill_tables<NT>(a, c);  // ends with a barrier
  const float* nb = a.ninv_band;
  float nsum = 0.f;
#pragma unroll
  for (int f = 0; f < 15; ++f) nsum += nb[f];
  double acc = 0.0;
  for (int cell = threadIdx.x; cell < c.ncell; cell += NT) {
    const int kd = c.trip[cell], kt = c.trip[c.ncell + cell], ks = c.trip[2 * c.ncell + cell];
    const float* pd = c.tab + kd * NB;
    const float* bt = c.tab + (c.Kd + kt) * NB;
    const float* dt = c.tab + (c.Kd + c.KT + kt) * NB;
    const float* ss = c.tab + (c.Kd + 2 * c.KT + ks) * NB;
    float T1[15], T2[15];
    float m01 = 0.f, m02 = 0.f, m11 = 0.f, m12 = 0.f, m22 = 0.f;
#pragma unroll
    for (int f = 0; f < 15; ++f) {
      const float a1 = pd[f] * bt[f], a2 = ss[f];
      T1[f] = nb[f] * a1;
      T2[f] = nb[f] * a2;
      m01 += T1[f];
      m02 += T2[f];
      m11 = fmaf(T1[f], a1, m11);
      m12 = fmaf(T1[f], a2, m12);
      m22 = fmaf(T2[f], a2, m22);
    }
    float B0[15], B1[15], B2[15];
#pragma unroll
    for (int f = 0; f < 15; ++f) B0[f] = B1[f] = B2[f] = 0.f;
    const float* Sc = c.mom + cell;
#pragma unroll
    for (int i = 0; i < 15; ++i) {
#pragma unroll
      for (int j = i; j < 15; ++j) {
        const float s = Sc[(long long)((i * (29 - i)) / 2 + j) * c.ncell];
        B0[i] = fmaf(s, nb[j], B0[i]);
        B1[i] = fmaf(s, T1[j], B1[i]);
        B2[i] = fmaf(s, T2[j], B2[i]);
        if (j != i) {
          B0[j] = fmaf(s, nb[i], B0[j]);
          B1[j] = fmaf(s, T1[i], B1[j]);
          B2[j] = fmaf(s, T2[i], B2[j]);
        }
      }
    }
    float G00 = 0.f, G01 = 0.f, G02 = 0.f, G11 = 0.f, G12 = 0.f, G22 = 0.f;
#pragma unroll
    for (int f = 0; f < 15; ++f) {
      G00 = fmaf(nb[f], B0[f], G00);
      G01 = fmaf(nb[f], B1[f], G01);
      G02 = fmaf(nb[f], B2[f], G02);
      G11 = fmaf(T1[f], B1[f], G11);
      G12 = fmaf(T1[f], B2[f], G12);
      G22 = fmaf(T2[f], B2[f], G22);
    }
    Chol3 ch;
    if (!chol3(nsum, m01, m02, m11, m12, m22, ch)) {
      acc += (double)nan_f();
      continue;
    }
    float v00, v01, v02, v11, v12, v22;
    chol3_inverse(ch, v00, v01, v02, v11, v12, v22);
    const float Lc = -(v00 * G00 + v11 * G11 + v22 * G22 + 2.f * (v01 * G01 + v02 * G02 + v12 * G12));
    acc += (double)Lc;
    // X = M^-1 G
    const float X00 = v00 * G00 + v01 * G01 + v02 * G02;
    const float X01 = v00 * G01 + v01 * G11 + v02 * G12;
    const float X02 = v00 * G02 + v01 * G12 + v02 * G22;
    const float X10 = v01 * G00 + v11 * G01 + v12 * G02;
    const float X11 = v01 * G01 + v11 * G11 + v12 * G12;
    const float X12 = v01 * G02 + v11 * G12 + v12 * G22;
    const float X20 = v02 * G00 + v12 * G01 + v22 * G02;
    const float X21 = v02 * G01 + v12 * G11 + v22 * G12;
    const float X22 = v02 * G02 + v12 * G12 + v22 * G22;
    float gbd = 0.f, gtd = 0.f, gbs = 0.f;
#pragma unroll
    for (int f = 0; f < 15; ++f) {
      const float a1 = pd[f] * bt[f], a2 = ss[f];
      const float e0 = B0[f] - X00 - a1 * X10 - a2 * X20;
      const float e1 = B1[f] - X01 - a1 * X11 - a2 * X21;
      const float e2 = B2[f] - X02 - a1 * X12 - a2 * X22;
      const float F1 = e0 * v01 + e1 * v11 + e2 * v12;
      const float F2 = e0 * v02 + e1 * v12 + e2 * v22;
      const float t1 = F1 * T1[f];
      gbd = fmaf(t1, a.bands.lnd[f], gbd);
      gtd = fmaf(t1, dt[f], gtd);
      gbs = fmaf(F2 * T2[f], a.bands.lns[f], gbs);
    }
    atomicAdd(c.gacc + kd, -2.f * gbd);
    atomicAdd(c.gacc + c.Kd + kt, -2.f * gtd);
    atomicAdd(c.gacc + c.Kd + c.KT + ks, -2.f * gbs);
    if (WANT_H) {
      // Q = M^-1 G M^-1 = sum_p w sum_s s_hat s_hat^T ; projected GN diagonal per parameter
      const float Q11 = X10 * v01 + X11 * v11 + X12 * v12;
      const float Q22 = X20 * v02 + X21 * v12 + X22 * v22;
      float n2[3] = {0.f, 0.f, 0.f}, u0[3] = {0.f, 0.f, 0.f}, u1[3] = {0.f, 0.f, 0.f},
            u2[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int f = 0; f < 15; ++f) {
        const float a1 = pd[f] * bt[f], a2 = ss[f];
        const float da[3] = {a1 * a.bands.lnd[f], a1 * dt[f], a2 * a.bands.lns[f]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float nda = nb[f] * da[k];
          n2[k] = fmaf(nda, da[k], n2[k]);
          u0[k] += nda;
          u1[k] = fmaf(nda, a1, u1[k]);
          u2[k] = fmaf(nda, a2, u2[k]);
        }
      }
      float h[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float quad = v00 * u0[k] * u0[k] + v11 * u1[k] * u1[k] + v22 * u2[k] * u2[k] +
                           2.f * (v01 * u0[k] * u1[k] + v02 * u0[k] * u2[k] + v12 * u1[k] * u2[k]);
        h[k] = 2.f * (k < 2 ? Q11 : Q22) * fmaxf(n2[k] - quad, 0.f);
      }
      atomicAdd(c.hacc + kd, h[0]);
      atomicAdd(c.hacc + c.Kd + kt, h[1]);
      atomicAdd(c.hacc + c.Kd + c.KT + ks, h[2]);
    }
  }
  return block_sum<NT>(acc, sh.red);
}

// -------------------------------------------------------------------- stream evaluation --------
// Returns chi2 (sum of residual norms) and, through dnd, sum d^T N d.
template <int NT, int NOISE, bool GRAD, bool WANT_H>
__device__ double eval_stream(const FitArgs& a, Ctx& c, Shared& sh, double& dnd_out) {
  if (GRAD || WANT_H) {
    for (int i = threadIdx.x; i < c.P; i += NT) {
      if (GRAD) c.gacc[i] = 0.f;
      if (WANT_H) c.hacc[i] = 0.f;
    }
  }
  fill_tables<NT>(a, c);
  float nb[NB];
#pragma unroll
  for (int f = 0; f < NB; ++f) nb[f] = a.ninv_band[f];
  double chi = 0.0, dn = 0.0;
  const int* ld = c.lab;
  const int* lt = c.lab + c.npix;
  const int* ls = c.lab + 2 * c.npix;
  for (int p = threadIdx.x; p < c.npix; p += NT) {
    const int kd = ld[p], kt = lt[p], ks = ls[p];
    if ((unsigned)kd >= (unsigned)c.Kd || (unsigned)kt >= (unsigned)c.KT ||
        (unsigned)ks >= (unsigned)c.Ks) {
      chi += (double)nan_f();
      continue;
    }
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
    PixOut o;
    if (!pixel_eval<GRAD, WANT_H>(dq, du, nn, c.tab + kd * NB, c.tab + (c.Kd + kt) * NB,
                                  c.tab + (c.Kd + c.KT + kt) * NB,
                                  c.tab + (c.Kd + 2 * c.KT + ks) * NB, a.bands, o)) {
      chi += (double)nan_f();
      continue;
    }
    chi += (double)o.chi2;
    dn += (double)o.dnd;
    if (GRAD) {
      atomicAdd(c.gacc + kd, o.gbd);
      atomicAdd(c.gacc + c.Kd + kt, o.gtd);
      atomicAdd(c.gacc + c.Kd + c.KT + ks, o.gbs);
    }
    if (WANT_H) {
      atomicAdd(c.hacc + kd, o.hbd);
      atomicAdd(c.hacc + c.Kd + kt, o.htd);
      atomicAdd(c.hacc + c.Kd + c.KT + ks, o.hbs);
    }
  }
  block_sum2<NT>(chi, dn, sh.red);
  dnd_out = dn;
  return chi;
}

// -------------------------------------------------------------------- objective ---------------
// f(x) at the physical parameters in c.x; gradient (physical units) in c.gacc.
template <int NT, int PATH, int GMODE, int NOISE, bool WANT_H>
__device__ double objective(const FitArgs& a, Ctx& c, Shared& sh, double& dnd) {
  if (PATH == CSX_PATH_MOMENT) {
    dnd = 0.0;
    return eval_moment<NT, WANT_H>(a, c, sh);
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
template <int NT, int PATH, int GMODE, int NOISE>
__device__ void fit_problem(const FitArgs& a, Ctx& c, Shared& sh, int q, long long poff) {
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
  double f = objective<NT, PATH, GMODE, NOISE, true>(a, c, sh, dnd);
  int status = CSX_FIT_MAXITER, it = 0;
  if (!isfinite(f)) {
    for (int i = tid; i < P; i += NT) a.beta_out[poff + i] = c.x[i];
    if (tid == 0) {
      a.L_out[q] = (double)nan_f();
      a.status[q] = CSX_FIT_NONPHYSICAL;
      a.iters[q] = 0;
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
  if (GMODE == CSX_GRAD_FD) fd_gradient<NT, NOISE>(a, c, sh, c.z, c.g);

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
    for (int j = 0; j < count; ++j) {
      const int k = (head - 1 - j + m) % m;
      const float* Sk = c.S + (long long)k * a.Pmax;
      double dot = 0.0;
      for (int i = tid; i < P; i += NT) dot += (double)Sk[i] * (double)c.p[i];
      dot = block_sum<NT>(dot, sh.red);
      const double al = sh.rho[k] * dot;
      if (tid == 0) sh.alpha[k] = al;
      const float* Yk = c.Y + (long long)k * a.Pmax;
      for (int i = tid; i < P; i += NT) c.p[i] -= (float)al * Yk[i];
    }
    for (int i = tid; i < P; i += NT) c.p[i] *= (float)gamma;
    for (int j = count - 1; j >= 0; --j) {
      const int k = (head - 1 - j + m) % m;
      const float* Yk = c.Y + (long long)k * a.Pmax;
      double dot = 0.0;
      for (int i = tid; i < P; i += NT) dot += (double)Yk[i] * (double)c.p[i];
      dot = block_sum<NT>(dot, sh.red);
      const double be = sh.rho[k] * dot;
      const float* Sk = c.S + (long long)k * a.Pmax;
      const float coef = (float)(sh.alpha[k] - be);
      for (int i = tid; i < P; i += NT) c.p[i] += coef * Sk[i];
    }
    // negate, mask the active set and outward steps at a bound, directional derivative, QN step
    double gp = 0.0;
    float stepn = 0.f;
    for (int i = tid; i < P; i += NT) {
      const int t = ptype(c, i);
      const float zl = c.hs[i] * a.lower[t], zu = c.hs[i] * a.upper[t];
      const float gi = c.g[i];
      const bool act = (c.z[i] <= zl && gi > 0.f) || (c.z[i] >= zu && gi < 0.f);
      float pi = act ? 0.f : -c.p[i];
      if ((c.z[i] <= zl && pi < 0.f) || (c.z[i] >= zu && pi > 0.f)) pi = 0.f;
      c.p[i] = pi;
      gp += (double)gi * (double)pi;
      stepn = fmaxf(stepn, fabsf(pi) / c.hs[i] / a.xtol[t]);
    }
    gp = block_sum<NT>(gp, sh.red);
    stepn = block_max<NT>(stepn, reinterpret_cast<float*>(sh.red));
    if (!(gp < 0.0)) {
      // not a descent direction: restart from the projected steepest descent
      count = 0;
      gamma = 1.0;
      gp = 0.0;
      stepn = 0.f;
      for (int i = tid; i < P; i += NT) {
        const int t = ptype(c, i);
        const float zl = c.hs[i] * a.lower[t], zu = c.hs[i] * a.upper[t];
        const float gi = c.g[i];
        const bool act = (c.z[i] <= zl && gi > 0.f) || (c.z[i] >= zu && gi < 0.f);
        float pi = act ? 0.f : -gi;
        if ((c.z[i] <= zl && pi < 0.f) || (c.z[i] >= zu && pi > 0.f)) pi = 0.f;
        c.p[i] = pi;
        gp += (double)gi * (double)pi;
        stepn = fmaxf(stepn, fabsf(pi) / c.hs[i] / a.xtol[t]);
      }
      gp = block_sum<NT>(gp, sh.red);
      stepn = block_max<NT>(stepn, reinterpret_cast<float*>(sh.red));
      if (!(gp < 0.0)) {
        status = CSX_FIT_CONVERGED;  // projected gradient vanishes
        break;
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
      if (GMODE == CSX_GRAD_FD) {
        fd_gradient<NT, NOISE>(a, c, sh, c.zt, c.gt);
      } else {
        for (int i = tid; i < P; i += NT) c.gt[i] = c.gacc[i] / c.hs[i];
      }
      double dphi = 0.0;
      for (int i = tid; i < P; i += NT) dphi += (double)c.gt[i] * (double)c.p[i];
      dphi = block_sum<NT>(dphi, sh.red);
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
      if (count > 0) {  // drop the curvature history and retry from steepest descent
        count = 0;
        gamma = 1.0;
        continue;
      }
      status = CSX_FIT_LINESEARCH;
      break;
    }
    // ---- accept: curvature pair and update --------------------------------------------
    double sy = 0.0, yy = 0.0;
    float sn = 0.f;
    float* Sn = c.S + (long long)head * a.Pmax;
    float* Yn = c.Y + (long long)head * a.Pmax;
    for (int i = tid; i < P; i += NT) {
      const int t = ptype(c, i);
      const float si = c.zt[i] - c.z[i], yi = c.gt[i] - c.g[i];
      Sn[i] = si;
      Yn[i] = yi;
      sy += (double)si * (double)yi;
      yy += (double)yi * (double)yi;
      sn = fmaxf(sn, fabsf(si) / c.hs[i] / a.xtol[t]);
      c.z[i] = c.zt[i];
      c.g[i] = c.gt[i];
    }
    block_sum2<NT>(sy, yy, sh.red);
    sn = block_max<NT>(sn, reinterpret_cast<float*>(sh.red));
    last_step = sn;
    f = ft;
    dnd = dnd_t;
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
    a.L_out[q] = (PATH == CSX_PATH_MOMENT) ? f : f - dnd;
    a.status[q] = status;
    a.iters[q] = it;
  }
  __syncthreads();
}

template <int NT, int PATH, int GMODE, int NOISE>
__global__ void __launch_bounds__(NT) k_fit(const __grid_constant__ FitArgs a) {
  __shared__ Shared sh;
  __shared__ int s_q;
  float* base = a.slots + (long long)blockIdx.x * a.slot_floats;
  const int Pm = a.Pmax;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(a.head, 1);
    __syncthreads();
    const int qi = s_q;
    __syncthreads();
    if (qi >= a.nprob) break;
    const int q = a.order[qi];
    const ProbDesc pd = a.probs[q];
    Ctx c;
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
    c.mom = c.tab + (long long)a.rows_max * NB;
    c.trip = reinterpret_cast<int*>(c.mom + (long long)NE * a.ncell_max);
    if (PATH == CSX_PATH_MOMENT)
      build_moments<NT, NOISE == CSX_NOISE_SEPARABLE>(a, c);
    fit_problem<NT, PATH, GMODE, NOISE>(a, c, sh, q, pd.poff);
  }
}

// ---------------------------------------------------------------------------- launcher --------
int fit_slot_floats(int Pmax, int rows_max, int ncell_max, int history, int path, long long* out) {
  long long n = (long long)(9 + 2 * history) * Pmax + (long long)rows_max * NB;
  if (path == CSX_PATH_MOMENT) n += (long long)NE * ncell_max + 3LL * ncell_max;
  n = (n + 63) & ~63LL;
  *out = n;
  return CSX_OK;
}

template <int NT, int PATH, int GMODE, int NOISE>
static int occupancy_grid(int* grid) {
  int dev = 0, sms = 0, per = 0;
  CSX_CUDA(cudaGetDevice(&dev));
  CSX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CSX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fit<NT, PATH, GMODE, NOISE>, NT, 0));
  if (per < 1) per = 1;
  *grid = sms * per;
  return CSX_OK;
}

int fit_grid(int threads, int path, int grad_mode, int* grid) {
  (void)threads;
  if (path == CSX_PATH_MOMENT) return occupancy_grid<256, CSX_PATH_MOMENT, CSX_GRAD_ADJOINT, CSX_NOISE_SEPARABLE>(grid);
  if (grad_mode == CSX_GRAD_FD) return occupancy_grid<256, CSX_PATH_STREAM, CSX_GRAD_FD, CSX_NOISE_SEPARABLE>(grid);
  return occupancy_grid<256, CSX_PATH_STREAM, CSX_GRAD_ADJOINT, CSX_NOISE_SEPARABLE>(grid);
}

int launch_fit(const FitArgs& a, int threads, int grid, cudaStream_t s) {
  (void)threads;
  if (a.nprob == 0) return CSX_OK;
  CSX_CUDA(cudaMemsetAsync(a.head, 0, sizeof(int), s));
  constexpr int NT = 256;
  if (a.path == CSX_PATH_MOMENT) {
    if (a.noise_kind == CSX_NOISE_SEPARABLE)
      k_fit<NT, CSX_PATH_MOMENT, CSX_GRAD_ADJOINT, CSX_NOISE_SEPARABLE><<<grid, NT, 0, s>>>(a);
    else
      k_fit<NT, CSX_PATH_MOMENT, CSX_GRAD_ADJOINT, CSX_NOISE_HOMOGENEOUS><<<grid, NT, 0, s>>>(a);
  } else if (a.grad_mode == CSX_GRAD_FD) {
    if (a.noise_kind == CSX_NOISE_SEPARABLE)
      k_fit<NT, CSX_PATH_STREAM, CSX_GRAD_FD, CSX_NOISE_SEPARABLE><<<grid, NT, 0, s>>>(a);
    else if (a.noise_kind == CSX_NOISE_HOMOGENEOUS)
      k_fit<NT, CSX_PATH_STREAM, CSX_GRAD_FD, CSX_NOISE_HOMOGENEOUS><<<grid, NT, 0, s>>>(a);
    else
      k_fit<NT, CSX_PATH_STREAM, CSX_GRAD_FD, CSX_NOISE_PERPIXEL><<<grid, NT, 0, s>>>(a);
  } else {
    if (a.noise_kind == CSX_NOISE_SEPARABLE)
      k_fit<NT, CSX_PATH_STREAM, CSX_GRAD_ADJOINT, CSX_NOISE_SEPARABLE><<<grid, NT, 0, s>>>(a);
    else if (a.noise_kind == CSX_NOISE_HOMOGENEOUS)
      k_fit<NT, CSX_PATH_STREAM, CSX_GRAD_ADJOINT, CSX_NOISE_HOMOGENEOUS><<<grid, NT, 0, s>>>(a);
    else
      k_fit<NT, CSX_PATH_STREAM, CSX_GRAD_ADJOINT, CSX_NOISE_PERPIXEL><<<grid, NT, 0, s>>>(a);
  }
  CSX_CUDA(cudaGetLastError());
  return CSX_OK;
}

}  // namespace csx
