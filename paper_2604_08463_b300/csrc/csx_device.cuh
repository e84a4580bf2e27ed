// Device building blocks shared by the csx kernels: band constants, SED tables (Eq. 5),
// the per-pixel residual-form likelihood/gradient (Eqs. 3-4, Sec. 3.3.1), a 3x3 Cholesky
// solve and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/csx.h"

namespace csx {

constexpr int NB = 16;     // padded band slots per pixel vector
constexpr int NE = 120;    // unique entries of a symmetric 15x15 band moment

// Per-band constants of the spectral model, computed on the host in double from csx_model.
struct Bands {
  int nf;
  float xk0;          // h nu0_dust / k  [K]
  float lnd[NB];      // ln(nu_f / nu0_dust)           (0 for f >= nf)
  float lns[NB];      // ln(nu_f / nu0_sync)
  float xk[NB];       // h nu_f / k  [K]
  float cd[NB];       // (nu_f / nu0_dust) * u_f / u_dust   (u = RJ->K_CMB factor, 1 in RJ units)
  float cs[NB];       // u_f / u_sync
};

// ---------------------------------------------------------------------------------------------
// SED tables. Rows of a problem with (Kd, KT, Ks) patches, 16 floats each:
//   [0, Kd)            P_d[k][f] = (nu_f/nu0_d)^beta_d,k
//   [Kd, Kd+KT)        B[j][f]   = (nu_f/nu0_d) (e^{x0}-1)/(e^{x_f}-1) u_f/u_d,  x = h nu / k T_d,j
//   [Kd+KT, Kd+2KT)    D[j][f]   = d ln B / dT = [x_f/(1-e^{-x_f}) - x0/(1-e^{-x0})] / T_d,j
//   [Kd+2KT, +Ks)      S[k][f]   = (nu_f/nu0_s)^beta_s,k u_f/u_s
// so that the dust column is A_d = P_d[l_d] * B[l_T] and the synchrotron column A_s = S[l_s].
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float nan_f() { return __int_as_float(0x7fffffff); }

__device__ __forceinline__ float table_entry(const Bands& b, int row, int f, int Kd, int KT,
                                             const float* __restrict__ x) {
  if (f >= b.nf) return 0.f;
  if (row < Kd) return expf(x[row] * b.lnd[f]);
  row -= Kd;
  if (row < KT) {
    const float T = x[Kd + row];
    if (!(T > 0.f)) return nan_f();
    return b.cd[f] * expm1f(b.xk0 / T) / expm1f(b.xk[f] / T);
  }
  row -= KT;
  if (row < KT) {
    const float T = x[Kd + row];
    if (!(T > 0.f)) return nan_f();
    const float xf = b.xk[f] / T, x0 = b.xk0 / T;
    return (xf / -expm1f(-xf) - x0 / -expm1f(-x0)) / T;
  }
  row -= KT;
  return b.cs[f] * expf(x[Kd + KT + row] * b.lns[f]);
}

// ---------------------------------------------------------------------------------------------
// 3x3 symmetric positive-definite factorisation M = L L^T (lower L, inverse diagonal kept).
// ---------------------------------------------------------------------------------------------
struct Chol3 {
  float l10, l20, l21, i00, i11, i22;
};

__device__ __forceinline__ bool chol3(float m00, float m01, float m02, float m11, float m12,
                                      float m22, Chol3& c) {
  if (!(m00 > 0.f)) return false;
  const float l00 = sqrtf(m00);
  c.i00 = 1.f / l00;
  c.l10 = m01 * c.i00;
  c.l20 = m02 * c.i00;
  const float t11 = fmaf(-c.l10, c.l10, m11);
  if (!(t11 > 0.f)) return false;
  const float l11 = sqrtf(t11);
  c.i11 = 1.f / l11;
  c.l21 = fmaf(-c.l20, c.l10, m12) * c.i11;
  const float t22 = fmaf(-c.l21, c.l21, fmaf(-c.l20, c.l20, m22));
  if (!(t22 > 0.f)) return false;
  c.i22 = 1.f / sqrtf(t22);
  return true;
}

// Solve M s = b with the factor of M.
__device__ __forceinline__ void chol3_solve(const Chol3& c, float b0, float b1, float b2,
                                            float& s0, float& s1, float& s2) {
  const float y0 = b0 * c.i00;
  const float y1 = fmaf(-c.l10, y0, b1) * c.i11;
  const float y2 = fmaf(-c.l21, y1, fmaf(-c.l20, y0, b2)) * c.i22;
  s2 = y2 * c.i22;
  s1 = fmaf(-c.l21, s2, y1) * c.i11;
  s0 = fmaf(-c.l20, s2, fmaf(-c.l10, s1, y0)) * c.i00;
}

// Symmetric inverse of M from its factor: returns (v00, v01, v02, v11, v12, v22).
__device__ __forceinline__ void chol3_inverse(const Chol3& c, float& v00, float& v01, float& v02,
                                              float& v11, float& v12, float& v22) {
  // L^-1 (lower): a00, a10, a11, a20, a21, a22
  const float a00 = c.i00, a11 = c.i11, a22 = c.i22;
  const float a10 = -c.l10 * a00 * a11;
  const float a21 = -c.l21 * a11 * a22;
  const float a20 = -(c.l20 * a00 + c.l21 * a10) * a22;
  // M^-1 = L^-T L^-1
  v00 = a00 * a00 + a10 * a10 + a20 * a20;
  v01 = a10 * a11 + a20 * a21;
  v02 = a20 * a22;
  v11 = a11 * a11 + a21 * a21;
  v12 = a21 * a22;
  v22 = a22 * a22;
}

// ---------------------------------------------------------------------------------------------
// Per-pixel likelihood in the residual form and adjoint gradient contributions.
//   s_hat = (A^T N A)^-1 A^T N d_s (Eq. 3), r_s = d_s - A s_hat,
//   chi2 = sum_s r_s^T N r_s, dnd = sum_s d_s^T N d_s  (L_pixel = chi2 - dnd),
//   dL/dtheta = -2 sum_s (N r_s)^T (dA/dtheta) s_hat_s   (Sec. 3.3.1)
// with dA_d/dbeta_d = A_d ln(nu/nu0_d), dA_d/dT_d = A_d D, dA_s/dbeta_s = A_s ln(nu/nu0_s).
// Optional Gauss-Newton diagonal h_theta = 2 sum_s s_hat_s,k^2 (dA/dtheta)^T N (dA/dtheta).
// Returns false when M is not positive definite (the caller turns that into NaN).
// ---------------------------------------------------------------------------------------------
struct PixOut {
  float chi2, dnd;
  float gbd, gtd, gbs;
  float hbd, htd, hbs;
};

// The GLS solve uses modified Gram-Schmidt on the columns (1, A_d, A_s) in the N-weighted inner
// product instead of the normal equations: the same result with rounding error growing with
// cond(N^1/2 A) rather than its square cond(A^T N A).
//   c1 = A_d - mu1,            mu1 = <1, A_d> / <1, 1>
//   c2 = A_s - mu2 - nu c1,    mu2 = <1, A_s> / <1, 1>,  nu = <c1, A_s> / <c1, c1>
//   t = (<1,d>/<1,1>, <c1,d>/<c1,c1>, <c2,d>/<c2,c2>),  r = d - t0 - t1 c1 - t2 c2,
//   s_hat = (t0 - mu1 s1 - mu2 s2, t1 - nu t2, t2).
struct Mgs3 {
  float mu1, mu2, nu, i0, i1, i2;  // i_k = 1 / <c_k, c_k>
};

__device__ __forceinline__ bool mgs3(const float (&nn)[NB], const float (&ad)[NB],
                                     const float (&as)[NB], float (&c1)[NB], float (&c2)[NB],
                                     Mgs3& g) {
  float n0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    n0 += nn[f];
    s1 = fmaf(nn[f], ad[f], s1);
    s2 = fmaf(nn[f], as[f], s2);
  }
  if (!(n0 > 0.f)) return false;
  g.i0 = 1.f / n0;
  g.mu1 = s1 * g.i0;
  g.mu2 = s2 * g.i0;
  float n1 = 0.f, x12 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    c1[f] = ad[f] - g.mu1;
    const float w = nn[f] * c1[f];
    n1 = fmaf(w, c1[f], n1);
    x12 = fmaf(w, as[f], x12);
  }
  if (!(n1 > 0.f)) return false;
  g.i1 = 1.f / n1;
  g.nu = x12 * g.i1;
  float n2 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    c2[f] = fmaf(-g.nu, c1[f], as[f] - g.mu2);
    n2 = fmaf(nn[f] * c2[f], c2[f], n2);
  }
  if (!(n2 > 0.f)) return false;
  g.i2 = 1.f / n2;
  return true;
}

// [(A^T N A)^-1]_00 from the Gram-Schmidt factors.
__device__ __forceinline__ float mgs3_var00(const Mgs3& g) {
  const float r02 = g.mu1 * g.nu - g.mu2;
  return g.i0 + g.mu1 * g.mu1 * g.i1 + r02 * r02 * g.i2;
}

template <bool GRAD, bool HESS>
__device__ __forceinline__ bool pixel_eval(const float (&dq)[NB], const float (&du)[NB],
                                           const float (&nn)[NB], const float* __restrict__ pd,
                                           const float* __restrict__ bt,
                                           const float* __restrict__ dt,
                                           const float* __restrict__ ss, const Bands& bc,
                                           PixOut& o) {
  float ad[NB], as[NB], c1[NB], c2[NB];
#pragma unroll
  for (int f4 = 0; f4 < NB; f4 += 4) {
    const float4 p4 = *reinterpret_cast<const float4*>(pd + f4);
    const float4 b4 = *reinterpret_cast<const float4*>(bt + f4);
    const float4 s4 = *reinterpret_cast<const float4*>(ss + f4);
    ad[f4 + 0] = p4.x * b4.x; ad[f4 + 1] = p4.y * b4.y;
    ad[f4 + 2] = p4.z * b4.z; ad[f4 + 3] = p4.w * b4.w;
    as[f4 + 0] = s4.x; as[f4 + 1] = s4.y; as[f4 + 2] = s4.z; as[f4 + 3] = s4.w;
  }
  Mgs3 g;
  if (!mgs3(nn, ad, as, c1, c2, g)) return false;
  float tq0 = 0.f, tq1 = 0.f, tq2 = 0.f, tu0 = 0.f, tu1 = 0.f, tu2 = 0.f, dnd = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    const float nq = nn[f] * dq[f], nu = nn[f] * du[f];
    tq0 += nq;
    tq1 = fmaf(nq, c1[f], tq1);
    tq2 = fmaf(nq, c2[f], tq2);
    tu0 += nu;
    tu1 = fmaf(nu, c1[f], tu1);
    tu2 = fmaf(nu, c2[f], tu2);
    dnd = fmaf(nq, dq[f], fmaf(nu, du[f], dnd));
  }
  tq0 *= g.i0; tq1 *= g.i1; tq2 *= g.i2;
  tu0 *= g.i0; tu1 *= g.i1; tu2 *= g.i2;
  const float sq2 = tq2, sq1 = fmaf(-g.nu, tq2, tq1);
  const float su2 = tu2, su1 = fmaf(-g.nu, tu2, tu1);
  float chi2 = 0.f, gbd = 0.f, gtd = 0.f, gbs = 0.f, hbd = 0.f, htd = 0.f, hbs = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    const float rq = dq[f] - fmaf(tq2, c2[f], fmaf(tq1, c1[f], tq0));
    const float ru = du[f] - fmaf(tu2, c2[f], fmaf(tu1, c1[f], tu0));
    const float nrq = nn[f] * rq, nru = nn[f] * ru;
    chi2 = fmaf(nrq, rq, fmaf(nru, ru, chi2));
    if (GRAD) {
      const float td = fmaf(nrq, sq1, nru * su1) * ad[f];
      const float ts = fmaf(nrq, sq2, nru * su2) * as[f];
      gbd = fmaf(td, bc.lnd[f], gbd);
      gtd = fmaf(td, dt[f], gtd);
      gbs = fmaf(ts, bc.lns[f], gbs);
    }
    if (HESS) {
      const float a1 = ad[f] * ad[f] * nn[f], a2 = as[f] * as[f] * nn[f];
      hbd = fmaf(a1 * bc.lnd[f], bc.lnd[f], hbd);
      htd = fmaf(a1 * dt[f], dt[f], htd);
      hbs = fmaf(a2 * bc.lns[f], bc.lns[f], hbs);
    }
  }
  o.chi2 = chi2;
  o.dnd = dnd;
  o.gbd = -2.f * gbd;
  o.gtd = -2.f * gtd;
  o.gbs = -2.f * gbs;
  if (HESS) {
    const float k1 = 2.f * fmaf(sq1, sq1, su1 * su1), k2 = 2.f * fmaf(sq2, sq2, su2 * su2);
    o.hbd = k1 * hbd;
    o.htd = k1 * htd;
    o.hbs = k2 * hbs;
  }
  return true;
}

// Load one pixel's Q and U vectors (one 128-byte line).
__device__ __forceinline__ void load_pixel(const float* __restrict__ p, float (&dq)[NB],
                                           float (&du)[NB]) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 a = __ldg(p4 + k);
    const float4 b = __ldg(p4 + 4 + k);
    dq[4 * k + 0] = a.x; dq[4 * k + 1] = a.y; dq[4 * k + 2] = a.z; dq[4 * k + 3] = a.w;
    du[4 * k + 0] = b.x; du[4 * k + 1] = b.y; du[4 * k + 2] = b.z; du[4 * k + 3] = b.w;
  }
}

// ---------------------------------------------------------------------------------------------
// Asynchronous 4-byte global -> shared copies (cp.async, L1-allocating); a thread waits for its
// own copies only.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Prefetch of the global line holding p into L1.
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p));
}
// Asynchronous prefetch of a global range into L2 (nothing to wait for): p 16-byte aligned, bytes
// a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Scatter-add of per-lane values into acc[key], combined over runs of equal keys in consecutive
// lanes: pixels in ring order fall into a patch in long runs, so a warp mostly carries one to three
// distinct keys and issues one atomic per run instead of 32 atomics on the same address. A
// segmented inclusive scan (shuffles) leaves each run's total in its last lane. Every lane of the
// warp must call it; lanes with key < 0 add nothing. Three keys are scanned together.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void warp_run_add3(float* acc0, int k0, float v0, float* acc1, int k1,
                                              float v1, float* acc2, int k2, float v2) {
  constexpr unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned upto = (2u << lane) - 1u;  // lanes 0..lane (lane 31: all bits, by wrap-around)
  const int p0 = __shfl_up_sync(full, k0, 1), p1 = __shfl_up_sync(full, k1, 1),
            p2 = __shfl_up_sync(full, k2, 1);
  const unsigned h0 = __ballot_sync(full, lane == 0 || k0 != p0);
  const unsigned h1 = __ballot_sync(full, lane == 0 || k1 != p1);
  const unsigned h2 = __ballot_sync(full, lane == 0 || k2 != p2);
  const int s0 = 31 - __clz(h0 & upto), s1 = 31 - __clz(h1 & upto), s2 = 31 - __clz(h2 & upto);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float t0 = __shfl_up_sync(full, v0, d), t1 = __shfl_up_sync(full, v1, d),
                t2 = __shfl_up_sync(full, v2, d);
    if (lane - d >= s0) v0 += t0;
    if (lane - d >= s1) v1 += t1;
    if (lane - d >= s2) v2 += t2;
  }
  // a run ends in lane 31 or before the next head
  const unsigned after = (lane == 31) ? 0xffffffffu : ((h0 >> (lane + 1)) & 1u) * 0x1u |
                                                        (((h1 >> (lane + 1)) & 1u) << 1) |
                                                        (((h2 >> (lane + 1)) & 1u) << 2);
  if (k0 >= 0 && (after & 1u)) atomicAdd(acc0 + k0, v0);
  if (k1 >= 0 && (after & 2u)) atomicAdd(acc1 + k1, v1);
  if (k2 >= 0 && (after & 4u)) atomicAdd(acc2 + k2, v2);
}

// ---------------------------------------------------------------------------------------------
// Deterministic variant of warp_run_add3 for a warp-private accumulator `acc` (a P-vector that no
// other warp writes): keys are indices into acc (three disjoint ranges), -1 = nothing to add.
// Runs of equal keys in consecutive lanes are combined by the same segmented shuffle scan; the run
// totals are then added in a fixed order. Totals with distinct keys are added at once; when several
// runs of one warp end on the same key (a label that reappears after another one), the lowest such
// lane adds their totals in increasing lane order. The result is independent of scheduling, so a
// reduction built from it gives the same bits on every run. `stage` holds 32 floats of this warp.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void warp_put_ordered(float* acc, int key, float v, bool end,
                                                 float* stage) {
  constexpr unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(full, end ? key : -1 - lane);
  if (!__any_sync(full, end && (grp & (grp - 1u)) != 0u)) {
    if (end) acc[key] += v;
    return;
  }
  stage[lane] = v;
  __syncwarp();
  if (end && (grp & ((1u << lane) - 1u)) == 0u) {
    float t = 0.f;
    for (unsigned m = grp; m; m &= m - 1u) t += stage[__ffs(m) - 1];
    acc[key] += t;
  }
  __syncwarp();
}

__device__ __forceinline__ void warp_run_accum3(float* acc, int k0, float v0, int k1, float v1,
                                                int k2, float v2, float* stage) {
  constexpr unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned upto = (2u << lane) - 1u;
  const int p0 = __shfl_up_sync(full, k0, 1), p1 = __shfl_up_sync(full, k1, 1),
            p2 = __shfl_up_sync(full, k2, 1);
  const unsigned h0 = __ballot_sync(full, lane == 0 || k0 != p0);
  const unsigned h1 = __ballot_sync(full, lane == 0 || k1 != p1);
  const unsigned h2 = __ballot_sync(full, lane == 0 || k2 != p2);
  const int s0 = 31 - __clz(h0 & upto), s1 = 31 - __clz(h1 & upto), s2 = 31 - __clz(h2 & upto);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float t0 = __shfl_up_sync(full, v0, d), t1 = __shfl_up_sync(full, v1, d),
                t2 = __shfl_up_sync(full, v2, d);
    if (lane - d >= s0) v0 += t0;
    if (lane - d >= s1) v1 += t1;
    if (lane - d >= s2) v2 += t2;
  }
  const bool last = lane == 31;
  const bool e0 = k0 >= 0 && (last || ((h0 >> (lane + 1)) & 1u));
  const bool e1 = k1 >= 0 && (last || ((h1 >> (lane + 1)) & 1u));
  const bool e2 = k2 >= 0 && (last || ((h2 >> (lane + 1)) & 1u));
  warp_put_ordered(acc, k0, v0, e0, stage);
  warp_put_ordered(acc, k1, v1, e1, stage);
  warp_put_ordered(acc, k2, v2, e2, stage);
  __syncwarp();
}

// ---------------------------------------------------------------------------------------------
// Block reductions: every thread of the block receives the total. `sbuf` holds NT/32 values.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int NT, typename T>
__device__ __forceinline__ T block_sum(T v, T* sbuf) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = ((threadIdx.x & 31) < NT / 32) ? sbuf[threadIdx.x & 31] : T(0);
  return warp_sum(t);
}

// Sum of FP32 per-thread partials: FP32 within each warp, FP64 across the warps (NT / 32 - 1
// additions, read from shared memory by every thread), the same value in every thread.
template <int NT>
__device__ __forceinline__ double block_sum_f(float v, double* sbuf) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  double t = sbuf[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) t += sbuf[w];
  return t;
}

// Two block_sum_f at once (one pair of barriers); sbuf holds 2 NT / 32 doubles.
template <int NT>
__device__ __forceinline__ void block_sum2_f(float a, float b, double* sbuf, double& ra, double& rb) {
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sbuf[threadIdx.x >> 5] = (double)a;
    sbuf[NT / 32 + (threadIdx.x >> 5)] = (double)b;
  }
  __syncthreads();
  ra = sbuf[0];
  rb = sbuf[NT / 32];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) {
    ra += sbuf[w];
    rb += sbuf[NT / 32 + w];
  }
}

// Two sums at once (one pair of barriers).
template <int NT, typename T>
__device__ __forceinline__ void block_sum2(T& a, T& b, T* sbuf) {
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    sbuf[threadIdx.x >> 5] = a;
    sbuf[NT / 32 + (threadIdx.x >> 5)] = b;
  }
  __syncthreads();
  const int l = threadIdx.x & 31;
  T ta = (l < NT / 32) ? sbuf[l] : T(0);
  T tb = (l < NT / 32) ? sbuf[NT / 32 + l] : T(0);
  a = warp_sum(ta);
  b = warp_sum(tb);
}

template <int NT, typename T>
__device__ __forceinline__ T block_max(T v, T* sbuf) {
  v = warp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = ((threadIdx.x & 31) < NT / 32) ? sbuf[threadIdx.x & 31] : sbuf[0];
  return warp_max(t);
}

template <int NT, typename T>
__device__ __forceinline__ T block_min(T v, T* sbuf) {
  v = warp_min(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = ((threadIdx.x & 31) < NT / 32) ? sbuf[threadIdx.x & 31] : sbuf[0];
  return warp_min(t);
}

// ---------------------------------------------------------------------------------------------
// Separable noise N_p^-1 = w_p diag(n) (homogeneous: w_p = 1). The Gram-Schmidt factors of mgs3
// do not depend on w_p, so every pixel of a cell (equal labels) shares them, and in that basis the
// likelihood term of Eq. 3 is a sum of squared projections (no residual needs forming):
//   b^T M^-1 b = w_p sum_k <e_k, d>^2 / <c_k, c_k>_n,   e = n (1, c1, c2),
// while the gradient of Sec. 3.3.1 needs, per parameter with dA/dbeta = column j scaled by l,
//   r^T N dA s_hat = w_p s_hat_j (<v, d> - sum_k s_hat_k <v, a_k>),   v = n a_j l,  a = (1, A_d, A_s).
// run_scalars: the per-cell scalars (1/<c_k,c_k>, mu1, mu2, nu and the nine <v, a_k>) of one cell,
// by one thread, written as 16 floats: i0, i1, i2, mu1, mu2, nu, u[0..8], 0.
// ---------------------------------------------------------------------------------------------
constexpr int NSC = 15;  // i0, i1, i2, mu1, mu2, nu, u[9] with u[3 j + k] = <v_j, a_k>

__device__ __forceinline__ void load_row16(const float* __restrict__ r, float (&x)[NB]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = *reinterpret_cast<const float4*>(r + 4 * k);
    x[4 * k] = v.x; x[4 * k + 1] = v.y; x[4 * k + 2] = v.z; x[4 * k + 3] = v.w;
  }
}

template <bool GRAD>
__device__ __forceinline__ void run_scalars(const float* __restrict__ pd,
                                            const float* __restrict__ bt,
                                            const float* __restrict__ dt,
                                            const float* __restrict__ ss, const float* nband,
                                            const Bands& bc, float n0, float* out,
                                            float* vec = nullptr) {
  float ad[NB], as[NB];
  {
    float p[NB], b[NB];
    load_row16(pd, p);
    load_row16(bt, b);
    load_row16(ss, as);
#pragma unroll
    for (int f = 0; f < NB; ++f) ad[f] = p[f] * b[f];
  }
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    s1 = fmaf(nband[f], ad[f], s1);
    s2 = fmaf(nband[f], as[f], s2);
  }
  const float i0 = 1.f / n0, mu1 = s1 * i0, mu2 = s2 * i0;
  float n1 = 0.f, x12 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    const float c1 = ad[f] - mu1, w = nband[f] * c1;
    n1 = fmaf(w, c1, n1);
    x12 = fmaf(w, as[f], x12);
  }
  const float i1 = 1.f / n1, nu = x12 * i1;
  float n2 = 0.f;
#pragma unroll
  for (int f = 0; f < NB; ++f) {
    const float c2 = fmaf(-nu, ad[f] - mu1, as[f] - mu2);
    n2 = fmaf(nband[f] * c2, c2, n2);
  }
  const float i2 = 1.f / n2;
  float u[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (GRAD) {
    float d[NB];
    load_row16(dt, d);
#pragma unroll
    for (int f = 0; f < NB; ++f) {
      const float nad = nband[f] * ad[f], nas = nband[f] * as[f];
      const float vb = nad * bc.lnd[f], vt = nad * d[f], vs = nas * bc.lns[f];
      u[0] += vb; u[1] = fmaf(vb, ad[f], u[1]); u[2] = fmaf(vb, as[f], u[2]);
      u[3] += vt; u[4] = fmaf(vt, ad[f], u[4]); u[5] = fmaf(vt, as[f], u[5]);
      u[6] += vs; u[7] = fmaf(vs, ad[f], u[7]); u[8] = fmaf(vs, as[f], u[8]);
    }
  }
  float4* o = reinterpret_cast<float4*>(out);
  o[0] = make_float4(i0, i1, i2, mu1);
  o[1] = make_float4(mu2, nu, u[0], u[1]);
  o[2] = make_float4(u[2], u[3], u[4], u[5]);
  o[3] = make_float4(u[6], u[7], u[8], 0.f);
  if (vec) {
    // the run's band vectors (see cell_pixel): e1 = n c1, e2 = n c2 and, for the gradient,
    // n A_d ln(nu/nu0_d), n A_d dlnB/dT, n A_s ln(nu/nu0_s); [5][16] floats
    float d[NB];
    if (GRAD) load_row16(dt, d);
#pragma unroll
    for (int f = 0; f < NB; ++f) {
      const float n = nband[f];
      const float e1 = n * (ad[f] - mu1);
      vec[f] = e1;
      vec[NB + f] = fmaf(-nu, e1, n * (as[f] - mu2));
      if (GRAD) {
        const float nad = n * ad[f];
        vec[2 * NB + f] = nad * bc.lnd[f];
        vec[3 * NB + f] = nad * d[f];
        vec[4 * NB + f] = n * as[f] * bc.lns[f];
      }
    }
  }
}

// One pixel in its run's basis with the run's band vectors precomputed (run_scalars `vec`):
// the same quantities as cell_pixel, from 12 dot products over the bands.
template <bool GRAD>
__device__ __forceinline__ float cell_pixel_vec(const float (&dq)[NB], const float (&du)[NB],
                                                const float* nband, const float* vec,
                                                const float (&sc)[15], float w, float& gbd,
                                                float& gtd, float& gbs) {
  float t0q = 0.f, t1q = 0.f, t2q = 0.f, t0u = 0.f, t1u = 0.f, t2u = 0.f;
  float bq = 0.f, tq = 0.f, sq = 0.f, bu = 0.f, tu = 0.f, su = 0.f;
  const float4* v4 = reinterpret_cast<const float4*>(vec);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 e1 = v4[k], e2 = v4[4 + k];
    float4 vb, vt, vs;
    if (GRAD) {
      vb = v4[8 + k];
      vt = v4[12 + k];
      vs = v4[16 + k];
    }
    const float a1[4] = {e1.x, e1.y, e1.z, e1.w}, a2[4] = {e2.x, e2.y, e2.z, e2.w};
    float b1[4], b2[4], b3[4];
    if (GRAD) {
      b1[0] = vb.x; b1[1] = vb.y; b1[2] = vb.z; b1[3] = vb.w;
      b2[0] = vt.x; b2[1] = vt.y; b2[2] = vt.z; b2[3] = vt.w;
      b3[0] = vs.x; b3[1] = vs.y; b3[2] = vs.z; b3[3] = vs.w;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int f = 4 * k + c;
      const float xq = dq[f], xu = du[f];
      t0q = fmaf(nband[f], xq, t0q);
      t0u = fmaf(nband[f], xu, t0u);
      t1q = fmaf(a1[c], xq, t1q);
      t1u = fmaf(a1[c], xu, t1u);
      t2q = fmaf(a2[c], xq, t2q);
      t2u = fmaf(a2[c], xu, t2u);
      if (GRAD) {
        bq = fmaf(b1[c], xq, bq);
        bu = fmaf(b1[c], xu, bu);
        tq = fmaf(b2[c], xq, tq);
        tu = fmaf(b2[c], xu, tu);
        sq = fmaf(b3[c], xq, sq);
        su = fmaf(b3[c], xu, su);
      }
    }
  }
  const float i0 = sc[0], i1 = sc[1], i2 = sc[2], mu1 = sc[3], mu2 = sc[4], nu = sc[5];
  if (GRAD) {
    const float s2q = t2q * i2, s2u = t2u * i2;
    const float s1q = fmaf(-nu, s2q, t1q * i1), s1u = fmaf(-nu, s2u, t1u * i1);
    const float s0q = t0q * i0 - mu1 * s1q - mu2 * s2q;
    const float s0u = t0u * i0 - mu1 * s1u - mu2 * s2u;
    const float rbq = bq - (s0q * sc[6] + s1q * sc[7] + s2q * sc[8]);
    const float rbu = bu - (s0u * sc[6] + s1u * sc[7] + s2u * sc[8]);
    const float rtq = tq - (s0q * sc[9] + s1q * sc[10] + s2q * sc[11]);
    const float rtu = tu - (s0u * sc[9] + s1u * sc[10] + s2u * sc[11]);
    const float rsq = sq - (s0q * sc[12] + s1q * sc[13] + s2q * sc[14]);
    const float rsu = su - (s0u * sc[12] + s1u * sc[13] + s2u * sc[14]);
    const float m2w = -2.f * w;
    gbd = m2w * fmaf(s1q, rbq, s1u * rbu);
    gtd = m2w * fmaf(s1q, rtq, s1u * rtu);
    gbs = m2w * fmaf(s2q, rsq, s2u * rsu);
  }
  return -w * (i0 * fmaf(t0q, t0q, t0u * t0u) + i1 * fmaf(t1q, t1q, t1u * t1u) +
               i2 * fmaf(t2q, t2q, t2u * t2u));
}

__device__ __forceinline__ void load_scalars(const float* __restrict__ src, float (&sc)[NSC]) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  const float4 a = s4[0], b = s4[1], c = s4[2], d = s4[3];
  sc[0] = a.x; sc[1] = a.y; sc[2] = a.z; sc[3] = a.w;
  sc[4] = b.x; sc[5] = b.y; sc[6] = b.z; sc[7] = b.w;
  sc[8] = c.x; sc[9] = c.y; sc[10] = c.z; sc[11] = c.w;
  sc[12] = d.x; sc[13] = d.y; sc[14] = d.z;
}

// One pixel in its cell's basis (scalars from run_scalars, band vectors rebuilt from the SED
// table rows): L_p = -b^T M^-1 b summed over Q and U, and (GRAD) its contributions to dL/dbeta_d,
// dL/dT_d, dL/dbeta_s.
template <bool GRAD>
__device__ __forceinline__ float cell_pixel(const float (&dq)[NB], const float (&du)[NB],
                                            const float* __restrict__ pd,
                                            const float* __restrict__ bt,
                                            const float* __restrict__ dt,
                                            const float* __restrict__ ss, const float* nband,
                                            const Bands& bc, const float (&sc)[NSC], float w,
                                            float& gbd, float& gtd, float& gbs) {
  const float mu1 = sc[3], mu2 = sc[4], nu = sc[5];
  float t0q = 0.f, t1q = 0.f, t2q = 0.f, t0u = 0.f, t1u = 0.f, t2u = 0.f;
  float bq = 0.f, tq = 0.f, sq = 0.f, bu = 0.f, tu = 0.f, su = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 p4 = *reinterpret_cast<const float4*>(pd + 4 * k);
    const float4 b4 = *reinterpret_cast<const float4*>(bt + 4 * k);
    const float4 s4 = *reinterpret_cast<const float4*>(ss + 4 * k);
    float4 d4;
    if (GRAD) d4 = *reinterpret_cast<const float4*>(dt + 4 * k);
    const float pa[4] = {p4.x, p4.y, p4.z, p4.w}, ba[4] = {b4.x, b4.y, b4.z, b4.w},
                sa[4] = {s4.x, s4.y, s4.z, s4.w};
    float da[4] = {0.f, 0.f, 0.f, 0.f};
    if (GRAD) { da[0] = d4.x; da[1] = d4.y; da[2] = d4.z; da[3] = d4.w; }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int f = 4 * k + c;
      const float n = nband[f];
      const float ad = pa[c] * ba[c];
      const float nad = n * ad, nas = n * sa[c];
      const float e1 = fmaf(-mu1, n, nad);
      const float e2 = fmaf(-nu, e1, fmaf(-mu2, n, nas));
      const float xq = dq[f], xu = du[f];
      t0q = fmaf(n, xq, t0q);
      t0u = fmaf(n, xu, t0u);
      t1q = fmaf(e1, xq, t1q);
      t1u = fmaf(e1, xu, t1u);
      t2q = fmaf(e2, xq, t2q);
      t2u = fmaf(e2, xu, t2u);
      if (GRAD) {
        const float vb = nad * bc.lnd[f], vt = nad * da[c], vs = nas * bc.lns[f];
        bq = fmaf(vb, xq, bq);
        bu = fmaf(vb, xu, bu);
        tq = fmaf(vt, xq, tq);
        tu = fmaf(vt, xu, tu);
        sq = fmaf(vs, xq, sq);
        su = fmaf(vs, xu, su);
      }
    }
  }
  const float i0 = sc[0], i1 = sc[1], i2 = sc[2];
  if (GRAD) {
    const float s2q = t2q * i2, s2u = t2u * i2;
    const float s1q = fmaf(-nu, s2q, t1q * i1), s1u = fmaf(-nu, s2u, t1u * i1);
    const float s0q = t0q * i0 - mu1 * s1q - mu2 * s2q;
    const float s0u = t0u * i0 - mu1 * s1u - mu2 * s2u;
    const float rbq = bq - (s0q * sc[6] + s1q * sc[7] + s2q * sc[8]);
    const float rbu = bu - (s0u * sc[6] + s1u * sc[7] + s2u * sc[8]);
    const float rtq = tq - (s0q * sc[9] + s1q * sc[10] + s2q * sc[11]);
    const float rtu = tu - (s0u * sc[9] + s1u * sc[10] + s2u * sc[11]);
    const float rsq = sq - (s0q * sc[12] + s1q * sc[13] + s2q * sc[14]);
    const float rsu = su - (s0u * sc[12] + s1u * sc[13] + s2u * sc[14]);
    const float m2w = -2.f * w;
    gbd = m2w * fmaf(s1q, rbq, s1u * rbu);
    gtd = m2w * fmaf(s1q, rtq, s1u * rtu);
    gbs = m2w * fmaf(s2q, rsq, s2u * rsu);
  }
  return -w * (i0 * fmaf(t0q, t0q, t0u * t0u) + i1 * fmaf(t1q, t1q, t1u * t1u) +
               i2 * fmaf(t2q, t2q, t2u * t2u));
}

}  // namespace csx
