"""Oracle: reconstruction s_hat = W d and the residual diagnostics (Eqs. 3, 8-9, 10-11, 14-15).

  W_p = (A_p^T N_p^-1 A_p)^-1 A_p^T N_p^-1                    (Eq. 3 / Eq. 8)
  s_hat_p = W_p d_p                                           [npix, 2, 3]
  CMB unit response: [W A_cmb]_cmb = 1                         (Eq. 10)
  systematic residual: r_sys,p = [W_p d_fg,p]_cmb              (Eq. 15, in map space)
  statistical residual variance per pixel: [M_p^-1]_cmb,cmb    (the noise covariance of s_hat)
  map variance: Var_{p in mask}[s_hat_cmb,p]                   (Eq. 9; Q and U summed)

Per configuration c with realizations n, the selection score (reading recorded in the design
notes) is the total residual variance
  V_tot(c) = mean_n [ mean_{p,s} r_sys^2 + mean_p [M_p^-1]_00 ],
and the selected configuration is argmin_c V_tot (ties go to the lowest index).

Parity pins: W A = I, unit response, [W(d_fg + cmb)]_cmb - cmb = [W d_fg]_cmb, Monte-Carlo
variance of s_hat_cmb -> [M^-1]_00.
"""
from __future__ import annotations

import numpy as np

from .likelihood import pixel_mixing


def weights(A, ninv):
    """W [npix, 3, F]."""
    na = ninv[:, :, None] * A
    M = np.einsum("pfi,pfj->pij", A, na)
    return np.linalg.solve(M, np.transpose(na, (0, 2, 1)))


def reconstruct(nu, d, ninv, labels, K, beta):
    """s_hat [npix, 2, 3]."""
    W = weights(pixel_mixing(nu, beta, labels, K), ninv)
    return np.einsum("pcf,psf->psc", W, d)


def stat_variance(nu, ninv, labels, K, beta):
    """[M_p^-1]_00 [npix]."""
    A = pixel_mixing(nu, beta, labels, K)
    M = np.einsum("pfi,pf,pfj->pij", A, ninv, A)
    return np.linalg.inv(M)[:, 0, 0]


def systematic_residual(nu, d_fg, ninv, labels, K, beta):
    """[W d_fg]_cmb [npix, 2]."""
    W = weights(pixel_mixing(nu, beta, labels, K), ninv)
    return np.einsum("pf,psf->ps", W[:, 0, :], d_fg)


def map_variance(s_hat):
    """Eq. 9 summed over Q and U: sum_s Var_p[s_hat_cmb,p,s]."""
    return float(np.sum(np.var(s_hat[:, :, 0], axis=0)))


def problem_metrics(nu, d, d_fg, ninv, labels, K, beta):
    """Per-problem sums used for the selection: dict of float64."""
    s = reconstruct(nu, d, ninv, labels, K, beta)
    rs = systematic_residual(nu, d_fg, ninv, labels, K, beta)
    sv = stat_variance(nu, ninv, labels, K, beta)
    cq, cu = s[:, 0, 0], s[:, 1, 0]
    return {
        "sys_sq": float(np.sum(rs ** 2)),
        "stat": float(np.sum(sv)),
        "cmb_q_sum": float(np.sum(cq)), "cmb_q_sumsq": float(np.sum(cq ** 2)),
        "cmb_u_sum": float(np.sum(cu)), "cmb_u_sumsq": float(np.sum(cu ** 2)),
    }


def total_residual_variance(metrics, npix):
    """metrics: list over configurations of lists over realizations of problem_metrics dicts.
    Returns (V_tot [C], argmin)."""
    v = np.array([np.mean([m["sys_sq"] / (2.0 * npix) + m["stat"] / npix for m in reals])
                  for reals in metrics])
    return v, int(np.argmin(v))
