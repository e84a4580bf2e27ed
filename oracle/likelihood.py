"""Oracle: the clustered spectral likelihood and its gradient (Eqs. 1-4, Sec. 2.2, Sec. 3.3.1).

Data model (Eq. 1): d_p = A_p(beta_p) s_p + n_p with diagonal noise N_p; patches (Sec. 2.2): every
spectral parameter is constant over a patch, beta_p = beta_k for p in P_k, with one independent
labeling per parameter (beta_d, T_d, beta_s). Parameters are packed [beta_d (K_d) | T_d (K_T) |
beta_s (K_s)].

Per pixel and Stokes s in {Q, U}:  M_p = A_p^T N_p^-1 A_p,  b_{p,s} = A_p^T N_p^-1 d_{p,s},
  s_hat = M_p^-1 b (Eq. 3).
Likelihood (sign and normalisation read as the negative of twice the beta-dependent part of Eq. 4):
  L(beta) = - sum_p sum_s b_{p,s}^T M_p^-1 b_{p,s}.
Equivalently L = chi2_min - sum_p sum_s d^T N^-1 d with chi2_min = sum (d - A s_hat)^T N^-1 (d - A s_hat).

Gradient (Sec. 3.3.1): with w_r = N^-1 (d - A s_hat) and s held at s_hat (s_hat minimises the GLS
objective, so its variation drops out), the paper gives grad(sum b^T M^-1 b) = 2 w_r^T d(A s)/dbeta;
hence grad L = -2 sum_p sum_s w_r^T (dA/dbeta) s_hat, routed to the patch that owns each pixel.

Array conventions: d [npix, 2, F], ninv [npix, F] (diagonal of N_p^-1), labels int [3, npix],
K = (K_d, K_T, K_s), beta [P].

Parity pins: W A = I, textbook least squares, chi2 >= 0 with equality for noise-free data at the true
beta, central finite differences of L, Monte-Carlo variance of s_hat.
"""
from __future__ import annotations

import numpy as np

from .mixing import mixing_derivatives, mixing_matrix


def split_params(beta, K):
    kd, kt, ks = (int(k) for k in K)
    beta = np.asarray(beta, dtype=np.float64)
    assert beta.shape[-1] == kd + kt + ks
    return beta[..., :kd], beta[..., kd:kd + kt], beta[..., kd + kt:]


def pixel_parameters(beta, labels, K):
    """Patch model: per-pixel (beta_d, T_d, beta_s), each [npix]."""
    bd, td, bs = split_params(beta, K)
    return bd[labels[0]], td[labels[1]], bs[labels[2]]


def pixel_mixing(nu, beta, labels, K):
    """A_p for every pixel: [npix, F, 3]."""
    return mixing_matrix(nu, *pixel_parameters(beta, labels, K))


def normal_equations(A, ninv, d):
    """M [npix, 3, 3] and b [npix, 2, 3] (Eq. 3)."""
    na = ninv[:, :, None] * A
    M = np.einsum("pfi,pfj->pij", A, na)
    b = np.einsum("pfi,psf->psi", na, d)
    return M, b


def gls_components(A, ninv, d):
    """s_hat = M^-1 b per pixel and Stokes: [npix, 2, 3]."""
    M, b = normal_equations(A, ninv, d)
    return np.linalg.solve(M[:, None, :, :], b[..., None])[..., 0]


def spectral_likelihood(nu, d, ninv, labels, K, beta):
    """L(beta) = - sum_p sum_s b^T M^-1 b."""
    A = pixel_mixing(nu, beta, labels, K)
    M, b = normal_equations(A, ninv, d)
    s = np.linalg.solve(M[:, None, :, :], b[..., None])[..., 0]
    return -float(np.sum(b * s))


def data_norm(d, ninv):
    """sum_p sum_s d^T N^-1 d (beta-independent)."""
    return float(np.sum(d * ninv[:, None, :] * d))


def chi2_min(nu, d, ninv, labels, K, beta):
    """sum_p sum_s (d - A s_hat)^T N^-1 (d - A s_hat)."""
    A = pixel_mixing(nu, beta, labels, K)
    s = gls_components(A, ninv, d)
    r = d - np.einsum("pfi,psi->psf", A, s)
    return float(np.sum(r * ninv[:, None, :] * r))


def spectral_gradient(nu, d, ninv, labels, K, beta):
    """(L, grad L) with grad L = -2 sum_p sum_s w_r^T (dA/dbeta) s_hat (Sec. 3.3.1)."""
    kd, kt, ks = (int(k) for k in K)
    bd, td, bs = pixel_parameters(beta, labels, K)
    A = mixing_matrix(nu, bd, td, bs)
    dbd, dtd, dbs = mixing_derivatives(nu, bd, td, bs)
    M, b = normal_equations(A, ninv, d)
    s = np.linalg.solve(M[:, None, :, :], b[..., None])[..., 0]
    L = -float(np.sum(b * s))
    r = d - np.einsum("pfi,psi->psf", A, s)
    wr = ninv[:, None, :] * r
    # d(A s)/d theta for the pixel's own patch parameter: only one column of A depends on theta.
    g_bd = -2.0 * np.einsum("psf,pf,ps->p", wr, dbd, s[:, :, 1])
    g_td = -2.0 * np.einsum("psf,pf,ps->p", wr, dtd, s[:, :, 1])
    g_bs = -2.0 * np.einsum("psf,pf,ps->p", wr, dbs, s[:, :, 2])
    grad = np.concatenate([
        np.bincount(labels[0], weights=g_bd, minlength=kd),
        np.bincount(labels[1], weights=g_td, minlength=kt),
        np.bincount(labels[2], weights=g_bs, minlength=ks),
    ])
    return L, grad


def gauss_newton_diagonal(nu, d, ninv, labels, K, beta):
    """H_theta = 2 sum over the pixels of theta's patch and the Stokes parameters of
    s_hat_j^2 (dA_j/dtheta)^T N^-1 (dA_j/dtheta), j the column theta enters (the Gauss-Newton
    diagonal of chi2 without the projection onto the complement of A): a curvature scale per
    parameter, |dL/dtheta| / H_theta estimating the distance to the optimum along theta."""
    kd, kt, ks = (int(k) for k in K)
    bd, td, bs = pixel_parameters(beta, labels, K)
    A = mixing_matrix(nu, bd, td, bs)
    dbd, dtd, dbs = mixing_derivatives(nu, bd, td, bs)
    M, b = normal_equations(A, ninv, d)
    s = np.linalg.solve(M[:, None, :, :], b[..., None])[..., 0]
    s1 = (s[:, :, 1] ** 2).sum(axis=1)
    s2 = (s[:, :, 2] ** 2).sum(axis=1)
    h_bd = 2.0 * s1 * np.einsum("pf,pf,pf->p", ninv, dbd, dbd)
    h_td = 2.0 * s1 * np.einsum("pf,pf,pf->p", ninv, dtd, dtd)
    h_bs = 2.0 * s2 * np.einsum("pf,pf,pf->p", ninv, dbs, dbs)
    return np.concatenate([
        np.bincount(labels[0], weights=h_bd, minlength=kd),
        np.bincount(labels[1], weights=h_td, minlength=kt),
        np.bincount(labels[2], weights=h_bs, minlength=ks),
    ])


def gauss_newton_hessian(nu, d, ninv, labels, K, beta):
    """The Gauss-Newton Hessian [P, P] of chi2_min(beta) with the amplitudes profiled out (variable
    projection): H = 2 sum_p sum_s J^T N J, J[:, theta] = P_perp (dA/dtheta) s_hat, where
    P_perp = I - A M^-1 A^T N projects onto the N-orthogonal complement of the columns of A. Per
    pixel, with delta_theta the derivative column of theta (dust for beta_d and T_d, synchrotron for
    beta_s) and j(theta) the column it enters:
      H_p[theta, phi] = 2 (delta_theta^T N P_perp delta_phi) sum_s s_hat_j(theta) s_hat_j(phi),
    added at the pixel's own patch parameters. It is the Hessian itself where the residual
    d - A s_hat vanishes (the terms it drops are proportional to the residual)."""
    kd, kt, ks = (int(k) for k in K)
    bd, td, bs = pixel_parameters(beta, labels, K)
    A = mixing_matrix(nu, bd, td, bs)
    dbd, dtd, dbs = mixing_derivatives(nu, bd, td, bs)
    M, b = normal_equations(A, ninv, d)
    s = np.linalg.solve(M[:, None, :, :], b[..., None])[..., 0]
    delta = np.stack([dbd, dtd, dbs], axis=2)                       # [npix, F, 3]
    nd = ninv[:, :, None] * delta
    G = np.einsum("pfi,pfj->pij", delta, nd)                        # delta^T N delta
    AtNd = np.einsum("pfk,pfi->pki", A, nd)                          # A^T N delta  [npix, 3, 3]
    G = G - np.einsum("pki,pkl,plj->pij", AtNd, np.linalg.inv(M), AtNd)
    col = np.array([1, 1, 2])
    W = np.einsum("psi,psj->pij", s[:, :, col], s[:, :, col])       # sum_s s_j(theta) s_j(phi)
    Hp = 2.0 * G * W
    idx = np.stack([labels[0], kd + labels[1], kd + kt + labels[2]], axis=1)  # [npix, 3]
    P = kd + kt + ks
    H = np.zeros((P, P))
    for i in range(3):
        for j in range(3):
            np.add.at(H, (idx[:, i], idx[:, j]), Hp[:, i, j])
    return H


def gradient_term_scale(nu, d, ninv, labels, K, beta, data_scale=False):
    """S_theta = 2 sum over the pixels of theta's patch, the Stokes parameters and the bands of
    |w_r (dA/dtheta) s_hat| : the summed magnitude of the terms whose signed sum is dL/dtheta.
    A finite-precision evaluation of dL/dtheta carries an error proportional to S_theta, however
    small the signed sum is.

    data_scale=True replaces |w_r| = |N^-1 (d - A s_hat)| by |N^-1 d|: the scale of the rounding
    made when the residual d - A s_hat is formed in finite precision (relative error u |d| / |r|)."""
    kd, kt, ks = (int(k) for k in K)
    bd, td, bs = pixel_parameters(beta, labels, K)
    A = mixing_matrix(nu, bd, td, bs)
    dbd, dtd, dbs = mixing_derivatives(nu, bd, td, bs)
    M, b = normal_equations(A, ninv, d)
    s = np.linalg.solve(M[:, None, :, :], b[..., None])[..., 0]
    wr = ninv[:, None, :] * (d if data_scale else d - np.einsum("pfi,psi->psf", A, s))
    t_bd = 2.0 * np.abs(np.einsum("psf,pf,ps->psf", wr, dbd, s[:, :, 1])).sum(axis=(1, 2))
    t_td = 2.0 * np.abs(np.einsum("psf,pf,ps->psf", wr, dtd, s[:, :, 1])).sum(axis=(1, 2))
    t_bs = 2.0 * np.abs(np.einsum("psf,pf,ps->psf", wr, dbs, s[:, :, 2])).sum(axis=(1, 2))
    return np.concatenate([np.bincount(labels[0], weights=t_bd, minlength=kd),
                           np.bincount(labels[1], weights=t_td, minlength=kt),
                           np.bincount(labels[2], weights=t_bs, minlength=ks)])


def ninv_from(ninv_band, w, npix):
    """Per-pixel diagonal N^-1 [npix, F] from per-band 1/sigma^2 and per-pixel weights (None = 1)."""
    ninv_band = np.asarray(ninv_band, dtype=np.float64)
    if w is None:
        return np.broadcast_to(ninv_band, (npix, ninv_band.size)).copy()
    return np.asarray(w, dtype=np.float64)[:, None] * ninv_band[None, :]
