"""Comparison helpers shared by the parity tests (tolerances stated in test_gpu_parity)."""
import numpy as np

from oracle import likelihood as lk

TOL_BETA = np.array([1e-3, 1e-2, 1e-3])


U32 = 2.0 ** -24  # unit roundoff of FP32


def assert_grad_close(g, r, S, Sd=None):
    """dL/dbeta of an FP32 evaluation against the oracle's: max-norm relative 1e-4 (the stated
    tolerance), and per component |g_i - r_i| <= 1e-4 |r_i| + max(1e-5 S_i, 32 u Sd_i), u = 2^-24.
    S_i sums the magnitudes of the terms whose signed sum is dL/dbeta_i (residual scale); Sd_i the
    same with N d in place of the residual N (d - A s_hat): forming a residual from the data in FP32
    rounds each band's term by about u |N d| (dot products over the 15 bands, a few roundings each),
    so a component that is a small remainder of terms carries an error of order u Sd_i.
    Returns (max-norm relative error, largest per-component ratio to the bound)."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    scale = np.abs(r).max()
    err = np.abs(g - r)
    assert err.max() <= 1e-4 * scale, (err.max() / scale)
    floor = 1e-5 * np.asarray(S, np.float64)
    if Sd is not None:
        floor = np.maximum(floor, 32 * U32 * np.asarray(Sd, np.float64))
    bound = 1e-4 * np.abs(r) + floor
    bad = err > bound
    assert not bad.any(), (np.nonzero(bad)[0][:10], g[bad][:5], r[bad][:5], S[bad][:5])
    return err.max() / scale, (err / bound).max()


def grad_ref(case, r, lab, K, beta, d64=None, ninv=None, data_scale=False):
    d64 = case.d64(r) if d64 is None else d64
    ninv = case.ninv64 if ninv is None else ninv
    L, g = lk.spectral_gradient(case.nu, d64, ninv, lab, K, beta)
    S = lk.gradient_term_scale(case.nu, d64, ninv, lab, K, beta)
    if data_scale:
        return L, g, S, lk.gradient_term_scale(case.nu, d64, ninv, lab, K, beta, data_scale=True)
    return L, g, S
