"""Comparison helpers shared by the parity tests (tolerances stated in test_gpu_parity)."""
import numpy as np

from oracle import likelihood as lk

TOL_BETA = np.array([1e-3, 1e-2, 1e-3])


def assert_grad_close(g, r, S):
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    scale = np.abs(r).max()
    assert np.abs(g - r).max() <= 1e-4 * scale, (np.abs(g - r).max() / scale)
    bad = np.abs(g - r) > 1e-4 * np.abs(r) + 1e-5 * S
    assert not bad.any(), (np.nonzero(bad)[0][:10], g[bad][:5], r[bad][:5], S[bad][:5])


def grad_ref(case, r, lab, K, beta, d64=None, ninv=None):
    d64 = case.d64(r) if d64 is None else d64
    ninv = case.ninv64 if ninv is None else ninv
    L, g = lk.spectral_gradient(case.nu, d64, ninv, lab, K, beta)
    return L, g, lk.gradient_term_scale(case.nu, d64, ninv, lab, K, beta)
