"""Oracle: the per-configuration fit beta* = argmin L(beta) in a box (Eq. 7, Sec. 3.3).

The paper maximises the spectral likelihood (Eq. 7) with quasi-Newton / AdaTopK optimisers inside
box bounds, working in the internal space y = (x - l) / (u - l) in [0, 1] (App. A, "Internal Parameter
Space"). The oracle's *result* is the local minimiser reached from the stated start point; its path
does not matter. It is computed with scipy's L-BFGS-B (the library routine) on chi2_min(beta) =
L(beta) + sum d^T N^-1 d with the analytic gradient, run to machine precision (ftol = 0), then, for
P <= 300, polished by Newton steps whose Hessian is the central difference of the analytic gradient.

Parity pins: brute-force grid minimum on tiny skies, recovery of the true beta for noise-free data
and for piecewise-constant truths as the noise goes to zero.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

from .likelihood import data_norm, spectral_gradient


def expand_bounds(K, lower, upper):
    lo = np.concatenate([np.full(int(K[j]), lower[j], dtype=np.float64) for j in range(3)])
    hi = np.concatenate([np.full(int(K[j]), upper[j], dtype=np.float64) for j in range(3)])
    return lo, hi


def fit(nu, d, ninv, labels, K, beta0, lower, upper, polish=True, maxiter=20000):
    """Return (beta_hat [P], L(beta_hat), info dict)."""
    lo, hi = expand_bounds(K, lower, upper)
    scale = hi - lo
    dn = data_norm(d, ninv)

    def fun(y):
        x = lo + scale * y
        L, g = spectral_gradient(nu, d, ninv, labels, K, x)
        return L + dn, g * scale

    y0 = (np.asarray(beta0, dtype=np.float64) - lo) / scale
    res = minimize(fun, y0, jac=True, method="L-BFGS-B", bounds=[(0.0, 1.0)] * y0.size,
                   options=dict(maxiter=maxiter, maxfun=5 * maxiter, ftol=0.0, gtol=1e-14,
                                maxcor=20))
    y = np.clip(res.x, 0.0, 1.0)
    info = {"nit": int(res.nit), "nfev": int(res.nfev), "message": str(res.message),
            "polished": 0}
    if polish and y.size <= 300:
        y, info["polished"] = _newton_polish(fun, y)
    x = lo + scale * y
    L, g = spectral_gradient(nu, d, ninv, labels, K, x)
    info["grad"] = g
    info["interior"] = (y > 1e-9) & (y < 1.0 - 1e-9)
    return x, L, info


def _newton_polish(fun, y, steps=3, h=1e-6):
    """Newton steps on the interior coordinates with a central-difference Hessian of the gradient."""
    done = 0
    f, g = fun(y)
    for _ in range(steps):
        free = np.nonzero((y > 1e-9) & (y < 1.0 - 1e-9))[0]
        if free.size == 0:
            break
        H = np.empty((free.size, free.size))
        for a, i in enumerate(free):
            e = np.zeros_like(y)
            e[i] = h
            H[:, a] = (fun(y + e)[1][free] - fun(y - e)[1][free]) / (2 * h)
        H = 0.5 * (H + H.T)
        try:
            step = -np.linalg.solve(H, g[free])
        except np.linalg.LinAlgError:
            break
        yn = y.copy()
        yn[free] = np.clip(y[free] + step, 0.0, 1.0)
        fn, gn = fun(yn)
        if fn <= f + 1e-12 * abs(f) or np.linalg.norm(gn[free]) < np.linalg.norm(g[free]):
            y, f, g = yn, fn, gn
            done += 1
        else:
            break
    return y, done
