"""Oracle: the per-configuration fit beta* = argmin L(beta) in a box (Eq. 7, Sec. 3.3).

The paper maximises the spectral likelihood (Eq. 7) with quasi-Newton / AdaTopK optimisers inside
box bounds, working in the internal space y = (x - l) / (u - l) in [0, 1] (App. A, "Internal Parameter
Space"). The oracle's *result* is the local minimiser reached from the stated start point; its path
does not matter. It is computed with scipy's L-BFGS-B (the library routine) on chi2_min(beta) =
L(beta) + sum d^T N^-1 d with the analytic gradient, run to machine precision (ftol = 0), then
polished: first by Gauss-Newton steps (the Gauss-Newton Hessian of the profiled chi2,
likelihood.gauss_newton_hessian, solved against the gradient on the free parameters, the step
clipped to the box and halved until chi2 does not increase), then by Newton steps with the exact
Hessian (central differences of the analytic gradient), which converge quadratically also along the
nearly flat directions where L-BFGS-B stalls and the Gauss-Newton model, lacking the residual's
curvature, converges slowly. The fixed point of both is a zero of the free gradient, so the result
is the minimiser to FP64 precision.

Parity pins: brute-force grid minimum on tiny skies, recovery of the true beta for noise-free data
and for piecewise-constant truths as the noise goes to zero, a stationary point with a positive
definite Hessian.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

from .likelihood import data_norm, gauss_newton_hessian, spectral_gradient


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
    x = lo + scale * y
    if polish:
        x, info["polished"] = gauss_newton_polish(nu, d, ninv, labels, K, x, lo, hi)
        x, info["newton"] = newton_polish(nu, d, ninv, labels, K, x, lo, hi)
    L, g = spectral_gradient(nu, d, ninv, labels, K, x)
    info["grad"] = g
    yy = (x - lo) / scale
    info["interior"] = (yy > 1e-9) & (yy < 1.0 - 1e-9)
    return x, L, info


def gauss_newton_polish(nu, d, ninv, labels, K, x, lo, hi, steps=40):
    """Gauss-Newton steps from x towards the local minimiser in the box [lo, hi]. Free parameters:
    inside the box, or on a bound with the gradient pointing into it. Each step solves
    H_free delta = -g_free (least squares if H_free is singular), is clipped to the box and halved
    until chi2 does not increase; the polish stops when a step moves no parameter by more than
    1e-13 of its box, when no decrease is found, or after `steps`. Returns (x, steps taken)."""
    dn = data_norm(d, ninv)
    L, g = spectral_gradient(nu, d, ninv, labels, K, x)
    f = L + dn
    done = 0
    for _ in range(steps):
        pinned = ((x <= lo) & (g > 0)) | ((x >= hi) & (g < 0))
        free = np.nonzero(~pinned)[0]
        if free.size == 0:
            break
        H = gauss_newton_hessian(nu, d, ninv, labels, K, x)[np.ix_(free, free)]
        try:
            step = -np.linalg.solve(H, g[free])
        except np.linalg.LinAlgError:
            step = -np.linalg.lstsq(H, g[free], rcond=None)[0]
        x, f, g, moved = _descend(nu, d, ninv, labels, K, x, f, free, step, lo, hi, dn)
        if moved is None:
            break
        done += 1
        if moved.max() <= 1e-13:
            break
    return x, done


def newton_polish(nu, d, ninv, labels, K, x, lo, hi, steps=4, h_rel=1e-6):
    """Newton steps with the exact Hessian of chi2 on the free parameters, formed by central
    differences of the analytic gradient (step h_rel of each parameter's box, symmetrised), clipped
    to the box and halved until chi2 does not increase; after the Gauss-Newton steps, whose model
    lacks the curvature carried by the residual, these converge quadratically also along nearly
    flat directions. Stops when a step moves no parameter by more than 1e-13 of its box."""
    dn = data_norm(d, ninv)
    L, g = spectral_gradient(nu, d, ninv, labels, K, x)
    f = L + dn
    done = 0
    for _ in range(steps):
        pinned = ((x <= lo) & (g > 0)) | ((x >= hi) & (g < 0))
        free = np.nonzero(~pinned)[0]
        if free.size == 0:
            break
        H = np.empty((free.size, free.size))
        for a, i in enumerate(free):
            h = h_rel * (hi[i] - lo[i])
            xp, xm = x.copy(), x.copy()
            xp[i] += h
            xm[i] -= h
            H[:, a] = (spectral_gradient(nu, d, ninv, labels, K, xp)[1][free] -
                       spectral_gradient(nu, d, ninv, labels, K, xm)[1][free]) / (2.0 * h)
        H = 0.5 * (H + H.T)
        try:
            step = -np.linalg.solve(H, g[free])
        except np.linalg.LinAlgError:
            step = -np.linalg.lstsq(H, g[free], rcond=None)[0]
        x, f, g, moved = _descend(nu, d, ninv, labels, K, x, f, free, step, lo, hi, dn)
        if moved is None:
            break
        done += 1
        if moved.max() <= 1e-13:
            break
    return x, done


def _descend(nu, d, ninv, labels, K, x, f, free, step, lo, hi, dn):
    """x + t step on the free parameters, clipped to the box, t = 1, 1/2, ... until chi2 does not
    increase. Returns (x, chi2, gradient, relative move) or the inputs with move None."""
    t = 1.0
    for _ in range(60):
        xn = x.copy()
        xn[free] = np.clip(x[free] + t * step, lo[free], hi[free])
        Ln, gn = spectral_gradient(nu, d, ninv, labels, K, xn)
        if Ln + dn <= f:
            return xn, Ln + dn, gn, np.abs(xn - x) / (hi - lo)
        t *= 0.5
    return x, f, spectral_gradient(nu, d, ninv, labels, K, x)[1], None
