"""Oracle: the AdaTopK optimiser of App. A, step by step, in FP64 (test infrastructure only).

App. A works in the internal space y = (x - l) / (u - l) in [0, 1] ("Internal Parameter Space"),
keeps a pivot p_i in {-1, 0, 1} (at the lower bound, free, at the upper bound), releases bound
constraints by a score ("Top-K Release Strategy"), projects the gradient onto the free set, rescales
the objective and the AdaBelief moments when the projected gradient norm leaves a safe range
("Dynamic State Rescaling"), takes an AdaBelief direction masked to the free set, limits the step by
the distance to the nearest bound and runs a backtracking line search; a step that reaches the
bound clamps the limiting parameter and pins it (Algorithm "AdaTopK Optimization Step").

Readings where App. A is silent or garbled (the CUDA path applies the same ones):
  - release score: the text defines it as the alignment of -g with the feasible direction into the
    box, which is -p_i at a bound, i.e. score_i = p_i * g_int_i; the printed formula p_i * (-g_int_i)
    has the opposite sign and would release the constraints the gradient pushes outward.
  - Top-K fraction K: the number released is max(1, floor(K * n)) of the n positive scores
    (K = 0: the single highest, as TNC; K = 1: all); ties to the lowest index.
  - AdaBelief (Zhuang et al. 2020) with its reference defaults beta1 = 0.9, beta2 = 0.999,
    eps = 1e-16, bias-corrected; the learning rate is the line search's step alpha.
  - line search: backtracking from alpha = min(eta, alpha_max), halving, Armijo c1 = 1e-4 on the
    (scaled) objective, a trial also accepted when its value exceeds f by at most eps_rel |f| and the
    slope g(y_trial).d is still downhill (eps_rel = 1e-5, the resolution of an FP32 likelihood in the
    residual-moment form; the same rule in both paths); eta starts at 0.1 (internal units) and becomes min(1, 2 alpha) after an
    accepted step. When the direction is not a descent direction or the search fails, the AdaBelief
    state is reset and the normalised projected steepest descent -g / |g|_inf is tried once.
  - stop: no positive release score, the largest accepted step below a threshold on two
    consecutive iterations and, where a curvature function is given (`fit`: the Gauss-Newton
    diagonal, evaluated at the candidate point), every free parameter's Newton-step estimate
    |g_i| / H_i below its xtol (a first-order step can be short while the optimum is still far); a
    candidate that fails this restarts the AdaBelief moments; else max_iter. A first-order step in an ill-conditioned valley (dust
    beta_d and T_d) is orders of magnitude shorter than the remaining distance, so `fit` sets the
    threshold to 0.003 xtol (physical units): with it the plain nside-8 fit, from the stated start
    and from every parameter on a bound, lands within 0.1 of the parity tolerances of the L-BFGS-B
    optimum.
  - pivots start from the start point: p_i = -1 where y_i <= 0, +1 where y_i >= 1.
  - the direction is also zeroed where a free parameter sits on a bound and d points out of the box
    (a just-released parameter whose AdaBelief momentum still points outward would otherwise make
    the step limit zero for every parameter); eta is kept after a zero-length step.

Parity pins (tests/test_oracle_adatopk.py): the Top-K release rule on hand-made pivots and scores
(K = 0 frees the single highest, K = 1 all, ties to the lowest index); a separable box quadratic
reaches clip(c, 0, 1) (the closed-form minimiser, two coordinates on bounds); a start with every
coordinate on a bound is released where the gradient points inward; rescaling the objective by
1e20 leaves the minimiser unchanged; on the plain nside-8 sky the fit lands on scipy's L-BFGS-B
optimum (a library routine) within the parity tolerances.
"""
from __future__ import annotations

import numpy as np

from .fit import expand_bounds
from .likelihood import data_norm, gauss_newton_diagonal, spectral_gradient

SAFE = (1e-15, 1e15)
STEP_FACTOR = 0.003  # stop threshold on the step, in units of xtol


def release(p, g_int, topk):
    """Pivots after the Top-K release: of the constrained parameters whose score p_i * g_i is
    positive, the max(1, floor(topk * n)) highest are freed (ties to the lowest index)."""
    p = p.copy()
    score = p * g_int
    cand = np.nonzero((p != 0) & (score > 0))[0]
    if cand.size == 0:
        return p, 0
    n = max(1, int(np.floor(topk * cand.size)))
    order = cand[np.lexsort((cand, -score[cand]))]  # highest score first, then lowest index
    p[order[:n]] = 0
    return p, n


def adabelief(g, m, s, t, beta1=0.9, beta2=0.999, eps=1e-16):
    """One AdaBelief update of the moments; returns (direction, m, s) with d = -m_hat/(sqrt(s_hat)+eps)."""
    m = beta1 * m + (1.0 - beta1) * g
    s = beta2 * s + (1.0 - beta2) * (g - m) ** 2 + eps
    mh = m / (1.0 - beta1 ** t)
    sh = s / (1.0 - beta2 ** t)
    return -mh / (np.sqrt(sh) + eps), m, s


def minimize(fun, y0, xtol_int, topk=0.0, max_iter=2000, max_ls=20, eta0=0.1, c1=1e-4,
             beta1=0.9, beta2=0.999, eps=1e-16, safe=SAFE, eps_rel=1e-5, gtol_int=None,
             trace=None):
    """AdaTopK on f(y), y in [0, 1]^P; fun(y) -> (f, grad). xtol_int: per-parameter step tolerance
    in internal units; gtol_int (optional): y -> per-parameter bound on the unscaled internal
    gradient of the free parameters at a candidate stop. Returns (y, f, info)."""
    y = np.clip(np.asarray(y0, dtype=np.float64), 0.0, 1.0)
    p = np.where(y <= 0.0, -1, np.where(y >= 1.0, 1, 0)).astype(np.int64)
    m = np.zeros_like(y)
    s = np.zeros_like(y)
    t = 0
    scale = 1.0
    eta = eta0
    f, g = fun(y)
    f, g = scale * f, scale * g
    nev, small, status, it = 1, 0, 1, 0
    for it in range(max_iter):
        p, nrel = release(p, g, topk)
        free = p == 0
        gp = np.where(free, g, 0.0)
        gn = np.linalg.norm(gp)
        if gn > 0.0 and (gn < safe[0] or gn > safe[1]):
            fs = 1.0 / gn
            scale *= fs
            f, g, gp, m, s = f * fs, g * fs, gp * fs, m * fs, s * fs * fs
        if nrel == 0 and not np.any(gp):
            status = 0  # no free direction and nothing to release
            break
        t += 1
        d, m, s = adabelief(gp, m, s, t, beta1, beta2, eps)
        d = np.where(free & ~((y <= 0.0) & (d < 0)) & ~((y >= 1.0) & (d > 0)), d, 0.0)
        slope = float(gp @ d)
        accepted = False
        for attempt in range(2):
            if attempt == 1 or not slope < 0.0:
                # restart: reset the AdaBelief state, normalised projected steepest descent
                m[:] = 0.0
                s[:] = 0.0
                t = 0
                gmax = np.abs(gp).max()
                if gmax == 0.0:
                    break
                d = -gp / gmax
                d = np.where(((y <= 0.0) & (d < 0)) | ((y >= 1.0) & (d > 0)), 0.0, d)
                slope = float(gp @ d)
            with np.errstate(divide="ignore", invalid="ignore"):
                lim = np.where(d < 0, -y / d, np.where(d > 0, (1.0 - y) / d, np.inf))
            j = int(np.argmin(lim))
            amax = float(lim[j])
            alpha = min(eta, amax)
            for _ in range(max_ls):
                yt = np.clip(y + alpha * d, 0.0, 1.0)
                if alpha == amax:
                    yt[j] = 0.0 if d[j] < 0 else 1.0
                ft, gt = fun(yt)
                ft, gt = scale * ft, scale * gt
                nev += 1
                if ft <= f + c1 * alpha * slope or (ft <= f + eps_rel * abs(f) and gt @ d <= 0.0):
                    accepted = True
                    break
                alpha *= 0.5
            if accepted:
                break
        if not accepted:
            status = 3
            break
        if trace is not None:
            trace.append(yt.copy())
        if alpha == amax:
            p[j] = -1 if d[j] < 0 else 1
        step = np.abs(yt - y) / xtol_int
        y, f, g = yt, ft, gt
        if alpha > 0.0:
            eta = min(1.0, 2.0 * alpha)
        small = small + 1 if step.max() <= 1.0 else 0
        if small >= 2 and not np.any((p != 0) & (p * g > 0)):
            if gtol_int is None:
                status = 0
                break
            gt_ = gtol_int(y)
            nev += 1
            if np.all(np.abs(g[p == 0]) / scale <= gt_[p == 0]):
                status = 0
                break
            small = 0  # still far along some parameter: restart the AdaBelief moments
            m[:] = 0.0
            s[:] = 0.0
            t = 0
    return y, f / scale, {"status": status, "iters": it + 1, "nev": nev, "scale": scale}


def fit(nu, d, ninv, labels, K, beta0, lower, upper, xtol=(1e-4, 1e-3, 1e-4), topk=0.0,
        max_iter=5000):
    """AdaTopK fit of one configuration (Eq. 7) on chi2_min = L + sum d^T N d. Returns
    (beta_hat [P], L(beta_hat), info)."""
    lo, hi = expand_bounds(K, lower, upper)
    sc = hi - lo
    dn = data_norm(d, ninv)
    xt = np.concatenate([np.full(int(K[j]), xtol[j], dtype=np.float64) for j in range(3)])

    def fun(y):
        L, g = spectral_gradient(nu, d, ninv, labels, K, lo + sc * y)
        return L + dn, g * sc

    y0 = np.clip((np.asarray(beta0, np.float64) - lo) / sc, 0.0, 1.0)
    gtol = lambda y: xt * sc * gauss_newton_diagonal(nu, d, ninv, labels, K, lo + sc * y)
    y, _, info = minimize(fun, y0, STEP_FACTOR * xt / sc, topk=topk, max_iter=max_iter,
                          gtol_int=gtol)
    x = lo + sc * y
    L, _ = spectral_gradient(nu, d, ninv, labels, K, x)
    return x, L, info
