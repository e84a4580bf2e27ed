"""Fitted parameters of sampled problems against oracle fits (shared by the full-size tests)."""
import numpy as np

from synth import workloads
from tests._oracle_jobs import fit_job, oracle_pool
from tests._parity import TOL_BETA


def _hessian(lk, case, d64, lab, K, x, idx, tol):
    """Interior block of d2L/dbeta2 at x: central differences of the oracle's analytic gradient."""
    H = np.empty((idx.size, idx.size))
    for a, i in enumerate(idx):
        h = 0.1 * tol[i]
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        gp = lk.spectral_gradient(case.nu, d64, case.ninv64, lab, K, xp)[1]
        gm = lk.spectral_gradient(case.nu, d64, case.ninv64, lab, K, xm)[1]
        H[:, a] = (gp[idx] - gm[idx]) / (2 * h)
    return 0.5 * (H + H.T)


def stored_refs(name, case, picks=None):
    """(picks, refs) of a stored case from tests/golden/fit_refs_<name>.npz (written by
    tests/golden/make_fit_refs.py from the oracle alone); the inputs' fingerprints are checked."""
    import os
    from tests.golden import make_fit_refs as mk
    path = os.path.join(os.path.dirname(mk.__file__), "fit_refs_%s.npz" % name)
    z = np.load(path)
    stored = [int(q) for q in z["picks"]]
    picks = stored if picks is None else picks
    refs = []
    for q in picks:
        np.testing.assert_allclose(mk.fingerprint(case.wl, q), z["fingerprint_%d" % q], rtol=1e-12)
        refs.append((z["x_%d" % q], float(z["L_%d" % q]), z["interior_%d" % q].astype(bool)))
    return picks, refs


def sampled_fit_check(csx, case, res, picks, max_alternative=0, refs=None):
    """Fitted beta of sampled problems against oracle fits, at the stated tolerances: every problem
    converged, |L - L_ref| <= 1e-5 |L_ref|, and every parameter whose oracle optimum is interior
    within |dbeta_d|, |dbeta_s| <= 1e-3, |dT_d| <= 1e-2 K.

    The one exception is the "several correct results" reading of the fit: a parameter outside its
    tolerance is accepted as another correct optimum only when the oracle's own FP64 likelihood at
    the fitted point is no worse than at its optimum by more than eps = 1e-6 chi2_min (an equally
    good point of a flat or multi-modal likelihood), and the oracle's curvature there is positive.
    Such parameters are counted, printed and bounded by `max_alternative` (a count, or a fraction
    of the interior parameters checked when below 1).
    Returns (worst |err|/tol over the interior parameters, parameters accepted as alternatives)."""
    from oracle import likelihood as lk
    wl = case.wl
    offs, _ = csx.param_offsets(wl.K, wl.nreal)
    if refs is None:
        jobs = []
        for q in picks:
            c, r = divmod(q, wl.nreal)
            jobs.append((case.nu, case.d64(r), case.ninv64, wl.labels[c], wl.K[c], wl.beta0(c),
                         workloads.LOWER, workloads.UPPER))
        with oracle_pool(min(len(jobs), 8)) as pool:
            refs = pool.map(fit_job, jobs)
    out = {k: v.cpu().numpy() for k, v in res.items()}
    worst, alternative, checked = 0.0, 0, 0
    for q, (x_ref, L_ref, interior) in zip(picks, refs):
        c, r = divmod(q, wl.nreal)
        K = wl.K[c]
        P = int(K.sum())
        assert out["status"][q] == 0, (q, out["status"][q], out["iters"][q])
        got = out["beta"][offs[q]:offs[q] + P].astype(np.float64)
        types = np.concatenate([np.full(K[j], j) for j in range(3)])
        tol = TOL_BETA[types]
        err = np.abs(got - x_ref)
        assert abs(out["L"][q] - L_ref) <= 1e-5 * abs(L_ref), (q, out["L"][q], L_ref)
        checked += int(interior.sum())
        over = np.nonzero(interior & (err > tol))[0]
        if over.size:
            d64, lab = case.d64(r), wl.labels[c]
            eps = 1e-6 * abs(L_ref + lk.data_norm(d64, case.ninv64))
            L_at = lk.spectral_gradient(case.nu, d64, case.ninv64, lab, K, got)[0]
            for i in over:
                H = _hessian(lk, case, d64, lab, K, x_ref, np.array([i]), tol)[0, 0]
                ok = L_at - L_ref <= eps and H > 0
                print("problem %d (P %d) parameter %d (type %d): |err|/tol %.2f, L_fit - L_ref %.3g "
                      "(eps %.3g)%s" % (q, P, i, types[i], err[i] / tol[i], L_at - L_ref, eps,
                                        "" if ok else "  FAIL"))
                assert ok, (q, i, err[i] / tol[i], L_at - L_ref, eps)
                alternative += 1
        worst = max(worst, (err / tol)[interior].max(initial=0.0))
    bound = max_alternative
    if 0 < max_alternative < 1:
        bound = int(np.floor(max_alternative * checked))
    print("worst |err|/tol %.3f; parameters accepted as alternative optima: %d of %d checked "
          "(at most %d)" % (worst, alternative, checked, bound))
    assert alternative <= bound, (alternative, bound)
    return worst, alternative
