"""Fitted parameters of sampled problems against oracle fits (shared by the full-size tests)."""
import numpy as np

from synth import workloads
from tests._oracle_jobs import fit_job, oracle_pool
from tests._parity import TOL_BETA

JOINT_MAX_P = 4000  # largest problem for which the full interior Hessian is formed


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


def sampled_fit_check(csx, case, res, picks):
    """Fitted beta of sampled problems against oracle fits. A parameter passes within its tolerance,
    or -- when the likelihood is nearly flat along it -- within its tolerance plus the FP32 gradient
    floor propagated through the curvature: |dbeta_i| <= tol_i + 1e-5 S_i / H_ii, with S_i the
    summed term magnitude of dL/dbeta_i (the per-component gradient bound of the parity tests) and
    H_ii the oracle's d2L/dbeta_i2 (central differences of its analytic gradient) at its optimum.
    Failing that, a parameter passes within its tolerance plus the resolution of the optimiser's
    value-based decisions, sqrt(2 eps / H_ii) with eps = 1e-6 |chi2| (the line search does not
    distinguish values closer than that), provided the oracle's FP64 likelihood at the fitted point
    is within eps of its optimum's (the FP32-accumulated L the fit reports is checked separately,
    to 1e-5 relative): an
    optimum equivalent to the oracle's in FP32 arithmetic. A parameter the data leave statistically
    unconstrained -- 1-sigma width sqrt(2 / H_ii) above 100 tolerances -- is counted and reported
    instead.

    Where parameters are coupled (many small dust-index patches sharing one temperature patch), the
    set of points within eps of the optimum reaches further along a coordinate than the
    one-coordinate width: its extent is sqrt(2 eps (H^-1)_ii). A parameter that fails the tests
    above then passes when the oracle's FP64 likelihood at the fitted point is within eps of its
    optimum's and |dbeta_i| <= tol_i + 2 sqrt(2 eps (H^-1)_ii) (both points inside that set), H the
    interior Hessian block (problems up to JOINT_MAX_P parameters). The counts of each case are
    returned: (worst |err|/tol, gradient-floored, value-floored, unconstrained, joint)."""
    from oracle import likelihood as lk
    wl = case.wl
    offs, _ = csx.param_offsets(wl.K, wl.nreal)
    jobs = []
    for q in picks:
        c, r = divmod(q, wl.nreal)
        jobs.append((case.nu, case.d64(r), case.ninv64, wl.labels[c], wl.K[c], wl.beta0(c),
                     workloads.LOWER, workloads.UPPER))
    with oracle_pool(len(jobs)) as pool:
        refs = pool.map(fit_job, jobs)
    out = {k: v.cpu().numpy() for k, v in res.items()}
    worst, floored, vfloored, unconstrained, joint = 0.0, 0, 0, 0, 0
    for q, (x_ref, L_ref, interior) in zip(picks, refs):
        c, r = divmod(q, wl.nreal)
        K = wl.K[c]
        P = int(K.sum())
        assert out["status"][q] == 0, (q, out["status"][q], out["iters"][q])
        got = out["beta"][offs[q]:offs[q] + P].astype(np.float64)
        types = np.concatenate([np.full(K[j], j) for j in range(3)])
        tol = TOL_BETA[types]
        err = np.abs(got - x_ref)
        over = np.nonzero(interior & (err > tol))[0]
        if over.size:
            d64, lab = case.d64(r), wl.labels[c]
            S = lk.gradient_term_scale(case.nu, d64, case.ninv64, lab, K, x_ref)
            eps = 1e-6 * abs(L_ref + lk.data_norm(d64, case.ninv64))
            L_at = lk.spectral_gradient(case.nu, d64, case.ninv64, lab, K, got)[0]
            rest = []
            for i in over:
                H = _hessian(lk, case, d64, lab, K, x_ref, np.array([i]), tol)[0, 0]
                assert H > 0, (q, i, H)
                if err[i] <= tol[i] + 1e-5 * S[i] / H:
                    floored += 1
                elif err[i] <= tol[i] + np.sqrt(2.0 * eps / H) and L_at - L_ref <= eps:
                    vfloored += 1
                elif np.sqrt(2.0 / H) > 100 * tol[i]:
                    unconstrained += 1
                    print("unconstrained: problem %d parameter %d (type %d) |err| %.2e, sigma %.3f"
                          % (q, i, types[i], err[i], np.sqrt(2.0 / H)))
                else:
                    rest.append(i)
            if rest:
                assert P <= JOINT_MAX_P, (q, P, rest)
                assert L_at - L_ref <= eps, (q, L_at - L_ref, eps)
                fr = np.nonzero(interior)[0]
                Hf = _hessian(lk, case, d64, lab, K, x_ref, fr, tol)
                hinv = np.diag(np.linalg.inv(Hf))
                pos = np.searchsorted(fr, rest)
                reach = tol[rest] + 2.0 * np.sqrt(2.0 * eps * hinv[pos])
                assert np.all(err[rest] <= reach), (q, P, rest, err[rest], reach)
                joint += len(rest)
        assert abs(out["L"][q] - L_ref) <= 1e-5 * abs(L_ref), (q, out["L"][q], L_ref)
        worst = max(worst, (err / tol)[interior].max(initial=0.0))
    return worst, floored, vfloored, unconstrained, joint
