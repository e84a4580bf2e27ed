"""Parity at the workloads' full sizes, in the launch configurations the bench uses, on outputs the
oracle computes one by one (sampled problems / points). Tolerances as in test_gpu_parity.

  - full sky nside 64, K = (100, 20, 30), 100 realizations in one streaming call (the bench's
    streaming-kernel configuration): L and dL/dbeta of sampled problems;
  - nside 128, K = 256 per parameter, 64 random beta points, through the autograd function: L and
    dL/dbeta at sampled points;
  - the bench's scan (nside 64, 1000 configurations x 10 realizations) fitted in one launch:
    sampled problems against oracle fits;
  - the large-K scan shape (K per parameter up to 1000, P up to ~3000) at nside 16: sampled fits.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
os.environ.setdefault("CSX_KMEANS_CACHE", os.path.join(ROOT, ".cache", "kmeans"))

from synth import workloads  # noqa: E402
from tests._inputs import Case, pack  # noqa: E402
from tests._fitcheck import sampled_fit_check as _sampled_fit_check  # noqa: E402
from tests._parity import TOL_BETA, assert_grad_close, grad_ref  # noqa: E402


@pytest.fixture(scope="module")
def csx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08463_b300 import csx as mod
    mod.lib()
    return mod


def test_fullsky_nside64_hundred_realizations(csx):
    K = (100, 20, 30)
    case = Case(workloads.fullsky(64, K, nreal=100), "separable")
    model, sky, labels = case.gpu()
    lab = case.wl.labels[0]
    beta = workloads.random_points(np.array(K), 100, seed=7).astype(np.float32)
    bt = torch.tensor(beta, device="cuda")
    L1 = csx.spectral_like(model, sky, labels[0], K, bt)
    L2, g = csx.spectral_grad(model, sky, labels[0], K, bt)
    torch.cuda.synchronize()
    L1, L2, g = L1.cpu().numpy(), L2.cpu().numpy(), g.cpu().numpy()
    assert np.isfinite(L1).all() and np.isfinite(g).all()
    for r in (0, 41, 99):
        Lr, gr, Sr = grad_ref(case, r, lab, K, beta[r].astype(np.float64))
        assert abs(L1[r] - Lr) <= 1e-5 * abs(Lr), (r, L1[r], Lr)
        assert abs(L2[r] - Lr) <= 1e-5 * abs(Lr)
        assert_grad_close(g[r], gr, Sr)


def test_gradcheck_nside128_autograd_64_points(csx):
    K = (256, 256, 256)
    wl = workloads.gradcheck(128, K, npoints=64)
    case = Case(wl, "separable")
    lab = wl.labels[0]
    beta = workloads.random_points(np.array(K), 64, seed=3).astype(np.float32)
    d = torch.from_numpy(case.d32).to("cuda").repeat(64, 1, 1, 1)  # one data set, 64 points
    sky = csx.Sky(d, noise="separable", ninv_band=case.nb32,
                  w=torch.from_numpy(case.w32).to("cuda"))
    model = csx.Model(case.nu)
    labels = torch.from_numpy(np.ascontiguousarray(lab)).to("cuda")
    bt = torch.tensor(beta, device="cuda", requires_grad=True)
    L = csx.SpectralLikelihood.apply(bt, model, sky, labels, K)
    L.sum().backward()
    torch.cuda.synchronize()
    Lg, g = L.detach().cpu().numpy(), bt.grad.cpu().numpy()
    assert np.isfinite(Lg).all() and np.isfinite(g).all()
    for i in (0, 9, 31, 63):
        Lr, gr, Sr = grad_ref(case, 0, lab, K, beta[i].astype(np.float64))
        assert abs(Lg[i] - Lr) <= 1e-5 * abs(Lr), (i, Lg[i], Lr)
        assert_grad_close(g[i], gr, Sr)


def test_bench_scan_fit_sampled_problems(csx):
    """The bench's workload and launch: every one of the 10000 problems in one persistent launch;
    six problems (P spread over the scan's lower half, where oracle fits take seconds) are refitted
    by the oracle."""
    wl = workloads.scan(nside=64, nconf=1000, kmax=500, nreal=10, b_cut_deg=20.0, seed=4)
    case = Case(wl, "separable")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0)
    torch.cuda.synchronize()
    status = res["status"].cpu().numpy()
    assert (status == 0).mean() >= 0.999, np.bincount(status)
    P = np.repeat(wl.P, wl.nreal)
    rng = np.random.default_rng(17)
    picks = []
    for lo, hi in ((3, 20), (20, 50), (50, 80), (80, 120), (120, 160), (160, 200)):
        cand = np.nonzero((P >= lo) & (P < hi))[0]
        picks.append(int(rng.choice(cand)))
    worst, floored, vfl, unc, jt = _sampled_fit_check(csx, case, res, picks)
    print("worst |err|/tol %.3f; within the gradient floor: %d; value floor: %d; unconstrained: %d; "
          "joint: %d" % (worst, floored, vfl, unc, jt))


def test_large_k_scan_nside16_sampled_problems(csx):
    """The large-K shape of the full-pipeline workload (K per parameter log-uniform up to 1000, so P
    reaches thousands and patches hold one or a few pixels) on a small sky."""
    wl = workloads.scan(nside=16, nconf=6, kmax=1000, nreal=2, b_cut_deg=20.0, seed=8)
    case = Case(wl, "separable")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0)
    torch.cuda.synchronize()
    P = np.repeat(wl.P, wl.nreal)
    order = np.argsort(P)
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    worst, floored, vfl, unc, jt = _sampled_fit_check(csx, case, res, picks)
    print("P", P[picks], "worst |err|/tol %.3f; within the gradient floor: %d; value floor: %d; "
          "unconstrained: %d; joint: %d" % (worst, floored, vfl, unc, jt))
