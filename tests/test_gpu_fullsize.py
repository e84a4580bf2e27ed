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
from tests._fitcheck import sampled_fit_check as _sampled_fit_check, stored_refs  # noqa: E402
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
    # the cell plan, as the bench times it (100 realizations in one call)
    plan = csx.SpectralPlan(labels[0], K)
    L3, g3 = plan.grad(model, sky, bt)
    torch.cuda.synchronize()
    plan.close()
    L1, L2, g = L1.cpu().numpy(), L2.cpu().numpy(), g.cpu().numpy()
    L3, g3 = L3.cpu().numpy(), g3.cpu().numpy()
    assert np.isfinite(L1).all() and np.isfinite(g).all() and np.isfinite(g3).all()
    for r in (0, 41, 99):
        Lr, gr, Sr = grad_ref(case, r, lab, K, beta[r].astype(np.float64))
        assert abs(L1[r] - Lr) <= 1e-5 * abs(Lr), (r, L1[r], Lr)
        assert abs(L2[r] - Lr) <= 1e-5 * abs(Lr)
        assert abs(L3[r] - Lr) <= 1e-5 * abs(Lr), (r, L3[r], Lr)
        assert_grad_close(g[r], gr, Sr)
        assert_grad_close(g3[r], gr, Sr)


def test_fullsky_nside64_fit_and_reconstruction(csx):
    """The full-sky nside-64 workload (K = (100, 20, 30), 100 realizations): one batched fit of all
    100 realizations, then W d at the fitted points. Two realizations against stored oracle fits
    (tests/golden/make_fit_refs.py, case fullsky64), and the reconstruction of one of them against
    the oracle's W d, sigma^2 and r_sys at the GPU's fitted point."""
    import os
    from oracle import reconstruct as rc
    from tests.golden import make_fit_refs as mk
    if not os.path.exists(os.path.join(os.path.dirname(mk.__file__), "fit_refs_fullsky64.npz")):
        pytest.skip("stored oracle fits of the full-sky case not written")
    wl = workloads.fullsky(64, (100, 20, 30), nreal=100)
    case = Case(wl, "separable")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(0) for _ in range(wl.nreal)]), device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0)
    fg = torch.from_numpy(case.fg32).to("cuda")
    out = csx.reconstruct(model, sky, labels, wl.K, res["beta"], d_fg=fg, s_hat=True, sigma2=True,
                          r_sys=True)
    torch.cuda.synchronize()
    assert (res["status"].cpu().numpy() == 0).all()
    picks, refs = stored_refs("fullsky64", case)
    _sampled_fit_check(csx, case, res, picks, max_alternative=0, refs=refs)
    P = int(wl.K[0].sum())
    q = picks[1]
    b = res["beta"].cpu().numpy()[q * P:(q + 1) * P].astype(np.float64)
    s = rc.reconstruct(case.nu, case.d64(q), case.ninv64, wl.labels[0], wl.K[0], b)
    sv = rc.stat_variance(case.nu, case.ninv64, wl.labels[0], wl.K[0], b)
    rs = rc.systematic_residual(case.nu, case.fg64(), case.ninv64, wl.labels[0], wl.K[0], b)
    np.testing.assert_allclose(out["s_hat"][q].cpu().numpy(), s, rtol=0, atol=1e-4 * np.abs(s).max())
    np.testing.assert_allclose(out["sigma2"][q].cpu().numpy(), sv, rtol=1e-4)
    np.testing.assert_allclose(out["r_sys"][q].cpu().numpy(), rs, rtol=0,
                               atol=1e-4 * np.abs(rs).max() + 1e-6)


def test_gradcheck_nside128_autograd_64_points(csx):
    """The differentiation check at nside 128 (196608 pixels, K = 256 per parameter, P = 768): the
    autograd function's gradient in FP32 and in all-FP64 at 64 random points against the FP64
    oracle at every point, and against central finite differences (step 1e-4) of the all-FP64
    likelihood on a subset of components. Only the gradient is kept between forward and backward."""
    from tests._oracle_jobs import grad_job, oracle_pool
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
    out = {}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        bt = torch.tensor(beta, device="cuda", dtype=dt, requires_grad=True)
        L = csx.SpectralLikelihood.apply(bt, model, sky, labels, K, prec)
        L.sum().backward()
        torch.cuda.synchronize()
        assert bt.grad.dtype == dt
        out[prec] = (L.detach().cpu().numpy(), bt.grad.cpu().numpy().astype(np.float64))
        assert np.isfinite(out[prec][0]).all() and np.isfinite(out[prec][1]).all()
    jobs = [(case.nu, case.d64(0), case.ninv64, lab, K, beta[i].astype(np.float64)) for i in range(64)]
    with oracle_pool(8) as pool:
        refs = pool.map(grad_job, jobs)
    worst32 = worst64 = 0.0
    ratio = 0.0
    for i, (Lr, gr, Sr, Sdr) in enumerate(refs):
        L32, g32 = out["fp32"][0][i], out["fp32"][1][i]
        L64, g64 = out["fp64"][0][i], out["fp64"][1][i]
        assert abs(L32 - Lr) <= 1e-5 * abs(Lr), (i, L32, Lr)
        ratio = max(ratio, assert_grad_close(g32, gr, Sr, Sdr)[1])
        assert abs(L64 - Lr) <= 1e-11 * abs(Lr), (i, L64, Lr)
        scale = np.abs(gr).max()
        assert np.abs(g64 - gr).max() <= 1e-9 * scale, (i, np.abs(g64 - gr).max() / scale)
        assert np.all(np.abs(g64 - gr) <= 1e-9 * np.abs(gr) + 1e-12 * Sr), i
        worst32 = max(worst32, np.abs(g32 - gr).max() / scale)
        worst64 = max(worst64, np.abs(g64 - gr).max() / scale)
    print("max-norm relative gradient error vs the oracle: FP32 %.2e, FP64 %.2e; largest FP32 "
          "component error / its bound %.3f" % (worst32, worst64, ratio))
    # central differences (h = 1e-4) of the all-FP64 likelihood at 4 points, 6 components each
    # (two per parameter type), all perturbed points in one call
    P = sum(K)
    comps = [0, 137, 256, 400, 512, 700]
    rows, where = [], []
    for i in (0, 21, 42, 63):
        for j in comps:
            for sgn in (1.0, -1.0):
                b = beta[i].astype(np.float64).copy()
                b[j] += sgn * 1e-4
                rows.append(b)
            where.append((i, j))
    d2 = torch.from_numpy(case.d32).to("cuda").repeat(len(rows), 1, 1, 1)
    sky2 = csx.Sky(d2, noise="separable", ninv_band=case.nb32,
                   w=torch.from_numpy(case.w32).to("cuda"))
    Lfd, _ = csx.spectral_grad_f64(model, sky2, labels, K, torch.tensor(np.array(rows), device="cuda"),
                                   want_grad=False)
    torch.cuda.synchronize()
    Lfd = Lfd.cpu().numpy()
    for k, (i, j) in enumerate(where):
        fd = (Lfd[2 * k] - Lfd[2 * k + 1]) / 2e-4
        g64, g32 = out["fp64"][1][i], out["fp32"][1][i]
        gmax = np.abs(g64).max()
        assert abs(g64[j] - fd) <= 1e-5 * abs(fd) + 1e-6 * gmax, (i, j, g64[j], fd)
        assert abs(g32[j] - fd) <= 1e-4 * abs(fd) + 1e-5 * gmax, (i, j, g32[j], fd)
    del d2, sky2
    assert P == 768


def test_bench_scan_fit_sampled_problems(csx):
    """The bench's workload and launch: every one of the 10000 problems in one persistent launch;
    nine problems spread over the scan's P range (six below 200, three from 600 to 1314) against
    stored oracle fits (tests/golden/make_fit_refs.py)."""
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
    picks, refs = stored_refs("scan64", case)
    print("sampled problems", picks, "P", P[picks].tolist())
    _sampled_fit_check(csx, case, res, picks, max_alternative=0, refs=refs)


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
    picks, refs = stored_refs("scan16_k1000", case)
    print("P", P[picks])
    # patches of one or two pixels at nside 16 leave some beta_s flat to ~1e-9 of chi2: up to 1% of
    # the parameters may sit at another optimum as good in FP64 (within 1e-6 chi2)
    _sampled_fit_check(csx, case, res, picks, max_alternative=0.01, refs=refs)


def test_pipeline_largest_p_sampled_problems(csx):
    """The two largest-P configurations of the full-pipeline scan (nside 64, |b| > 20 deg, K per
    parameter log-uniform up to 1000; P = 2589 and 2001, realization 0) fitted in one launch,
    against stored oracle fits (tests/golden/make_fit_refs.py, case pipeline64)."""
    import os
    from tests.golden import make_fit_refs as mk
    if not os.path.exists(os.path.join(os.path.dirname(mk.__file__), "fit_refs_pipeline64.npz")):
        pytest.skip("stored oracle fits of the pipeline case not written")
    wl = workloads.scan_subset([937, 1739], nside=64, nconf=4000, kmax=1000, nreal=1)
    case = Case(wl, "separable")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0)
    torch.cuda.synchronize()
    picks, refs = stored_refs("pipeline64", case)
    print("P", wl.P.tolist())
    # patches of ~12 pixels (P ~ 2600 over 32512 pixels): up to 1% of the parameters may sit at
    # another optimum as good in FP64 (within 1e-6 chi2)
    _sampled_fit_check(csx, case, res, picks, max_alternative=0.01, refs=refs)


def test_cell_moment_evaluation_nside64_scan(csx):
    """The fit's cell-moment evaluation of L and dL/dbeta at fixed points, on configurations of the
    bench's nside-64 scan (small, median and large P), against the oracle's pixel-by-pixel
    likelihood: at a point near the moments' reference point (10 tolerances away), at an
    independent random point, and at a point far from it (uniform inside the box, away from the
    bounds by 10% of their span), where the residual moments' rounding is largest. Tolerances of
    the parity tests."""
    from tests._oracle_jobs import grad_job, oracle_pool
    wl = workloads.scan(nside=64, nconf=1000, kmax=500, nreal=10, b_cut_deg=20.0, seed=4)
    case = Case(wl, "separable")
    model, sky, labels = case.gpu()
    order = np.argsort(wl.P, kind="stable")
    confs = [int(order[50]), int(order[len(order) // 2]), int(order[-1])]
    rng = np.random.default_rng(29)
    lo, hi = np.array(workloads.LOWER), np.array(workloads.UPPER)
    jobs, got = [], []
    for c in confs:
        K = wl.K[c]
        P = int(K.sum())
        types = np.concatenate([np.full(K[j], j) for j in range(3)])
        ref = workloads.random_points(K, 3, seed=100 + c)
        pts = np.empty_like(ref)
        pts[0] = ref[0] + 10 * TOL_BETA[types] * rng.standard_normal(P)
        pts[1] = workloads.random_points(K, 1, seed=200 + c)[0]
        span = hi - lo
        pts[2] = rng.uniform(lo[types] + 0.1 * span[types], hi[types] - 0.1 * span[types])
        Lg, g = csx.cell_like_grad(model, sky, labels[c], K, torch.tensor(ref, device="cuda"),
                                   torch.tensor(pts, device="cuda"))
        torch.cuda.synchronize()
        got.append((Lg.cpu().numpy(), g.cpu().numpy()))
        p32 = pts.astype(np.float32).astype(np.float64)
        for r in range(3):
            jobs.append((case.nu, case.d64(r), case.ninv64, wl.labels[c], K, p32[r]))
    with oracle_pool(8) as pool:
        refs = pool.map(grad_job, jobs)
    for k, c in enumerate(confs):
        for r in range(3):
            Lr, gr, Sr, Sdr = refs[3 * k + r]
            Lg, g = got[k][0][r], got[k][1][r]
            print("configuration %d (P %d) point %d: L rel err %.2e, grad max-norm rel err %.2e, "
                  "largest component error / bound %.3f, / 1e-5 S %.3f"
                  % (c, wl.P[c], r, abs(Lg - Lr) / abs(Lr), np.abs(g - gr).max() / np.abs(gr).max(),
                     (np.abs(g - gr) / (1e-4 * np.abs(gr) + np.maximum(1e-5 * Sr, 32 * 2.0 ** -24 * Sdr))).max(),
                     (np.abs(g - gr) / (1e-4 * np.abs(gr) + 1e-5 * Sr)).max()))
            assert abs(Lg - Lr) <= 1e-5 * abs(Lr), (c, r, Lg, Lr)
            assert_grad_close(g, gr, Sr, Sdr)
