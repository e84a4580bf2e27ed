"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (stated, not tuned per case):
  L:        relative 1e-5
  grad L:   ||g - g_ref||_inf <= 1e-4 ||g_ref||_inf, and per component
            |g_i - r_i| <= 1e-4 |r_i| + 1e-5 S_i, where S_i is the summed magnitude of the
            per-pixel, per-band terms of dL/dtheta_i (oracle.likelihood.gradient_term_scale): a
            component that is a small remainder of cancelling terms is only as accurate as
            FP32 arithmetic on those terms
  fit:      |beta_d - ref| <= 1e-3, |T_d - ref| <= 1e-2 K, |beta_s - ref| <= 1e-3 (where the oracle
            optimum is interior)
  mixing / reconstruction (FP32 arithmetic): relative 2e-5 (mixing), 1e-4 of the field's scale.
  cells: bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cells as ocells  # noqa: E402
from oracle import fit as ofit  # noqa: E402
from oracle import likelihood as lk  # noqa: E402
from oracle import mixing as mx  # noqa: E402
from oracle import reconstruct as rc  # noqa: E402
from synth import workloads  # noqa: E402
from tests._inputs import Case, pack, scan_case, small_case  # noqa: E402

from tests._parity import TOL_BETA, assert_grad_close, grad_ref  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08463_b300 import csx
    csx.lib()
    yield


def _csx():
    from paper_2604_08463_b300 import csx
    return csx


# ------------------------------------------------------------------------------ mixing --------
def test_mixing_matches_oracle():
    csx = _csx()
    case = small_case()
    model = csx.Model(case.nu)
    rng = np.random.default_rng(0)
    beta = np.stack([rng.uniform(0.6, 2.9, 500), rng.uniform(6, 59, 500), rng.uniform(-4.9, -1.1, 500)], 1)
    A, dA = csx.mixing(model, torch.tensor(beta, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    A, dA = A.cpu().numpy(), dA.cpu().numpy()
    b32 = beta.astype(np.float32).astype(np.float64)
    ref = mx.mixing_matrix(case.nu, b32[:, 0], b32[:, 1], b32[:, 2])
    dref = np.stack(mx.mixing_derivatives(case.nu, b32[:, 0], b32[:, 1], b32[:, 2]), 1)
    F = case.nu.size
    np.testing.assert_allclose(A[:, :F, :], ref, rtol=2e-5, atol=0)
    np.testing.assert_allclose(dA[:, :, :F], dref, rtol=5e-5, atol=1e-6 * np.abs(dref).max())
    assert np.all(A[:, F:, :] == 0) and np.all(dA[:, :, F:] == 0)


# ------------------------------------------------------------- likelihood and gradient --------
@pytest.mark.parametrize("noise", ["homogeneous", "separable", "perpixel"])
@pytest.mark.parametrize("nside,K", [(8, (5, 3, 4)), (16, (40, 7, 12))])
def test_spectral_like_and_grad(noise, nside, K):
    csx = _csx()
    case = small_case(nside=nside, K=K, nreal=3, noise=noise)
    model, sky, labels = case.gpu()
    lab = case.wl.labels[0]
    beta = workloads.random_points(np.array(K), 3, seed=nside).astype(np.float32)
    bt = torch.tensor(beta, device="cuda")
    L1 = csx.spectral_like(model, sky, labels[0], K, bt)
    L2, g = csx.spectral_grad(model, sky, labels[0], K, bt)
    torch.cuda.synchronize()
    L1, L2, g = L1.cpu().numpy(), L2.cpu().numpy(), g.cpu().numpy()
    for r in range(3):
        Lr, gr, Sr = grad_ref(case, r, lab, K, beta[r].astype(np.float64))
        assert abs(L1[r] - Lr) <= 1e-5 * abs(Lr), (L1[r], Lr)
        assert abs(L2[r] - Lr) <= 1e-5 * abs(Lr)
        assert_grad_close(g[r], gr, Sr)


@pytest.mark.parametrize("noise", ["homogeneous", "separable", "perpixel"])
def test_spectral_kmeans_patches(noise):
    """K-means patches, as in the workloads: the 32 pixels of a warp of the streaming kernel fall
    into one to several runs of equal label triples. With separable / homogeneous noise the
    Gram-Schmidt scalars are formed once per run; warps with one run and with many must all match
    the oracle."""
    csx = _csx()
    K = (12, 3, 6)
    case = Case(workloads.fullsky(16, K, nreal=2), noise)
    lab = case.wl.labels[0]
    groups = lab[:, : lab.shape[1] // 32 * 32].reshape(3, -1, 32)
    ncells = [len(set(zip(*groups[:, w, :]))) for w in range(groups.shape[1])]
    assert min(ncells) == 1 and max(ncells) >= 5, np.bincount(ncells)
    model, sky, labels = case.gpu()
    beta = workloads.random_points(np.array(K), 2, seed=11).astype(np.float32)
    bt = torch.tensor(beta, device="cuda")
    L1 = csx.spectral_like(model, sky, labels[0], K, bt)
    L2, g = csx.spectral_grad(model, sky, labels[0], K, bt)
    torch.cuda.synchronize()
    L1, L2, g = L1.cpu().numpy(), L2.cpu().numpy(), g.cpu().numpy()
    for r in range(2):
        Lr, gr, Sr = grad_ref(case, r, lab, K, beta[r].astype(np.float64))
        assert abs(L1[r] - Lr) <= 1e-5 * abs(Lr), (L1[r], Lr)
        assert abs(L2[r] - Lr) <= 1e-5 * abs(Lr)
        assert_grad_close(g[r], gr, Sr)


@pytest.mark.parametrize("noise", ["homogeneous", "separable"])
@pytest.mark.parametrize("nside,K", [(8, (5, 3, 4)), (16, (12, 3, 6)), (16, (40, 7, 12))])
def test_spectral_plan_matches_oracle(noise, nside, K):
    """The cell-plan evaluation (scalars and band vectors formed per (problem, cell) before the
    streaming kernel): L and the adjoint gradient against the oracle, L alone as well, at K-means
    patches (warps holding one to several runs of a cell) and random beta."""
    csx = _csx()
    case = Case(workloads.fullsky(nside, K, nreal=3), noise)
    model, sky, labels = case.gpu()
    lab = case.wl.labels[0]
    plan = csx.SpectralPlan(labels[0], K)
    assert plan.ncell == len(set(zip(*lab)))
    beta = workloads.random_points(np.array(K), 3, seed=nside + 7).astype(np.float32)
    bt = torch.tensor(beta, device="cuda")
    L2, g = plan.grad(model, sky, bt)
    L1, none = plan.grad(model, sky, bt, want_grad=False)
    torch.cuda.synchronize()
    assert none is None
    L1, L2, g = L1.cpu().numpy(), L2.cpu().numpy(), g.cpu().numpy()
    for r in range(3):
        Lr, gr, Sr = grad_ref(case, r, lab, K, beta[r].astype(np.float64))
        assert abs(L1[r] - Lr) <= 1e-5 * abs(Lr), (L1[r], Lr)
        assert abs(L2[r] - Lr) <= 1e-5 * abs(Lr), (L2[r], Lr)
        assert_grad_close(g[r], gr, Sr)
    plan.close()


def test_spectral_plan_ragged_tail_one_pixel_cells_and_refusals():
    """300 pixels (a ragged last tile), every pixel its own beta_d patch (one-pixel cells); labels
    outside [0, K_j) refuse the plan on the host; per-pixel noise and a sky of another size refuse
    the evaluation."""
    csx = _csx()
    case = small_case(nside=8, K=(768, 2, 3), nreal=1, noise="separable")
    keep = 300
    lab = np.ascontiguousarray(case.wl.labels[0][:, :keep])
    lab[0] = np.arange(keep)
    K = (keep, 2, 3)
    d = torch.tensor(case.d32[:, :keep], device="cuda")
    sky = csx.Sky(d, noise="separable", ninv_band=case.nb32,
                  w=torch.tensor(case.w32[:keep], device="cuda"))
    model = csx.Model(case.nu)
    beta = workloads.random_points(np.array(K), 1, seed=5).astype(np.float32)
    plan = csx.SpectralPlan(torch.tensor(lab, device="cuda"), K)
    assert plan.ncell == keep
    L, g = plan.grad(model, sky, torch.tensor(beta, device="cuda"))
    torch.cuda.synchronize()
    Lr, gr, Sr = grad_ref(case, 0, lab, K, beta[0].astype(np.float64),
                          d64=case.d64(0)[:keep], ninv=case.ninv64[:keep])
    assert abs(L.item() - Lr) <= 1e-5 * abs(Lr)
    Sd = lk.gradient_term_scale(case.nu, case.d64(0)[:keep], case.ninv64[:keep], lab, K,
                                beta[0].astype(np.float64), data_scale=True)
    assert_grad_close(g.cpu().numpy()[0], gr, Sr + 16 * 2.0 ** -24 / 1e-5 * Sd)
    assert_grad_close(g.cpu().numpy()[0][keep:], gr[keep:], Sr[keep:])
    bad = lab.copy()
    bad[1, 17] = 2  # K_T = 2
    with pytest.raises(csx.CsxError, match="outside"):
        csx.SpectralPlan(torch.tensor(bad, device="cuda"), K)
    other = small_case(nside=8, K=(5, 3, 4), nreal=1, noise="perpixel")
    m2, sky_pp, _ = other.gpu()
    with pytest.raises(csx.CsxError, match="per-pixel|homogeneous or separable"):
        plan.grad(m2, sky_pp, torch.zeros((1, sum(K)), device="cuda"))
    sep = small_case(nside=8, K=(5, 3, 4), nreal=1, noise="separable")
    m3, sky_768, _ = sep.gpu()
    with pytest.raises(csx.CsxError, match="npix"):
        plan.grad(m3, sky_768, torch.zeros((1, sum(K)), device="cuda"))


def test_spectral_misaligned_data_is_refused():
    """Data not 16-byte aligned cannot be read as 16-byte pixel vectors nor staged by tensor copies:
    the call is refused on the host with CSX_EINVAL, nothing is launched, and the same data from an
    aligned buffer evaluates normally afterwards."""
    csx = _csx()
    K = (12, 3, 6)
    case = Case(workloads.fullsky(16, K, nreal=2), "separable")
    model, sky, labels = case.gpu()
    n = case.d32.size
    raw = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    raw[1:] = torch.from_numpy(case.d32.reshape(-1)).to("cuda")
    d_off = raw[1:].view(case.d32.shape)
    assert d_off.data_ptr() % 16 != 0
    sky_off = csx.Sky(d_off, noise="separable", ninv_band=case.nb32, w=sky.w)
    beta = torch.tensor(workloads.random_points(np.array(K), 2, seed=12), dtype=torch.float32,
                        device="cuda")
    with pytest.raises(csx.CsxError, match="16-byte aligned"):
        csx.spectral_grad(model, sky_off, labels[0], K, beta)
    La, ga = csx.spectral_grad(model, sky, labels[0], K, beta)
    torch.cuda.synchronize()
    Lr, gr, Sr = grad_ref(case, 0, case.wl.labels[0], K, beta[0].cpu().numpy().astype(np.float64))
    assert abs(La[0].item() - Lr) <= 1e-5 * abs(Lr)
    assert_grad_close(ga[0].cpu().numpy(), gr, Sr)


def test_spectral_ragged_tails_and_one_pixel_patches():
    csx = _csx()
    # 300 pixels (not a multiple of the block size), every pixel its own beta_d patch
    case = small_case(nside=8, K=(768, 2, 3), nreal=1, noise="separable")
    keep = 300
    wl = case.wl
    lab = np.ascontiguousarray(wl.labels[0][:, :keep])
    lab[0] = np.arange(keep)
    K = (keep, 2, 3)
    d = torch.tensor(case.d32[:, :keep], device="cuda")
    sky = csx.Sky(d, noise="separable", ninv_band=case.nb32,
                  w=torch.tensor(case.w32[:keep], device="cuda"))
    model = csx.Model(case.nu)
    beta = workloads.random_points(np.array(K), 1, seed=5).astype(np.float32)
    L, g = csx.spectral_grad(model, sky, torch.tensor(lab, device="cuda"), K,
                             torch.tensor(beta, device="cuda"))
    torch.cuda.synchronize()
    Lr, gr, Sr = grad_ref(case, 0, lab, K, beta[0].astype(np.float64),
                          d64=case.d64(0)[:keep], ninv=case.ninv64[:keep])
    assert abs(L.item() - Lr) <= 1e-5 * abs(Lr)
    # A one-pixel patch has no sum to average rounding over: at nside 8 (|d| / |r| ~ 3e3 per band)
    # its gradient is bounded by the FP32 forming of r = d - A s_hat, error <= ~4 u |d| per band,
    # i.e. 4 u S_d with S_d the data-scaled term magnitude (u = 2^-24); checked with a factor 4.
    Sd = lk.gradient_term_scale(case.nu, case.d64(0)[:keep], case.ninv64[:keep], lab, K,
                                beta[0].astype(np.float64), data_scale=True)
    assert_grad_close(g.cpu().numpy()[0], gr, Sr + 16 * 2.0 ** -24 / 1e-5 * Sd)
    # the beta_d components of the T_d / beta_s patches (many pixels) keep the plain bound
    assert_grad_close(g.cpu().numpy()[0][keep:], gr[keep:], Sr[keep:])


def test_out_of_range_label_poisons_L():
    csx = _csx()
    case = small_case(nside=8, K=(5, 3, 4), nreal=1)
    model, sky, labels = case.gpu()
    lab = labels[0].clone()
    lab[1, 17] = 3  # K_T = 3
    beta = torch.tensor(workloads.random_points(np.array((5, 3, 4)), 1), dtype=torch.float32,
                        device="cuda")
    L = csx.spectral_like(model, sky, lab, (5, 3, 4), beta)
    torch.cuda.synchronize()
    assert np.isnan(L.item())


def test_bad_arguments_are_rejected():
    csx = _csx()
    case = small_case(nside=8, K=(5, 3, 4), nreal=1)
    model, sky, labels = case.gpu()
    beta = torch.zeros((2, 12), device="cuda")
    with pytest.raises(csx.CsxError) as e:
        csx.spectral_like(model, sky, labels[0], (5, 3, 4), beta)  # nprob 2 > nreal 1
    assert e.value.code == -1
    with pytest.raises(csx.CsxError):
        csx.spectral_like(model, sky, labels[0], (0, 3, 4), beta[:1])


def test_empty_batch_is_a_no_op():
    csx = _csx()
    case = small_case(nside=8, K=(5, 3, 4), nreal=1)
    model, sky, labels = case.gpu()
    L = csx.spectral_like(model, sky, labels[0], (5, 3, 4), torch.zeros((0, 12), device="cuda"))
    assert L.numel() == 0


def test_autograd_function():
    csx = _csx()
    K = (6, 3, 2)
    case = small_case(nside=8, K=K, nreal=2, noise="separable")
    model, sky, labels = case.gpu()
    beta = torch.tensor(workloads.random_points(np.array(K), 2, seed=3), dtype=torch.float32,
                        device="cuda", requires_grad=True)
    L = csx.SpectralLikelihood.apply(beta, model, sky, labels[0], K)
    (3.0 * L[0] - 0.5 * L[1]).backward()
    torch.cuda.synchronize()
    b = beta.detach().cpu().numpy().astype(np.float64)
    _, g0, S0 = grad_ref(case, 0, case.wl.labels[0], K, b[0])
    _, g1, S1 = grad_ref(case, 1, case.wl.labels[0], K, b[1])
    got = beta.grad.cpu().numpy()
    assert_grad_close(got[0], 3.0 * g0, 3.0 * S0)
    assert_grad_close(got[1], -0.5 * g1, 0.5 * S1)


# ------------------------------------------------------------------------------- cells --------
def test_cells_bit_exact():
    csx = _csx()
    case = scan_case(nside=16, nconf=8, kmax=60, nreal=1)
    wl = case.wl
    labels = torch.tensor(wl.labels, device="cuda")
    perm, off, nc = csx.build_cells(labels, wl.K)
    torch.cuda.synchronize()
    perm, off, nc = perm.cpu().numpy(), off.cpu().numpy(), nc.cpu().numpy()
    for c in range(wl.nconf):
        p, o, _ = ocells.cells(wl.labels[c])
        assert nc[c] == o.size - 1
        np.testing.assert_array_equal(perm[c], p)
        np.testing.assert_array_equal(off[c, :nc[c] + 1], o)


def test_cells_wide_labels_and_bad_label():
    csx = _csx()
    rng = np.random.default_rng(1)
    npix = 5000
    K = np.array([[4000, 300, 70000], [1, 1, 1], [2, 65536, 3]], np.int32)
    lab = np.stack([np.stack([rng.integers(0, k, npix) for k in row]) for row in K]).astype(np.int32)
    perm, off, nc = csx.build_cells(torch.tensor(lab, device="cuda"), K)
    torch.cuda.synchronize()
    for c in range(3):
        p, o, _ = ocells.cells(lab[c])
        np.testing.assert_array_equal(perm.cpu().numpy()[c], p)
        assert nc[c].item() == o.size - 1
    lab[1, 0, 7] = 1  # K_d = 1
    _, _, nc = csx.build_cells(torch.tensor(lab, device="cuda"), K)
    torch.cuda.synchronize()
    assert nc.cpu().numpy()[1] == -1


# --------------------------------------------------------------------------------- fit --------
def _oracle_fit(case, c, r):
    wl = case.wl
    K = wl.K[c]
    return ofit.fit(case.nu, case.d64(r), case.ninv64, wl.labels[c], K, wl.beta0(c),
                    workloads.LOWER, workloads.UPPER)


def _check_fit(case, res, c, r, P_off):
    wl = case.wl
    K = wl.K[c]
    P = int(K.sum())
    x_ref, L_ref, info = _oracle_fit(case, c, r)
    got = res["beta"][P_off:P_off + P]
    types = np.concatenate([np.full(K[j], j) for j in range(3)])
    tol = TOL_BETA[types]
    interior = info["interior"]
    err = np.abs(got - x_ref)
    assert np.all(err[interior] <= tol[interior]), (err[interior] / tol[interior]).max()
    return err / tol, L_ref


@pytest.mark.parametrize("path", ["moment", "stream"])
def test_fit_plain_nside8(path):
    """Uniform sky, homogeneous noise, one patch each, one realization, start (1.5, 19, -2.9)."""
    csx = _csx()
    wl = workloads.plain(8)
    case = Case(wl, "homogeneous")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(wl.beta0(0), dtype=torch.float32, device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0, path=path)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items()}
    assert out["status"][0] == 0, out
    ratio, L_ref = _check_fit(case, out, 0, 0, 0)
    assert abs(out["L"][0] - L_ref) <= 1e-5 * abs(L_ref)


@pytest.mark.parametrize("path", ["moment", "stream"])
def test_fit_small_scan(path):
    csx = _csx()
    case = scan_case(nside=16, nconf=5, kmax=30, nreal=2)
    wl = case.wl
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0, path=path)
    torch.cuda.synchronize()
    # every problem at the plain tolerances (tests/_fitcheck.py); the fit is deterministic, so a
    # second call returns the same bits
    from tests._fitcheck import sampled_fit_check
    worst, alt = sampled_fit_check(csx, case, res, list(range(wl.nconf * wl.nreal)),
                                   max_alternative=0)
    res2 = csx.fit_batch(model, sky, labels, wl.K, beta0, path=path)
    torch.cuda.synchronize()
    for k in ("beta", "L", "status", "iters", "nevals"):
        assert torch.equal(res[k], res2[k]), k


@pytest.mark.parametrize("path", ["moment", "stream"])
def test_fit_is_deterministic(path):
    """The same inputs give bit-identical fits on every call (fixed-order gradient sums), also when
    the problems are queued differently (a second configuration batch with the order reversed)."""
    csx = _csx()
    case = scan_case(nside=16, nconf=6, kmax=40, nreal=2)
    wl = case.wl
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    outs = [csx.fit_batch(model, sky, labels, wl.K, beta0, path=path) for _ in range(3)]
    torch.cuda.synchronize()
    for o in outs[1:]:
        for k in ("beta", "L", "status", "iters", "nevals"):
            assert torch.equal(outs[0][k], o[k]), k
    # the last configuration alone: its problems run in other CTA slots, same bits
    offs, P = csx.param_offsets(wl.K, wl.nreal)
    c = wl.nconf - 1
    q0 = c * wl.nreal
    one = csx.fit_batch(model, sky, labels[c:c + 1].contiguous(), wl.K[c:c + 1],
                        beta0[int(offs[q0]):].contiguous(), path=path)
    torch.cuda.synchronize()
    assert torch.equal(one["beta"], outs[0]["beta"][int(offs[q0]):])
    assert torch.equal(one["L"], outs[0]["L"][q0:])


# ------------------------------------------------------------------------------ AdaTopK -------
@pytest.mark.parametrize("path", ["moment", "stream"])
def test_adatopk_fit_plain_nside8(path):
    """AdaTopK (App. A) reaches the oracle optimum; its value agrees with the AdaTopK oracle's."""
    from oracle import adatopk as oat
    csx = _csx()
    wl = workloads.plain(8)
    case = Case(wl, "homogeneous")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(wl.beta0(0), dtype=torch.float32, device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0, path=path, solver="adatopk", max_iter=5000)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items()}
    assert out["status"][0] == 0, out
    ratio, L_ref = _check_fit(case, out, 0, 0, 0)
    assert abs(out["L"][0] - L_ref) <= 1e-5 * abs(L_ref)
    x_at, L_at, info = oat.fit(case.nu, case.d64(0), case.ninv64, wl.labels[0], wl.K[0], wl.beta0(0),
                               workloads.LOWER, workloads.UPPER)
    assert info["status"] == 0 and abs(out["L"][0] - L_at) <= 1e-5 * abs(L_at)


def test_adatopk_start_on_bounds_is_released():
    """Every parameter starts on a bound (beta_d at its upper, T_d at its lower, beta_s at its upper
    bound); the gradient points into the box, the constraints are released one per iteration
    (K = 0) and the fit reaches the interior optimum."""
    csx = _csx()
    wl = workloads.plain(8)
    case = Case(wl, "homogeneous")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor([workloads.UPPER[0], workloads.LOWER[1], workloads.UPPER[2]],
                         dtype=torch.float32, device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0, solver="adatopk", max_iter=5000)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items()}
    assert out["status"][0] == 0, out
    _check_fit(case, out, 0, 0, 0)


@pytest.mark.parametrize("path", ["moment", "stream"])
def test_adatopk_fit_small_scan(path):
    csx = _csx()
    case = scan_case(nside=16, nconf=5, kmax=30, nreal=2)
    wl = case.wl
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    res = csx.fit_batch(model, sky, labels, wl.K, beta0, path=path, solver="adatopk",
                        max_iter=5000)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in res.items()}
    offs, _ = csx.param_offsets(wl.K, wl.nreal)
    worst = 0.0
    for c in range(wl.nconf):
        for r in range(wl.nreal):
            q = c * wl.nreal + r
            assert out["status"][q] == 0, (q, out["status"][q], out["iters"][q])
            ratio, L_ref = _check_fit(case, out, c, r, offs[q])
            worst = max(worst, ratio.max())
            assert abs(out["L"][q] - L_ref) <= 1e-5 * abs(L_ref)
    print("worst |err|/tol", worst, "iterations", out["iters"].mean())


def test_adatopk_options_are_checked():
    csx = _csx()
    wl = workloads.plain(8)
    case = Case(wl, "homogeneous")
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(wl.beta0(0), dtype=torch.float32, device="cuda")
    with pytest.raises(csx.CsxError, match="adjoint"):
        csx.fit_batch(model, sky, labels, wl.K, beta0, solver="adatopk", grad_mode="fd")
    with pytest.raises(csx.CsxError, match="topk"):
        csx.fit_batch(model, sky, labels, wl.K, beta0, solver="adatopk", topk=1.5)


# ------------------------------------------------------------------------ reconstruction ------
def test_reconstruct_and_select():
    csx = _csx()
    case = scan_case(nside=16, nconf=4, kmax=20, nreal=2)
    wl = case.wl
    model, sky, labels = case.gpu()
    rng = np.random.default_rng(8)
    per = []
    for c in range(wl.nconf):
        for r in range(wl.nreal):
            per.append(workloads.random_points(wl.K[c], 1, seed=int(rng.integers(1e6)))[0])
    beta = pack(wl, per)
    fg = torch.tensor(case.fg32, device="cuda")
    out = csx.reconstruct(model, sky, labels, wl.K, torch.tensor(beta, device="cuda"), d_fg=fg,
                          s_hat=True, sigma2=True, r_sys=True, metrics=True)
    vt, best = csx.select(out["metrics"], wl.nconf, wl.nreal)
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    offs, P = csx.param_offsets(wl.K, wl.nreal)
    metrics = []
    for c in range(wl.nconf):
        row = []
        for r in range(wl.nreal):
            q = c * wl.nreal + r
            b = beta[offs[q]:offs[q] + P[c]].astype(np.float64)
            s = rc.reconstruct(case.nu, case.d64(r), case.ninv64, wl.labels[c], wl.K[c], b)
            sv = rc.stat_variance(case.nu, case.ninv64, wl.labels[c], wl.K[c], b)
            rs = rc.systematic_residual(case.nu, case.fg64(), case.ninv64, wl.labels[c], wl.K[c], b)
            np.testing.assert_allclose(o["s_hat"][q], s, rtol=0, atol=1e-4 * np.abs(s).max())
            np.testing.assert_allclose(o["sigma2"][q], sv, rtol=1e-4)
            np.testing.assert_allclose(o["r_sys"][q], rs, rtol=0, atol=1e-4 * np.abs(rs).max() + 1e-6)
            m = rc.problem_metrics(case.nu, case.d64(r), case.fg64(), case.ninv64, wl.labels[c],
                                   wl.K[c], b)
            got = o["metrics"][q]
            assert abs(got[csx.M_SYS_SQ] - m["sys_sq"]) <= 1e-3 * m["sys_sq"] + 1e-9
            assert abs(got[csx.M_STAT] - m["stat"]) <= 1e-4 * m["stat"]
            assert abs(got[csx.M_CMB_Q2] - m["cmb_q_sumsq"]) <= 1e-4 * m["cmb_q_sumsq"]
            assert got[csx.M_NPIX] == wl.npix
            row.append(m)
        metrics.append(row)
    v_ref, best_ref = rc.total_residual_variance(metrics, wl.npix)
    np.testing.assert_allclose(vt.cpu().numpy(), v_ref, rtol=1e-3)
    assert best.item() == best_ref
