"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a wrong unit factor) fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import cells as ocells
from oracle import fit as ofit
from oracle import likelihood as lk
from oracle import mixing as mx
from oracle import reconstruct as rc
from synth import healpix, sky as S, workloads

NU = S.BANDS_GHZ
HERE = os.path.dirname(os.path.abspath(__file__))

# -- independent physical route for the SED columns (Planck's law, SI constants) -------------
H, KB, C, TCMB = 6.62607015e-34, 1.380649e-23, 299792458.0, 2.7255


def _planck(nu_ghz, t):
    nu = nu_ghz * 1e9
    return 2 * H * nu ** 3 / C ** 2 / np.expm1(H * nu / (KB * t))


def _dbdt_cmb(nu_ghz):
    nu = nu_ghz * 1e9
    x = H * nu / (KB * TCMB)
    return 2 * H * nu ** 3 / C ** 2 * x / TCMB * np.exp(x) / np.expm1(x) ** 2


def _physical_dust(nu, bd, td, nu0=353.0):
    # K_CMB response to a dust intensity I ∝ nu^bd B_nu(T_d), unit K_CMB at nu0
    i = nu ** bd * _planck(nu, td)
    i0 = nu0 ** bd * _planck(nu0, td)
    return (i / _dbdt_cmb(nu)) / (i0 / _dbdt_cmb(nu0))


def _physical_sync(nu, bs, nu0=23.0):
    # K_CMB response to a Rayleigh-Jeans brightness T_RJ ∝ nu^bs, unit K_CMB at nu0
    i = nu ** bs * 2 * KB * (nu * 1e9) ** 2 / C ** 2
    i0 = nu0 ** bs * 2 * KB * (nu0 * 1e9) ** 2 / C ** 2
    return (i / _dbdt_cmb(nu)) / (i0 / _dbdt_cmb(nu0))


# ---------------------------------------------------------------- HEALPix geometry -------
def test_healpix_nside1_centres():
    z, phi = healpix.pixel_centres(1)
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    q = np.pi / 4
    np.testing.assert_allclose(phi, [q, 3 * q, 5 * q, 7 * q, 0, 2 * q, 4 * q, 6 * q,
                                     q, 3 * q, 5 * q, 7 * q], atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 64])
def test_healpix_structure(nside):
    z, phi = healpix.pixel_centres(nside)
    assert z.size == 12 * nside * nside
    assert abs(z.sum()) < 1e-9 * z.size  # north/south symmetry
    assert np.all(np.diff(z) <= 1e-15)   # rings run north to south
    assert np.all((phi >= 0) & (phi < 2 * np.pi))
    # equal area: the number of centres above z0 tracks npix (1 - z0) / 2 to within one ring
    for z0 in (0.9, 0.5, 0.2, -0.3):
        n = np.sum(z > z0)
        assert abs(n - z.size * (1 - z0) / 2) <= 4 * nside + 1
    v = healpix.unit_vectors(nside)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)


def test_galactic_cut_count():
    # |b| > 20 deg at nside 64 keeps 32512 of 49152 pixels (f_sky = 0.661)
    pix = healpix.galactic_cut(64, 20.0)
    assert pix.size == 32512
    assert abs(pix.size / 49152 - (1 - np.sin(np.deg2rad(20)))) < 0.01


# ---------------------------------------------------------------- mixing matrix ----------
def test_mixing_hand_values():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "mixing_hand_values.txt"))
            if l.strip() and not l.startswith("#")]
    A = mx.mixing_matrix(NU, 1.54, 20.0, -3.0)
    for nu, col, val in rows:
        nu, val = float(nu), float(val)
        if col == "g":
            got = mx.rj_to_cmb(nu)
        else:
            f = int(np.nonzero(NU == nu)[0][0])
            got = A[f, 1 if col == "dust" else 2]
        assert abs(got - val) / abs(val) < 1e-3, (nu, col, got, val)


@pytest.mark.parametrize("bd,td,bs", [(1.54, 20.0, -3.0), (0.7, 8.0, -1.5), (2.6, 55.0, -4.4)])
def test_mixing_matches_planck_law(bd, td, bs):
    A = mx.mixing_matrix(NU, bd, td, bs)
    np.testing.assert_allclose(A[:, 0], 1.0)
    np.testing.assert_allclose(A[:, 1], _physical_dust(NU, bd, td), rtol=1e-12)
    np.testing.assert_allclose(A[:, 2], _physical_sync(NU, bs), rtol=1e-12)
    # the sky simulator (input generator) uses the same physics
    np.testing.assert_allclose(S.dust_kcmb(NU, 1.0, bd, td) / S.rj_to_kcmb(353.0), A[:, 1],
                               rtol=1e-12)
    np.testing.assert_allclose(S.sync_kcmb(NU, 1.0, bs) / S.rj_to_kcmb(23.0), A[:, 2], rtol=1e-12)


def test_mixing_normalisation_and_limits():
    # unit response at the reference frequencies
    assert abs(mx.mixing_matrix(np.array([353.0]), 1.3, 17.0, -2.0)[0, 1] - 1) < 1e-14
    assert abs(mx.mixing_matrix(np.array([23.0]), 1.3, 17.0, -2.0)[0, 2] - 1) < 1e-14
    # Rayleigh-Jeans limit: T_d -> infinity gives (nu/nu0)^beta_d times the unit conversion
    A = mx.mixing_matrix(NU, 1.6, 1e7, -3.0)
    rj = (NU / 353.0) ** 1.6 * mx.rj_to_cmb(NU) / mx.rj_to_cmb(353.0)
    np.testing.assert_allclose(A[:, 1], rj, rtol=1e-5)
    # RJ units drop the conversion
    Arj = mx.mixing_matrix(NU, 1.6, 20.0, -3.0, units="RJ")
    np.testing.assert_allclose(Arj[:, 2], (NU / 23.0) ** -3.0, rtol=1e-14)


def test_mixing_derivatives_fd():
    p = np.array([1.47, 23.0, -3.1])
    dbd, dtd, dbs = mx.mixing_derivatives(NU, *p)
    h = 1e-6
    fd = lambda i, col: (mx.mixing_matrix(NU, *(p + h * np.eye(3)[i]))[:, col] -
                         mx.mixing_matrix(NU, *(p - h * np.eye(3)[i]))[:, col]) / (2 * h)
    np.testing.assert_allclose(dbd, fd(0, 1), rtol=1e-7)
    np.testing.assert_allclose(dtd, fd(1, 1), rtol=1e-6)
    np.testing.assert_allclose(dbs, fd(2, 2), rtol=1e-7)


# ---------------------------------------------------------------- GLS / likelihood --------
def _small_problem(nside=4, K=(3, 2, 2), hitcount=True, seed=0, truth="smooth"):
    sk = S.make_sky(nside, truth=truth, hitcount=hitcount)
    rng = np.random.default_rng(seed)
    labels = np.stack([rng.integers(0, K[j], sk.npix) for j in range(3)]).astype(np.int64)
    for j in range(3):  # make every patch non-empty
        labels[j, :K[j]] = np.arange(K[j])
    d = sk.data(0)
    ninv = sk.ninv_pixel()
    return sk, labels, np.array(K), d, ninv


def test_gls_is_textbook_least_squares():
    sk, labels, K, d, ninv = _small_problem()
    beta = workloads.random_points(K, 1)[0]
    A = lk.pixel_mixing(NU, beta, labels, K)
    s = lk.gls_components(A, ninv, d)
    for p in range(0, sk.npix, 17):
        sw = np.sqrt(ninv[p])
        for st in range(2):
            ref = np.linalg.lstsq(sw[:, None] * A[p], sw * d[p, st], rcond=None)[0]
            np.testing.assert_allclose(s[p, st], ref, rtol=1e-9, atol=1e-9)


def test_WA_identity_and_unit_response():
    sk, labels, K, d, ninv = _small_problem()
    beta = workloads.random_points(K, 1)[0]
    A = lk.pixel_mixing(NU, beta, labels, K)
    W = rc.weights(A, ninv)
    WA = np.einsum("pcf,pfk->pck", W, A)
    np.testing.assert_allclose(WA, np.broadcast_to(np.eye(3), WA.shape), atol=1e-10)
    # Eq. 10: [W A_cmb]_cmb = 1 with A_cmb = 1 in every band
    np.testing.assert_allclose(W[:, 0, :].sum(axis=1), 1.0, atol=1e-10)


def test_likelihood_identity_and_bound():
    sk, labels, K, d, ninv = _small_problem()
    beta = workloads.random_points(K, 1)[0]
    L = lk.spectral_likelihood(NU, d, ninv, labels, K, beta)
    chi2 = lk.chi2_min(NU, d, ninv, labels, K, beta)
    dn = lk.data_norm(d, ninv)
    assert chi2 > 0
    assert abs((L + dn) - chi2) <= 1e-9 * dn
    assert L >= -dn


def test_noise_free_minimum_at_truth():
    # uniform truth, one patch: chi2_min(beta_true) = 0, grad = 0; elsewhere L > -sum d N d
    sk = S.make_sky(4, truth="uniform", hitcount=True)
    labels = np.zeros((3, sk.npix), np.int64)
    K = np.array([1, 1, 1])
    d = sk.data(None)
    ninv = sk.ninv_pixel()
    truth = np.array([1.54, 20.0, -3.0])
    dn = lk.data_norm(d, ninv)
    assert lk.chi2_min(NU, d, ninv, labels, K, truth) < 1e-14 * dn
    L, g = lk.spectral_gradient(NU, d, ninv, labels, K, truth)
    assert abs(L + dn) < 1e-12 * dn
    _, g_off = lk.spectral_gradient(NU, d, ninv, labels, K, truth + [0.01, 0.5, 0.01])
    assert np.all(np.abs(g) < 1e-6 * np.abs(g_off))
    for dv in ([0.02, 0, 0], [0, 1.0, 0], [0, 0, -0.02]):
        assert lk.spectral_likelihood(NU, d, ninv, labels, K, truth + dv) > -dn


@pytest.mark.parametrize("hitcount", [False, True])
def test_gradient_central_fd(hitcount):
    sk, labels, K, d, ninv = _small_problem(hitcount=hitcount)
    beta = workloads.random_points(K, 1, seed=11)[0]
    L, g = lk.spectral_gradient(NU, d, ninv, labels, K, beta)
    assert abs(L - lk.spectral_likelihood(NU, d, ninv, labels, K, beta)) < 1e-12 * abs(L)
    # chi2_min differs from L by a beta-independent constant: difference it (no cancellation)
    h = np.where(np.arange(K.sum()) < K[0], 1e-5, 1e-5)
    h[K[0]:K[0] + K[1]] = 1e-4  # T_d in K
    fd = np.empty_like(g)
    for i in range(K.sum()):
        e = np.zeros(K.sum())
        e[i] = h[i]
        fd[i] = (lk.chi2_min(NU, d, ninv, labels, K, beta + e) -
                 lk.chi2_min(NU, d, ninv, labels, K, beta - e)) / (2 * h[i])
    np.testing.assert_allclose(g, fd, rtol=2e-6, atol=1e-6 * np.abs(g).max())


def test_gradient_term_scale_bounds_the_gradient():
    sk, labels, K, d, ninv = _small_problem()
    beta = workloads.random_points(K, 1, seed=4)[0]
    _, g = lk.spectral_gradient(NU, d, ninv, labels, K, beta)
    sc = lk.gradient_term_scale(NU, d, ninv, labels, K, beta)
    assert sc.shape == g.shape and np.all(sc > 0)
    assert np.all(sc >= np.abs(g) * (1 - 1e-12))  # triangle inequality
    # one patch per parameter, one pixel: S is the sum of the band terms' magnitudes
    lab1 = np.zeros((3, 1), np.int64)
    _, g1 = lk.spectral_gradient(NU, d[:1], ninv[:1], lab1, np.array([1, 1, 1]), beta[[0, 3, 5]])
    s1 = lk.gradient_term_scale(NU, d[:1], ninv[:1], lab1, np.array([1, 1, 1]), beta[[0, 3, 5]])
    assert np.all(s1 >= np.abs(g1))


def test_gls_statistics_monte_carlo():
    # at fixed beta, Var[s_hat_cmb] over noise draws -> [M^-1]_00 and <s_hat> = s at beta_true
    sk = S.make_sky(2, truth="uniform", hitcount=True)
    labels = np.zeros((3, sk.npix), np.int64)
    K = np.array([1, 1, 1])
    beta = np.array([1.54, 20.0, -3.0])
    ninv = sk.ninv_pixel()
    var = rc.stat_variance(NU, ninv, labels, K, beta)
    ndraw = 4000
    s = np.empty((ndraw, sk.npix, 2))
    for n in range(ndraw):
        s[n] = rc.reconstruct(NU, sk.signal + sk.noise(n), ninv, labels, K, beta)[:, :, 0]
    emp = s.var(axis=0).mean(axis=1)
    rel = emp / var - 1
    assert np.all(np.abs(rel) < 5 * np.sqrt(2.0 / ndraw) * 1.5), rel
    bias = (s.mean(axis=0) - sk.cmb) / np.sqrt(var[:, None] / ndraw)
    assert np.all(np.abs(bias) < 5.0)


# ---------------------------------------------------------------- fit ----------------------
def test_bruteforce_grid_minimum():
    # tiny sky, one patch per parameter: the 41^3 grid minimum is within one grid step of the fit
    sk = S.make_sky(2, truth="uniform", hitcount=False)
    sk.sigma = sk.sigma * 30.0  # lower SNR so the minimum lies away from the truth
    d = sk.data(3)
    ninv = sk.ninv_pixel()
    labels = np.zeros((3, sk.npix), np.int64)
    K = np.array([1, 1, 1])
    x, L, info = ofit.fit(NU, d, ninv, labels, K, [1.5, 19.0, -2.9], workloads.LOWER,
                          workloads.UPPER)
    step = np.array([0.002, 0.1, 0.004])
    axes = [x[i] + step[i] * np.arange(-20, 21) + 0.37 * step[i] for i in range(3)]
    gd, gt, gs = np.meshgrid(*axes, indexing="ij")
    A = mx.mixing_matrix(NU, gd.ravel(), gt.ravel(), gs.ravel())  # [G, F, 3]
    nb = ninv[0]
    M = np.einsum("gfi,f,gfj->gij", A, nb, A)
    Sd = np.einsum("psf,psg->fg", d, d)
    G = np.einsum("gfi,f,fh,h,ghj->gij", A, nb, Sd, nb, A)
    Lg = -np.sum(np.linalg.inv(M) * G, axis=(1, 2))
    i = np.unravel_index(np.argmin(Lg), gd.shape)
    best = np.array([axes[0][i[0]], axes[1][i[1]], axes[2][i[2]]])
    assert np.all(np.abs(best - x) <= step * 1.0001), (best, x)
    assert L <= Lg.min() + 1e-9 * abs(L)


def test_known_truth_recovery_as_noise_vanishes():
    # piecewise-constant truth on known labels; sigma -> 0 drives beta_hat -> beta_true (Sec. 4.1)
    sk = S.make_sky(4, truth="uniform", hitcount=True)
    rng = np.random.default_rng(5)
    K = np.array([3, 2, 2])
    labels = np.stack([rng.integers(0, K[j], sk.npix) for j in range(3)])
    for j in range(3):
        labels[j, :K[j]] = np.arange(K[j])
    truth = np.array([1.45, 1.6, 1.52, 18.0, 23.0, -2.95, -3.1])
    S2 = S.Sky(4, sk.pix, np.stack(lk.pixel_parameters(truth, labels, K), 1), sk.cmb,
               sk.dust_amp, sk.sync_amp, sk.w)
    errs = []
    for scale in (1.0, 1e-3):
        S2.sigma = S.white_noise_sigma(4) * scale
        d = S2.data(0)
        x, _, _ = ofit.fit(NU, d, S2.ninv_pixel(), labels, K, np.r_[[1.5] * 3, [19.0] * 2,
                                                                     [-2.9] * 2],
                           workloads.LOWER, workloads.UPPER)
        errs.append(np.abs(x - truth))
    # the error is linear in the noise rms: shrinking sigma by 1e3 shrinks it by ~1e3
    ratio = errs[1] / errs[0]
    assert np.all((ratio > 0.3e-3) & (ratio < 3e-3)), ratio


def test_fit_is_stationary_and_pd():
    sk, labels, K, d, ninv = _small_problem(nside=4, K=(2, 2, 1), seed=3)
    x, L, info = ofit.fit(NU, d, ninv, labels, K, np.r_[[1.5] * 2, [19.0] * 2, [-2.9]],
                          workloads.LOWER, workloads.UPPER)
    assert info["interior"].all()
    _, g = lk.spectral_gradient(NU, d, ninv, labels, K, x)
    _, g0 = lk.spectral_gradient(NU, d, ninv, labels, K, np.r_[[1.5] * 2, [19.0] * 2, [-2.9]])
    assert np.abs(g).max() < 1e-6 * np.abs(g0).max()


# ---------------------------------------------------------------- cells / moments ----------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cells_match_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = 500
    labels = np.stack([rng.integers(0, k, n) for k in (7, 3, 5)])
    a = ocells.cells(labels)
    b = ocells.cells_bruteforce(labels)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_moment_form_equals_pixel_form():
    sk, labels, K, d, ninv = _small_problem(nside=4, K=(4, 3, 2))
    beta = workloads.random_points(K, 1, seed=7)[0]
    Sm, trip = ocells.cell_moments(d, sk.w, labels)
    Lm = ocells.moment_likelihood(NU, Sm, trip, sk.ninv_band, K, beta)
    L = lk.spectral_likelihood(NU, d, ninv, labels, K, beta)
    assert abs(Lm - L) < 1e-10 * abs(L)


# ---------------------------------------------------------------- reconstruction ------------
def test_systematic_residual_via_unit_response():
    sk, labels, K, d, ninv = _small_problem()
    beta = workloads.random_points(K, 1, seed=2)[0]
    with_cmb = rc.reconstruct(NU, sk.signal, ninv, labels, K, beta)[:, :, 0] - sk.cmb
    rs = rc.systematic_residual(NU, sk.foreground, ninv, labels, K, beta)
    np.testing.assert_allclose(with_cmb, rs, atol=1e-8 * np.abs(sk.signal).max())


def test_selection_argmin_and_ties():
    m = lambda s, t: {"sys_sq": s, "stat": t}
    v, best = rc.total_residual_variance([[m(2.0, 1.0)], [m(0.0, 1.0)], [m(0.0, 1.0)]], npix=1)
    np.testing.assert_allclose(v, [2.0, 1.0, 1.0])
    assert best == 1


def test_gauss_newton_diagonal_is_the_exact_curvature_at_a_noiseless_truth():
    """With noise-free data d = A(beta_true) s and the amplitudes held at s, the residual vanishes at
    beta_true, so the second derivative of f(beta) = sum_p sum_s (d - A(beta) s)^T N^-1 (d - A(beta) s)
    there is exactly 2 sum (dA/dtheta s)^T N^-1 (dA/dtheta s): the Gauss-Newton diagonal. f is
    formed here from the mixing matrix alone and differenced twice (central, O(h^2))."""
    sk = S.make_sky(4, truth="uniform", hitcount=True)
    rng = np.random.default_rng(5)
    K = np.array([3, 2, 2])
    labels = np.stack([rng.integers(0, K[j], sk.npix) for j in range(3)]).astype(np.int64)
    for j in range(3):
        labels[j, :K[j]] = np.arange(K[j])
    beta = np.concatenate([np.full(K[0], 1.54), np.full(K[1], 20.0), np.full(K[2], -3.0)])
    d = sk.data(None)
    ninv = sk.ninv_pixel()
    s = lk.gls_components(lk.pixel_mixing(NU, beta, labels, K), ninv, d)  # = the true amplitudes

    def f(b):
        r = d - np.einsum("pfi,psi->psf", lk.pixel_mixing(NU, b, labels, K), s)
        return float(np.sum(r * ninv[:, None, :] * r))

    assert f(beta) < 1e-20 * lk.data_norm(d, ninv)
    H = lk.gauss_newton_diagonal(NU, d, ninv, labels, K, beta)
    fd = np.empty_like(H)
    for i in range(K.sum()):
        h = 1e-3 if K[0] <= i < K[0] + K[1] else 1e-4
        e = np.zeros(K.sum())
        e[i] = h
        fd[i] = (f(beta + e) - 2.0 * f(beta) + f(beta - e)) / h ** 2
    np.testing.assert_allclose(H, fd, rtol=1e-5)


def test_gauss_newton_hessian_is_the_exact_hessian_at_a_noiseless_truth():
    """Where the residual vanishes (noise-free data at the true parameters) the Hessian of the
    profiled chi2_min(beta) is exactly the Gauss-Newton form 2 J^T N J: compared with central
    differences of the analytic gradient (itself pinned against differences of chi2_min). The
    off-diagonal blocks couple the parameters of patches that share pixels."""
    sk = S.make_sky(4, truth="uniform", hitcount=True)
    rng = np.random.default_rng(6)
    K = np.array([3, 2, 2])
    labels = np.stack([rng.integers(0, K[j], sk.npix) for j in range(3)]).astype(np.int64)
    for j in range(3):
        labels[j, :K[j]] = np.arange(K[j])
    beta = np.concatenate([np.full(K[0], 1.54), np.full(K[1], 20.0), np.full(K[2], -3.0)])
    d = sk.data(None)
    ninv = sk.ninv_pixel()
    H = lk.gauss_newton_hessian(NU, d, ninv, labels, K, beta)
    P = K.sum()
    fd = np.empty((P, P))
    for i in range(P):
        h = 1e-4 if K[0] <= i < K[0] + K[1] else 1e-5
        e = np.zeros(P)
        e[i] = h
        fd[:, i] = (lk.spectral_gradient(NU, d, ninv, labels, K, beta + e)[1] -
                    lk.spectral_gradient(NU, d, ninv, labels, K, beta - e)[1]) / (2 * h)
    np.testing.assert_allclose(H, 0.5 * (fd + fd.T), rtol=2e-5, atol=2e-6 * np.abs(H).max())
    assert np.allclose(H, H.T) and np.linalg.eigvalsh(H).min() > 0
    # its diagonal lies below the plain (unprojected) Gauss-Newton diagonal
    assert np.all(np.diag(H) <= lk.gauss_newton_diagonal(NU, d, ninv, labels, K, beta) * (1 + 1e-12))
