"""Pins of the pseudo-C_ell oracle (Sec. 2.5 residual spectra) against what the mathematics fixes:
a library routine for the spin-0 case, the closed form, orthonormality, the parity identity of
spin-weighted harmonics and the exact power of rotated pure-E / pure-B quadrupole patterns."""
import numpy as np
from scipy import special

from oracle import spectra as sp
from synth import healpix

THETA = np.array([0.05, 0.3, 1.1, 1.5707963, 2.0, 2.9])


def test_closed_form_spin0_is_scipy_sph_harm():
    for l in range(0, 11):
        for m in range(0, l + 1):
            ref = special.sph_harm_y(l, m, THETA, 0.0).real
            np.testing.assert_allclose(sp.goldberg(0, l, m, THETA), ref, rtol=0, atol=1e-12)


def test_recursion_matches_closed_form():
    for s in (2, -2):
        for m in range(0, 13):
            lam = sp.spin_lambda(s, m, THETA, 12)
            for l in range(0, 13):
                np.testing.assert_allclose(lam[l], sp.goldberg(s, l, m, THETA), rtol=0, atol=1e-11)


def test_spin2_functions_are_orthonormal():
    """2 pi int s_lambda_lm s_lambda_l'm sin(theta) dtheta = delta_ll' (Gauss-Legendre, exact for
    these polynomial products in cos(theta))."""
    x, w = np.polynomial.legendre.leggauss(100)
    t = np.arccos(x)
    for s in (2, -2):
        for m in (0, 1, 2, 3, 17, 60, 96):
            lam = sp.spin_lambda(s, m, t, 96)
            l0 = max(m, 2)
            G = 2.0 * np.pi * (lam * w) @ lam.T
            np.testing.assert_allclose(G[l0:, l0:], np.eye(97 - l0), rtol=0, atol=1e-11)
            assert not np.any(lam[:l0])


def test_parity_identity_relates_the_two_spins():
    """(-2)lambda_lm(theta) = (-1)^(l+m) (2)lambda_lm(pi - theta), every l <= 191."""
    for m in (0, 1, 2, 7, 100, 191):
        lp = sp.spin_lambda(2, m, np.pi - THETA, 191)
        lm = sp.spin_lambda(-2, m, THETA, 191)
        sign = (-1.0) ** (np.arange(192) + m)
        np.testing.assert_allclose(lm, sign[:, None] * lp, rtol=0, atol=1e-10)


def _quadrupole(nside, n0, mode):
    """Q, U of the pattern 2 sin^2(gamma) e^{2 i psi} (times i for B) around the axis n0: radial /
    tangential polarisation about an axis is pure E (45 degrees rotated: pure B), a pure l = 2
    field whose spectrum is rotation invariant: C_2 = 128 pi / 75 (|a_20|^2 / 5 about the axis,
    a_20 = 8 sqrt(2 pi / 15))."""
    z, phi = healpix.pixel_centres(nside)
    st = np.sqrt(1.0 - z * z)
    n = np.stack([st * np.cos(phi), st * np.sin(phi), z], 1)
    e_t = np.stack([z * np.cos(phi), z * np.sin(phi), -st], 1)
    e_p = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(z)], 1)
    cg = n @ n0
    sg = np.sqrt(np.maximum(1.0 - cg * cg, 0.0))
    e_g = (n * cg[:, None] - n0[None]) / sg[:, None]  # away from the axis
    psi = np.arctan2((e_g * e_p).sum(1), (e_g * e_t).sum(1))
    P = 2.0 * sg ** 2 * np.exp(2j * psi) * (1j if mode == "B" else 1.0)
    return np.stack([P.real, P.imag], 1)


def test_rotated_quadrupoles_are_pure_e_and_pure_b():
    nside = 16
    pix = np.arange(healpix.npix(nside))
    rng = np.random.default_rng(3)
    c2 = 128.0 * np.pi / 75.0
    for _ in range(2):
        n0 = rng.normal(size=3)
        n0 /= np.linalg.norm(n0)
        for k, mode in enumerate("EB"):
            cl = sp.pseudo_cl(nside, pix, _quadrupole(nside, n0, mode)[None], 10)[0]
            assert abs(cl[k, 2] / c2 - 1.0) < 1e-3          # pixel-quadrature error at nside 16
            assert cl[1 - k, 2] < 1e-10 * c2                 # no quadrupole in the other mode
            assert cl[1 - k].max() < 1e-5 * c2               # (pixel-quadrature aliasing only)
            assert np.abs(cl[k, 3:]).max() < 1e-5 * c2       # nor at other multipoles
            assert cl[k, 0] == 0.0 and cl[k, 1] == 0.0


def test_masked_spectrum_is_the_zero_filled_full_sky_spectrum():
    """The pseudo-spectrum of the observed pixels equals the full-sky spectrum of the map set to zero
    elsewhere; it is additive in nothing else, so a cut changes it."""
    nside = 8
    rng = np.random.default_rng(5)
    full = rng.normal(size=(healpix.npix(nside), 2))
    z, _ = healpix.pixel_centres(nside)
    pix = np.nonzero(np.abs(z) > 0.35)[0]
    zero = np.zeros_like(full)
    zero[pix] = full[pix]
    a = sp.pseudo_cl(nside, pix, full[pix][None], 23)[0]
    b = sp.pseudo_cl(nside, np.arange(healpix.npix(nside)), zero[None], 23)[0]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
    c = sp.pseudo_cl(nside, np.arange(healpix.npix(nside)), full[None], 23)[0]
    assert np.abs(a - c).max() > 1e-3 * c.max()


def test_residual_spectra_definitions():
    """tot / syst / stat are the averages over realizations of the spectra of s_hat - s_true,
    r_sys and their difference; with r_sys = 0 the statistical spectrum is the total one."""
    nside, lmax = 4, 11
    rng = np.random.default_rng(6)
    pix = np.arange(healpix.npix(nside))
    s_hat = rng.normal(size=(3, pix.size, 2))
    s_true = rng.normal(size=(pix.size, 2))
    r_sys = rng.normal(size=(3, pix.size, 2))
    out = sp.residual_spectra(nside, pix, s_hat, s_true, np.zeros_like(r_sys), lmax)
    np.testing.assert_allclose(out["stat"], out["tot"], rtol=1e-14)
    assert not np.any(out["syst"])
    out = sp.residual_spectra(nside, pix, s_hat, s_true, r_sys, lmax)
    one = sp.pseudo_cl(nside, pix, (s_hat - s_true[None] - r_sys), lmax)
    np.testing.assert_allclose(out["stat"], one.mean(axis=0), rtol=1e-14)
