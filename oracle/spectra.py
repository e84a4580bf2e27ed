"""Oracle: pseudo-C_ell spectra of polarisation residual maps (Sec. 2.5: the systematic residual
spectrum C_ell^syst = C_ell^BB([W d_fg]_CMB), the statistical one C_ell^stat = < C_ell^BB(
[s_hat^(n) - s_true] - [W d_fg]_CMB) >_n and the total < C_ell^BB(s_hat^(n) - s_true) >_n, taken as
pseudo-spectra of the masked residual maps), in FP64 (test infrastructure only).

The paper relies on the HEALPix conventions without restating them; the readings used here:
  - spin-weighted harmonics sY_lm in the closed form of Goldberg et al. (1967),
        sY_lm(theta, phi) = (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)] sin^{2l}(theta/2)
                            sum_r C(l-s, r) C(l+s, r+s-m) (-1)^(l-r-s) cot^(2r+s-m)(theta/2) e^{i m phi},
    and sY_lm = s_lambda_lm(theta) e^{i m phi};
  - polarisation (Zaldarriaga & Seljak 1997): (Q +- iU)(n) = sum a_{+-2,lm} (+-2)Y_lm(n),
    a^E = -(a_2 + a_-2) / 2, a^B = i (a_2 - a_-2) / 2;
  - analysis on the pixel grid with equal weights: a_{+-2,lm} = (4 pi / N_pix) sum_p (Q +- iU)_p
    conj((+-2)Y_lm(n_p)) over the observed pixels only, i.e. the map is zero off the mask (the
    pseudo-spectrum; the f_sky correction belongs to the r-likelihood, out of scope);
  - C_l = (1 / (2l + 1)) sum_{m=-l..l} |a_lm|^2 = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1) for
    real maps; l = 0, 1 carry no spin-2 power and are zero.
s_lambda_lm for l > l0 = max(m, |s|) follows from the three-term relation of cos(theta) in the
orthonormal basis of fixed (s, m),
    cos(theta) s_lambda_l = a_l s_lambda_{l+1} + b_l s_lambda_l + a_{l-1} s_lambda_{l-1},
    a_l = sqrt(((l+1)^2 - m^2)((l+1)^2 - s^2) / ((l+1)^2 (2l+1)(2l+3))),  b_l = -m s / (l (l+1)),
solved upward from the closed form at l0 (a single term of the sum there).

Parity pins (tests/test_oracle_spectra.py): the closed form against scipy's spherical harmonics
for s = 0; the recursion against the closed form (exact integer coefficients) for l <= 12;
orthonormality on Gauss-Legendre nodes up to l = 96; the parity identity
(-s)lambda_lm(theta) = (-1)^(l+m) s_lambda_lm(pi - theta) at every l, m; the power of rotated pure-E
and pure-B quadrupole patterns (128 pi / 75 in C_2, none elsewhere, none in the other mode).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from synth import healpix


def goldberg(s: int, l: int, m: int, theta) -> np.ndarray:
    """s_lambda_lm(theta) from the closed form (exact integer coefficients, FP64 powers)."""
    theta = np.asarray(theta, dtype=np.float64)
    if l < abs(s) or l < abs(m):
        return np.zeros_like(theta)
    pre = Fraction(math.factorial(l + m) * math.factorial(l - m) * (2 * l + 1),
                   math.factorial(l + s) * math.factorial(l - s))
    lpre = 0.5 * (math.log(pre.numerator) - math.log(pre.denominator) - math.log(4.0 * math.pi))
    ls, lc = np.log(np.sin(0.5 * theta)), np.log(np.cos(0.5 * theta))
    out = np.zeros_like(theta)
    for r in range(0, l - s + 1):
        k = r + s - m
        if k < 0 or k > l + s:
            continue
        c = math.comb(l - s, r) * math.comb(l + s, k) * (-1) ** ((l - r - s) & 1)
        e = 2 * r + s - m  # power of cot(theta/2): sin^(2l - e) cos^e
        out += c * np.exp(lpre + (2 * l - e) * ls + e * lc)
    return (-1) ** (m & 1) * out


def spin_lambda(s: int, m: int, theta, lmax: int) -> np.ndarray:
    """s_lambda_lm(theta) for l = 0 .. lmax (rows; zero below l0) by the upward recursion."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.zeros((lmax + 1,) + theta.shape)
    l0 = max(m, abs(s))
    if l0 > lmax:
        return out
    x = np.cos(theta)
    out[l0] = goldberg(s, l0, m, theta)

    def a(l):
        n = (l + 1) ** 2
        return math.sqrt((n - m * m) * (n - s * s) / (n * (2 * l + 1) * (2 * l + 3)))

    prev = np.zeros_like(theta)
    for l in range(l0, lmax):
        b = -m * s / (l * (l + 1)) if m * s else 0.0
        nxt = ((x - b) * out[l] - (a(l - 1) if l > l0 else 0.0) * prev) / a(l)
        prev = out[l]
        out[l + 1] = nxt
    return out


def alm_eb(nside: int, pix, Q, U, lmax: int):
    """a^E_lm, a^B_lm (complex [lmax+1][lmax+1], index [l][m], m >= 0) of maps given on the RING
    pixels `pix` (zero elsewhere). Q, U: [npix_obs] or [nmaps][npix_obs] (then leading axis kept)."""
    z, phi = healpix.pixel_centres(nside)
    pix = np.asarray(pix)
    theta_u, inv = np.unique(np.arccos(z[pix]), return_inverse=True)  # one row per ring
    ph = phi[pix]
    Q = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    w = 4.0 * np.pi / healpix.npix(nside)
    pp, pm = Q + 1j * U, Q - 1j * U  # [nmaps][npix_obs]
    aE = np.zeros((Q.shape[0], lmax + 1, lmax + 1), dtype=np.complex128)
    aB = np.zeros_like(aE)
    for m in range(lmax + 1):
        e = np.exp(-1j * m * ph)
        lp = spin_lambda(2, m, theta_u, lmax)[:, inv]   # [l][npix_obs]
        lm = spin_lambda(-2, m, theta_u, lmax)[:, inv]
        a2 = w * (pp * e) @ lp.T                        # [nmaps][l]
        am2 = w * (pm * e) @ lm.T
        aE[:, :, m] = -0.5 * (a2 + am2)
        aB[:, :, m] = 0.5j * (a2 - am2)
    return aE, aB


def cl_from_alm(alm) -> np.ndarray:
    """C_l = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l + 1) over the last two axes [l][m]."""
    lmax = alm.shape[-2] - 1
    p = np.abs(alm) ** 2
    tot = p[..., 0] + 2.0 * p[..., 1:].sum(axis=-1)
    return tot / (2.0 * np.arange(lmax + 1) + 1.0)


def pseudo_cl(nside: int, pix, maps, lmax: int) -> np.ndarray:
    """(EE, BB) pseudo-spectra [nmaps][2][lmax+1] of maps [nmaps][npix_obs][2] (Q, U)."""
    maps = np.asarray(maps, dtype=np.float64)
    aE, aB = alm_eb(nside, pix, maps[..., 0], maps[..., 1], lmax)
    return np.stack([cl_from_alm(aE), cl_from_alm(aB)], axis=1)


def residual_spectra(nside: int, pix, s_hat_cmb, s_true, r_sys, lmax: int):
    """The residual spectra of one configuration over its noise realizations n (Sec. 2.5):
    s_hat_cmb [nreal][npix_obs][2], s_true [npix_obs][2], r_sys [nreal][npix_obs][2] (the
    foreground leakage [W d_fg]_CMB at each realization's fitted parameters). Returns a dict of
    [2][lmax+1] (EE, BB) arrays: 'tot' = < C(s_hat - s_true) >_n, 'syst' = < C(r_sys) >_n (one
    map when the parameters do not depend on n), 'stat' = < C(s_hat - s_true - r_sys) >_n."""
    s_hat_cmb = np.asarray(s_hat_cmb, dtype=np.float64)
    res = s_hat_cmb - np.asarray(s_true, dtype=np.float64)[None]
    r_sys = np.asarray(r_sys, dtype=np.float64)
    return {"tot": pseudo_cl(nside, pix, res, lmax).mean(axis=0),
            "syst": pseudo_cl(nside, pix, r_sys, lmax).mean(axis=0),
            "stat": pseudo_cl(nside, pix, res - r_sys, lmax).mean(axis=0)}
