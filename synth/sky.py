"""Seeded synthetic LiteBIRD-like polarised skies (stand-in for the paper's PySM3 simulations,
Sec. 4): instrument, white noise, hit-count weights, smooth truth fields and the noisy
multi-frequency Q/U maps.

This is a sky *simulator*, the role PySM plays for the paper. It evaluates emission laws in
physical form (Planck's law B_nu(T), Rayleigh-Jeans brightness, dB/dT at T_CMB) to produce
the data d_p = sum_c (emission of component c at each band) + n_p (Eq. 1); it computes none of the
component-separation steps (no mixing matrix in the paper's normalised form, no normal
equations, no solves, likelihood, gradient, fit or reconstruction).

Units: every map is in micro-K_CMB (thermodynamic), bands in GHz.
"""
from __future__ import annotations

import numpy as np

from . import healpix

# LiteBIRD-like instrument: band centres (GHz) and polarisation depths (uK.arcmin).
BANDS_GHZ = np.array([40, 50, 60, 68, 78, 89, 100, 119, 140, 166, 195, 235, 280, 337, 402],
                     dtype=np.float64)
DEPTH_UK_ARCMIN = np.array([37.4, 33.5, 21.3, 19.9, 15.6, 12.3, 11.7, 8.3, 6.6, 6.4, 7.2, 10.8,
                            13.6, 21.5, 46.0], dtype=np.float64)

# Physical constants of the simulator (SI, exact CODATA-2019 values for h, k and c).
PLANCK_H = 6.62607015e-34
BOLTZMANN_K = 1.380649e-23
LIGHT_C = 299792458.0
T_CMB_K = 2.7255

# Fiducial foreground parameters and amplitude reference frequencies.
BETA_D0, TEMP_D0, BETA_S0 = 1.54, 20.0, -3.0
NU_REF_DUST, NU_REF_SYNC = 353.0, 23.0

# North ecliptic pole in Galactic coordinates (l, b) in degrees.
NEP_L_DEG, NEP_B_DEG = 96.384, 29.811

PADDED_BANDS = 16  # one 128-byte line per pixel and Stokes pair: [2][16] float32


def planck_intensity(nu_ghz, temp_k):
    """Planck's law B_nu(T) in W m^-2 Hz^-1 sr^-1."""
    nu = np.asarray(nu_ghz, dtype=np.float64) * 1e9
    x = PLANCK_H * nu / (BOLTZMANN_K * np.asarray(temp_k, dtype=np.float64))
    return 2.0 * PLANCK_H * nu ** 3 / LIGHT_C ** 2 / np.expm1(x)


def rj_intensity_per_kelvin(nu_ghz):
    """Intensity of a 1 K Rayleigh-Jeans brightness temperature: 2 k nu^2 / c^2."""
    nu = np.asarray(nu_ghz, dtype=np.float64) * 1e9
    return 2.0 * BOLTZMANN_K * nu ** 2 / LIGHT_C ** 2


def cmb_intensity_per_kelvin(nu_ghz):
    """dB_nu/dT at T_CMB: intensity of a 1 K thermodynamic (K_CMB) fluctuation."""
    nu = np.asarray(nu_ghz, dtype=np.float64) * 1e9
    x = PLANCK_H * nu / (BOLTZMANN_K * T_CMB_K)
    ex = np.exp(x)
    return 2.0 * PLANCK_H * nu ** 3 / LIGHT_C ** 2 * (x / T_CMB_K) * ex / np.expm1(x) ** 2


def dust_kcmb(nu_ghz, amp_rj_ref, beta_d, temp_d):
    """Modified-blackbody dust in uK_CMB at nu, for a polarised amplitude given in uK_RJ at 353 GHz.

    Intensity I(nu) = I(353) * (nu/353)^beta_d * B_nu(T_d) / B_353(T_d), converted to K_CMB at nu."""
    i_ref = rj_intensity_per_kelvin(NU_REF_DUST) * amp_rj_ref
    shape = (np.asarray(nu_ghz) / NU_REF_DUST) ** beta_d * planck_intensity(nu_ghz, temp_d) / \
        planck_intensity(NU_REF_DUST, temp_d)
    return i_ref * shape / cmb_intensity_per_kelvin(nu_ghz)


def sync_kcmb(nu_ghz, amp_rj_ref, beta_s):
    """Power-law synchrotron in uK_CMB at nu, amplitude in uK_RJ at 23 GHz: T_RJ ∝ nu^beta_s."""
    t_rj = amp_rj_ref * (np.asarray(nu_ghz) / NU_REF_SYNC) ** beta_s
    return t_rj * rj_intensity_per_kelvin(nu_ghz) / cmb_intensity_per_kelvin(nu_ghz)


def rj_to_kcmb(nu_ghz):
    """Factor converting a Rayleigh-Jeans temperature at nu to a K_CMB temperature."""
    return rj_intensity_per_kelvin(nu_ghz) / cmb_intensity_per_kelvin(nu_ghz)


def white_noise_sigma(nside: int) -> np.ndarray:
    """Per-pixel noise rms per band (uK_CMB): depth / pixel side, pixel side = sqrt(pixel area)."""
    return DEPTH_UK_ARCMIN / np.sqrt(healpix.pixel_solid_angle_arcmin2(nside))


def hitcount_weights(nside: int, pix: np.ndarray) -> np.ndarray:
    """w_p = h_p / mean_full_sky(h), h = 1 + 0.5 cos^2(ecliptic latitude); N^-1_{p,f} = w_p / sigma_f^2."""
    vec = healpix.unit_vectors(nside)
    l, b = np.deg2rad(NEP_L_DEG), np.deg2rad(NEP_B_DEG)
    nep = np.array([np.cos(b) * np.cos(l), np.cos(b) * np.sin(l), np.sin(b)])
    sin_ecl = vec @ nep
    h = 1.0 + 0.5 * (1.0 - sin_ecl ** 2)
    return (h[pix] / h.mean()).astype(np.float64)


def smooth_field(nside: int, pix: np.ndarray, rms: float, seed: int, fwhm_deg: float = 10.0):
    """Seeded smooth Gaussian random field on the pixels `pix`: white noise on nside-16 pixel
    centres convolved with a Gaussian beam of the given FWHM, rescaled to exact rms (zero mean)."""
    rng = np.random.default_rng(seed)
    src = healpix.unit_vectors(16)
    amp = rng.standard_normal(src.shape[0])
    tgt = healpix.unit_vectors(nside)[pix]
    sigma = np.deg2rad(fwhm_deg) / np.sqrt(8.0 * np.log(2.0))
    out = np.empty(tgt.shape[0])
    for s in range(0, tgt.shape[0], 4096):
        cosang = np.clip(tgt[s:s + 4096] @ src.T, -1.0, 1.0)
        ang = np.arccos(cosang)
        out[s:s + 4096] = np.exp(-0.5 * (ang / sigma) ** 2) @ amp
    out -= out.mean()
    out *= rms / np.sqrt(np.mean(out ** 2))
    return out


def polarised_amplitudes(rng, n, median):
    """Q, U of a lognormal polarised amplitude (median given, sigma_ln = 0.5) at a uniform angle."""
    p = median * np.exp(0.5 * rng.standard_normal(n))
    psi = rng.uniform(0.0, np.pi, n)
    return p * np.cos(2 * psi), p * np.sin(2 * psi)


class Sky:
    """A simulated sky on the pixel subset `pix` of an nside map.

    Attributes (float64 unless noted):
      nu [F], sigma [F] (noise rms per band, uK_CMB), w [npix] (hit-count weights, 1 if homogeneous),
      beta_true [npix, 3] (beta_d, T_d, beta_s per pixel),
      cmb [npix, 2] (Q, U, uK_CMB), dust_amp / sync_amp [npix, 2] (uK_RJ at 353 / 23 GHz),
      signal [npix, 2, F] (noise-free data), foreground [npix, 2, F] (noise-free dust+sync only).
    """

    def __init__(self, nside, pix, beta_true, cmb, dust_amp, sync_amp, w):
        self.nside = nside
        self.pix = np.asarray(pix, dtype=np.int64)
        self.npix = self.pix.size
        self.nu = BANDS_GHZ.copy()
        self.nfreq = self.nu.size
        self.sigma = white_noise_sigma(nside)
        self.w = np.asarray(w, dtype=np.float64)
        self.beta_true = beta_true
        self.cmb = cmb
        self.dust_amp = dust_amp
        self.sync_amp = sync_amp
        nu = self.nu[None, None, :]
        bd = beta_true[:, 0][:, None, None]
        td = beta_true[:, 1][:, None, None]
        bs = beta_true[:, 2][:, None, None]
        dust = dust_kcmb(nu, dust_amp[:, :, None], bd, td)
        sync = sync_kcmb(nu, sync_amp[:, :, None], bs)
        self.foreground = dust + sync
        self.signal = self.foreground + cmb[:, :, None]

    @property
    def ninv_band(self):
        """Per-band inverse noise variance 1/sigma_f^2 for w = 1."""
        return 1.0 / self.sigma ** 2

    def ninv_pixel(self):
        """N^-1 per pixel and band, [npix, F] = w_p / sigma_f^2."""
        return self.w[:, None] / self.sigma[None, :] ** 2

    def noise(self, realization: int) -> np.ndarray:
        """Noise realization n (seed 1000 + n): [npix, 2, F] with rms sigma_f / sqrt(w_p)."""
        rng = np.random.default_rng(1000 + realization)
        g = rng.standard_normal((self.npix, 2, self.nfreq))
        return g * (self.sigma[None, None, :] / np.sqrt(self.w)[:, None, None])

    def data(self, realization=None) -> np.ndarray:
        """Noisy data [npix, 2, F]; realization None gives the noise-free signal."""
        if realization is None:
            return self.signal.copy()
        return self.signal + self.noise(realization)

    def data_stack(self, nreal: int, first: int = 0, padded: bool = True) -> np.ndarray:
        """float32 [nreal, npix, 2, 16] (band 15 zero) for realizations first .. first+nreal-1."""
        f = PADDED_BANDS if padded else self.nfreq
        out = np.zeros((nreal, self.npix, 2, f), dtype=np.float32)
        for r in range(nreal):
            out[r, :, :, :self.nfreq] = self.data(first + r)
        return out

    def padded(self, x: np.ndarray) -> np.ndarray:
        """Pad the band axis of a [..., F] array to 16 with zeros, as float32."""
        out = np.zeros(x.shape[:-1] + (PADDED_BANDS,), dtype=np.float32)
        out[..., :self.nfreq] = x
        return out


def make_sky(nside: int, pix=None, truth: str = "uniform", hitcount: bool = False,
             seed: int = 1, truth_seed: int = 2) -> Sky:
    """Build a seeded sky.

    truth: "uniform" (beta_d 1.54, T_d 20 K, beta_s -3 everywhere) or "smooth" (fiducial values
    plus seeded Gaussian random fields of rms 0.05, 1 K, 0.05 smoothed at 10 deg FWHM).
    Amplitudes: CMB Q/U ~ N(0, 0.5 uK_CMB); dust lognormal median 10 uK_RJ at 353 GHz;
    synchrotron lognormal median 5 uK_RJ at 23 GHz; polarisation angles uniform.
    """
    if pix is None:
        pix = np.arange(healpix.npix(nside))
    pix = np.asarray(pix, dtype=np.int64)
    n = pix.size
    rng = np.random.default_rng(seed)
    cmb = 0.5 * rng.standard_normal((n, 2))
    dq, du = polarised_amplitudes(rng, n, 10.0)
    sq, su = polarised_amplitudes(rng, n, 5.0)
    beta = np.empty((n, 3))
    if truth == "uniform":
        beta[:] = (BETA_D0, TEMP_D0, BETA_S0)
    elif truth == "smooth":
        beta[:, 0] = BETA_D0 + smooth_field(nside, pix, 0.05, truth_seed)
        beta[:, 1] = TEMP_D0 + smooth_field(nside, pix, 1.0, truth_seed + 10)
        beta[:, 2] = BETA_S0 + smooth_field(nside, pix, 0.05, truth_seed + 20)
    else:
        raise ValueError(truth)
    w = hitcount_weights(nside, pix) if hitcount else np.ones(n)
    return Sky(nside, pix, beta, cmb, np.stack([dq, du], 1), np.stack([sq, su], 1), w)
