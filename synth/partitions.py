"""Alternative patch partitions (inputs to the same fit): multi-resolution HEALPix superpixels per
Galactic region (the fixed configuration the paper compares K-means against, Sec. 4.3, table of
HEALPix N_side levels) and post-clustering binning of fitted spectral-parameter maps (Sec. 4.5).

The Planck Galactic masks that define the paper's regions are not available: the regions here are
latitude bands holding the same sky fractions (hi-lat: the 20% of the sky farthest from the plane,
mid-lat the next 20%, low-lat the next 20%). Smoothing for the binning is a direct-space Gaussian
on the sphere (the paper smooths with spherical harmonics). Generates inputs only.
"""
from __future__ import annotations

import numpy as np

from . import healpix

# Table "multi-resolution configuration" (N_side per region; 0 = one patch for the whole region,
# 64 = one patch per pixel at N_side 64): rows beta_d, T_d, beta_s; columns hi, mid, low latitude.
MULTIRES_LEVELS = ((64, 64, 64), (0, 4, 8), (2, 2, 4))
REGION_FSKY = (0.2, 0.4, 0.6)  # cumulative sky fractions closing hi, mid, low latitude


def ang2pix_ring(nside: int, z: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """RING index of the pixel containing each direction (z = cos theta, phi in [0, 2 pi)), from the
    HEALPix geometry (Gorski et al. 2005): equatorial belt |z| <= 2/3 by the two families of pixel
    edge lines, polar caps by the distance from the pole in sqrt(3 (1 - |z|)) units."""
    z = np.asarray(z, dtype=np.float64)
    phi = np.mod(np.asarray(phi, dtype=np.float64), 2.0 * np.pi)
    tt = phi / (0.5 * np.pi)  # in [0, 4)
    za = np.abs(z)
    pix = np.empty(z.shape, dtype=np.int64)
    eq = za <= 2.0 / 3.0
    # equatorial belt: edge lines of slope +-1 in (phi, z) measured in pixel units
    t1 = nside * (0.5 + tt[eq])
    t2 = nside * z[eq] * 0.75
    jp = np.floor(t1 - t2).astype(np.int64)  # ascending edge line index
    jm = np.floor(t1 + t2).astype(np.int64)  # descending edge line index
    ir = nside + 1 + jp - jm                 # ring counted from z = 2/3, 1 .. 2 nside + 1
    kshift = 1 - (ir & 1)
    ip = (jp + jm - nside + kshift + 1) // 2
    ip = np.mod(ip, 4 * nside)
    pix[eq] = 2 * nside * (nside - 1) + 4 * nside * (ir - 1) + ip
    # polar caps
    cap = ~eq
    tp = tt[cap] - np.floor(tt[cap])
    tmp = nside * np.sqrt(3.0 * (1.0 - za[cap]))
    jp = np.floor(tp * tmp).astype(np.int64)
    jm = np.floor((1.0 - tp) * tmp).astype(np.int64)
    ir = jp + jm + 1                              # ring counted from the nearer pole
    ip = np.mod(np.floor(tt[cap] * ir).astype(np.int64), 4 * ir)
    north = z[cap] > 0
    pix[cap] = np.where(north, 2 * ir * (ir - 1) + ip, 12 * nside * nside - 2 * ir * (ir + 1) + ip)
    return pix


def latitude_regions(nside: int, pix: np.ndarray, fsky=REGION_FSKY) -> np.ndarray:
    """Region of each pixel of `pix`: 0 hi-lat, 1 mid-lat, 2 low-lat, -1 outside (|b| bands holding
    the cumulative sky fractions `fsky`: |sin b| > 1 - f)."""
    z, _ = healpix.pixel_centres(nside)
    s = np.abs(z[pix])
    reg = np.full(pix.size, -1, dtype=np.int64)
    lo = 1.0
    for r, f in enumerate(fsky):
        hi_edge = lo
        lo = 1.0 - f
        reg[(s > lo) & (s <= hi_edge) & (reg < 0)] = r
    return reg


def _compact(keys: np.ndarray) -> np.ndarray:
    """Labels 0..K-1 numbered by first appearance of each distinct key."""
    _, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")
    rank = np.empty(order.size, dtype=np.int64)
    rank[order] = np.arange(order.size)
    return rank[inv].astype(np.int32)


def multires_labels(nside: int, pix: np.ndarray, levels=MULTIRES_LEVELS, fsky=REGION_FSKY):
    """Labels [3][len(pix)] (int32) and K [3] of the multi-resolution configuration on the pixels
    `pix` (RING, nside): per parameter and region, the superpixel at N_side `level` containing the
    pixel centre (0: one patch per region); patches never span two regions. Pixels outside every
    region must not be passed."""
    reg = latitude_regions(nside, pix, fsky)
    if np.any(reg < 0):
        raise ValueError("pixels outside the regions")
    z, phi = healpix.pixel_centres(nside)
    labels, K = [], []
    for j in range(3):
        sup = np.zeros(pix.size, dtype=np.int64)
        for r in range(len(fsky)):
            m = reg == r
            lev = levels[j][r]
            if lev > 0:
                sup[m] = ang2pix_ring(lev, z[pix[m]], phi[pix[m]])
        lab = _compact(reg * (12 * max(max(lv) for lv in levels) ** 2 + 1) + sup)
        labels.append(lab)
        K.append(int(lab.max()) + 1)
    return np.stack(labels).astype(np.int32), np.array(K, dtype=np.int32)


def smooth_on_sphere(values: np.ndarray, vec: np.ndarray, fwhm_deg: float, chunk: int = 1024):
    """Gaussian-weighted average of `values` over the pixels `vec` (unit vectors), kernel of the
    given FWHM truncated at 3 sigma: the direct-space stand-in for harmonic smoothing."""
    sig = np.deg2rad(fwhm_deg) / np.sqrt(8.0 * np.log(2.0))
    cmin = np.cos(3.0 * sig)
    out = np.empty(values.size)
    for s in range(0, vec.shape[0], chunk):
        dots = np.clip(vec[s:s + chunk] @ vec.T, -1.0, 1.0)
        w = np.where(dots >= cmin, np.exp(-np.arccos(dots) ** 2 / (2.0 * sig * sig)), 0.0)
        out[s:s + chunk] = (w @ values) / w.sum(axis=1)
    return out


def binned_labels(values: np.ndarray, vec: np.ndarray, nbin: int, fwhm_deg: float = 5.0):
    """Post-clustering binning: smooth the per-pixel map of a fitted parameter, cut its range into
    `nbin` equal-width intervals and make each non-empty interval a patch (possibly disconnected on
    the sky). Returns (labels int32, K)."""
    sm = smooth_on_sphere(np.asarray(values, dtype=np.float64), vec, fwhm_deg)
    lo, hi = sm.min(), sm.max()
    if hi - lo <= 1e-12 * max(abs(hi), abs(lo), 1.0):  # a constant map (up to rounding)
        return np.zeros(sm.size, dtype=np.int32), 1
    b = np.minimum(((sm - lo) / (hi - lo) * nbin).astype(np.int64), nbin - 1)
    lab = _compact(b)
    return lab, int(lab.max()) + 1
