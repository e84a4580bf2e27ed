"""HEALPix RING-ordered pixel centres, written from the geometry of Gorski et al. 2005
(the pixelisation the paper works on, Sec. 2.2 and Sec. 3.2).

The sphere is cut into 4*nside-1 iso-latitude rings. Counting rings i = 1 .. 4*nside-1 from the
north pole:

* north cap, i < nside: ring i holds 4*i pixels, cos(theta) = 1 - i^2 / (3 nside^2), and the
  pixel centres sit at phi = (pi / (2 i)) * (j + 1/2), j = 0 .. 4i-1;
* equatorial belt, nside <= i <= 3*nside: every ring holds 4*nside pixels,
  cos(theta) = (4/3) - 2 i / (3 nside); centres sit at phi = (pi / (2 nside)) * (j + shift) with
  shift = 1/2 when i + nside is even and 0 when it is odd;
* south cap mirrors the north cap.

Pixels are numbered ring by ring from the north pole, west to east inside a ring (RING order).
This module generates inputs only; it holds none of the component-separation arithmetic.
"""
from __future__ import annotations

import numpy as np


def npix(nside: int) -> int:
    return 12 * nside * nside


def ring_layout(nside: int):
    """Return per-ring (n_pixels, z, phi_offset_in_units_of_dphi, dphi) lists, north to south."""
    rings = []
    for i in range(1, 4 * nside):
        if i < nside:  # north cap
            n = 4 * i
            z = 1.0 - (i * i) / (3.0 * nside * nside)
            rings.append((n, z, 0.5, np.pi / (2.0 * i)))
        elif i <= 3 * nside:  # equatorial belt
            n = 4 * nside
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
            shift = 0.5 if ((i + nside) % 2 == 0) else 0.0
            rings.append((n, z, shift, np.pi / (2.0 * nside)))
        else:  # south cap, mirror of ring 4*nside - i
            k = 4 * nside - i
            n = 4 * k
            z = -(1.0 - (k * k) / (3.0 * nside * nside))
            rings.append((n, z, 0.5, np.pi / (2.0 * k)))
    return rings


def pixel_centres(nside: int):
    """(z, phi) of every pixel centre in RING order, float64 arrays of length 12*nside^2."""
    zs, phis = [], []
    for n, z, shift, dphi in ring_layout(nside):
        j = np.arange(n, dtype=np.float64)
        zs.append(np.full(n, z))
        phis.append(dphi * (j + shift))
    z = np.concatenate(zs)
    phi = np.concatenate(phis)
    assert z.size == npix(nside)
    return z, phi


def unit_vectors(nside: int) -> np.ndarray:
    """Pixel-centre unit vectors (x, y, z) = (cos b cos l, cos b sin l, sin b), shape [npix, 3].

    The maps are in Galactic coordinates, so z = sin(b) (b = Galactic latitude)."""
    z, phi = pixel_centres(nside)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def pixel_solid_angle_arcmin2(nside: int) -> float:
    """All HEALPix pixels have the same area 4 pi / (12 nside^2) sr; returned in arcmin^2."""
    sr = 4.0 * np.pi / npix(nside)
    arcmin_per_rad = 180.0 * 60.0 / np.pi
    return sr * arcmin_per_rad ** 2


def galactic_cut(nside: int, b_min_deg: float) -> np.ndarray:
    """Indices (RING order, ascending) of pixels with |b| > b_min_deg."""
    z, _ = pixel_centres(nside)
    return np.nonzero(np.abs(z) > np.sin(np.deg2rad(b_min_deg)))[0].astype(np.int64)
