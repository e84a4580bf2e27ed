"""Pins of the alternative partitions (inputs of the same fit): the HEALPix point-to-pixel map
against the pixel centres and the nested hierarchy, the latitude regions' sky fractions, the
multi-resolution configuration's patch structure, and the post-clustering binning."""
import numpy as np

from synth import healpix, partitions as pt


def test_ang2pix_ring_returns_each_pixel_for_its_centre():
    for nside in (1, 2, 4, 8, 16, 32):
        z, phi = healpix.pixel_centres(nside)
        assert np.array_equal(pt.ang2pix_ring(nside, z, phi), np.arange(z.size))


def test_ang2pix_ring_hierarchy_four_children():
    for nside in (1, 2, 4, 8, 16):
        z, phi = healpix.pixel_centres(2 * nside)
        parent = pt.ang2pix_ring(nside, z, phi)
        assert np.all(np.bincount(parent, minlength=12 * nside * nside) == 4)


def test_latitude_regions_hold_their_sky_fractions():
    nside = 64  # rings quantise the bands: 0.5% at nside 64
    reg = pt.latitude_regions(nside, np.arange(healpix.npix(nside)))
    frac = np.bincount(reg[reg >= 0]) / healpix.npix(nside)
    np.testing.assert_allclose(frac, [0.2, 0.2, 0.2], atol=0.005)
    # hi-lat is the band farthest from the plane
    z, _ = healpix.pixel_centres(nside)
    assert np.abs(z[reg == 0]).min() > np.abs(z[reg == 1]).max()


def test_multires_patches():
    nside = 16
    reg = pt.latitude_regions(nside, np.arange(healpix.npix(nside)))
    pix = np.nonzero(reg >= 0)[0]
    levels = ((16, 16, 16), (0, 2, 4), (1, 1, 2))
    lab, K = pt.multires_labels(nside, pix, levels)
    r = reg[pix]
    # beta_d at the map's own N_side: one pixel per patch
    assert K[0] == pix.size and np.unique(lab[0]).size == pix.size
    # T_d at level 0 in hi-lat: one patch for the region
    assert np.unique(lab[1][r == 0]).size == 1
    z, phi = healpix.pixel_centres(nside)
    for j in (1, 2):
        for rr in range(3):
            lev = levels[j][rr]
            m = r == rr
            if lev == 0:
                continue
            sup = pt.ang2pix_ring(lev, z[pix[m]], phi[pix[m]])
            # a patch is one superpixel of the region, and each superpixel one patch
            for patch in np.unique(lab[j][m]):
                assert np.unique(sup[lab[j][m] == patch]).size == 1
            assert np.unique(lab[j][m]).size == np.unique(sup).size
    # patches never span two regions
    for j in range(3):
        for patch in np.unique(lab[j]):
            assert np.unique(r[lab[j] == patch]).size == 1


def test_binned_labels():
    nside = 8
    vec = healpix.unit_vectors(nside)
    # a constant map stays constant under smoothing: one patch
    lab, K = pt.binned_labels(np.full(vec.shape[0], 1.7), vec, 10)
    assert K == 1 and np.all(lab == 0)
    # a map monotone in z: bins follow the smoothed values, at most nbin patches
    vals = vec[:, 2] * 0.3 + 1.5
    lab, K = pt.binned_labels(vals, vec, 6, fwhm_deg=10.0)
    sm = pt.smooth_on_sphere(vals, vec, 10.0)
    assert 2 <= K <= 6
    lo, hi = sm.min(), sm.max()
    expect = np.minimum(((sm - lo) / (hi - lo) * 6).astype(int), 5)
    # equal-width intervals of the smoothed map: the same partition as the interval index
    for b in np.unique(expect):
        assert np.unique(lab[expect == b]).size == 1
    assert np.unique(expect).size == K
    # a very narrow kernel leaves the map unchanged
    np.testing.assert_allclose(pt.smooth_on_sphere(vals, vec, 0.01), vals, rtol=0, atol=1e-12)
