"""Pins of the AdaTopK oracle (App. A): the release rule, the active set on a box-constrained
quadratic with a known minimiser, invariance under the dynamic rescaling, and agreement with the
library L-BFGS-B optimum on the plain nside-8 likelihood."""
import numpy as np

from oracle import adatopk as at
from oracle import fit as ofit
from synth import workloads


def test_release_rule_top_k():
    p = np.array([-1, -1, 1, 1, 0, -1])
    g = np.array([-2.0, 3.0, 5.0, -1.0, 7.0, 3.0])  # scores p*g: 2, -3, 5, -1, 0, -3
    # K = 0: only the single highest positive score (index 2) is released
    q, n = at.release(p, g, 0.0)
    assert n == 1 and q.tolist() == [-1, -1, 0, 1, 0, -1]
    # K = 1: every positive score (indices 0 and 2); a constraint pushed outward stays
    q, n = at.release(p, g, 1.0)
    assert n == 2 and q.tolist() == [0, -1, 0, 1, 0, -1]
    # ties: the lowest index first
    q, n = at.release(np.array([1, 1]), np.array([4.0, 4.0]), 0.0)
    assert n == 1 and q.tolist() == [0, 1]
    # nothing positive: nothing released
    q, n = at.release(np.array([-1, 1]), np.array([1.0, -1.0]), 0.0)
    assert n == 0 and q.tolist() == [-1, 1]


def _quad(a, c):
    return lambda y: (0.5 * np.sum(a * (y - c) ** 2), a * (y - c))


def test_box_quadratic_reaches_the_clipped_minimiser():
    # separable quadratic: the box minimiser is clip(c, 0, 1) (two coordinates end on bounds)
    a = np.array([1.0, 10.0, 100.0, 0.5, 3.0])
    c = np.array([0.3, 1.4, -0.2, 0.7, 0.55])
    y, f, info = at.minimize(_quad(a, c), np.full(5, 0.5), np.full(5, 1e-7), max_iter=5000)
    assert info["status"] == 0
    np.testing.assert_allclose(y, np.clip(c, 0.0, 1.0), atol=1e-5)
    assert y[1] == 1.0 and y[2] == 0.0  # clamped exactly by the step limit


def test_start_on_a_bound_is_released_when_pushed_inward():
    # start with every coordinate on a bound; the minimiser is interior for the first two
    a = np.array([2.0, 2.0, 2.0])
    c = np.array([0.4, 0.6, -0.5])
    y, f, info = at.minimize(_quad(a, c), np.array([0.0, 1.0, 0.0]), np.full(3, 1e-7),
                             max_iter=5000)
    np.testing.assert_allclose(y, [0.4, 0.6, 0.0], atol=1e-5)


def test_dynamic_rescaling_keeps_the_minimiser():
    a = np.array([1.0, 10.0, 100.0])
    c = np.array([0.3, 0.8, 0.1])
    big = lambda y: tuple(1e20 * v for v in _quad(a, c)(y))
    y1, _, i1 = at.minimize(_quad(a, c), np.full(3, 0.5), np.full(3, 1e-7), max_iter=5000)
    y2, _, i2 = at.minimize(big, np.full(3, 0.5), np.full(3, 1e-7), max_iter=5000)
    assert i1["scale"] == 1.0 and i2["scale"] < 1e-18  # the rescaling fired for the large objective
    np.testing.assert_allclose(y2, c, atol=1e-5)
    np.testing.assert_allclose(y1, c, atol=1e-5)


def test_plain_likelihood_matches_the_library_optimum():
    wl = workloads.plain(8)
    sk = wl.sky
    d = sk.data(0)
    ninv = np.broadcast_to(sk.ninv_band, (sk.npix, sk.nfreq)).copy()
    args = (sk.nu, d, ninv, wl.labels[0], wl.K[0], wl.beta0(0), workloads.LOWER, workloads.UPPER)
    x, L, info = at.fit(*args)
    xr, Lr, _ = ofit.fit(*args)
    assert info["status"] == 0
    assert np.all(np.abs(x - xr) <= 0.5 * np.array([1e-3, 1e-2, 1e-3])), (x, xr)
    assert L >= Lr - 1e-9 * abs(Lr) and L - Lr <= 1e-6 * abs(Lr)


def test_adabelief_two_steps_by_hand():
    """AdaBelief (Zhuang et al. 2020) with bias correction, worked by hand for two steps of a
    two-component gradient, beta1 = 0.9, beta2 = 0.999 (eps = 1e-16 is far below these digits):
      component A, g = 1 then 3:
        m1 = 0.1, s1 = 0.001 (1 - 0.1)^2 = 8.1e-4; m_hat = 1, s_hat = 0.81  ->  d1 = -1 / 0.9 = -10/9
        m2 = 0.09 + 0.3 = 0.39, s2 = 0.999 * 8.1e-4 + 0.001 (3 - 0.39)^2 = 7.62129e-3;
        m_hat = 0.39 / 0.19 = 39/19, s_hat = 7.62129e-3 / 1.999e-3  ->  d2 = -(39/19) / sqrt(762129/199900)
      component B, g = -2 then 0:
        m1 = -0.2, s1 = 0.001 (1.8)^2 = 3.24e-3  ->  d1 = 2 / 1.8 = 10/9
        m2 = -0.18, s2 = 0.999 * 3.24e-3 + 0.001 (0.18)^2 = 3.26916e-3  ->  d2 = (18/19) / sqrt(326916/199900)
    Adam's g^2 in place of (g - m)^2 gives -1 and -0.918 for component A, and dropping the bias
    correction gives d1 = -0.1 / sqrt(8.1e-4) = -3.51: both fail here."""
    m = np.zeros(2)
    s = np.zeros(2)
    d1, m, s = at.adabelief(np.array([1.0, -2.0]), m, s, 1)
    np.testing.assert_allclose(d1, [-10.0 / 9.0, 10.0 / 9.0], rtol=1e-12)
    np.testing.assert_allclose(m, [0.1, -0.2], rtol=1e-12)
    np.testing.assert_allclose(s, [8.1e-4, 3.24e-3], rtol=1e-12)
    d2, m, s = at.adabelief(np.array([3.0, 0.0]), m, s, 2)
    np.testing.assert_allclose(m, [0.39, -0.18], rtol=1e-12)
    np.testing.assert_allclose(s, [7.62129e-3, 3.26916e-3], rtol=1e-12)
    np.testing.assert_allclose(d2, [-(39.0 / 19.0) / np.sqrt(762129.0 / 199900.0),
                                    (18.0 / 19.0) / np.sqrt(326916.0 / 199900.0)], rtol=1e-12)
