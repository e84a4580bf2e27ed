"""Pins of the seeded spherical K-means patch generator (Sec. 2.2), which both the oracle's inputs and
the GPU K-means kernel's reference come from: what Lloyd's algorithm fixes (at the labels it returns,
every pixel's label maximises the dot product with its cluster's renormalised member mean), two
small cases worked by hand, and the K <= 1 / K >= n rules (Table 1 caption)."""
import numpy as np
import pytest

from synth import healpix, kmeans as km


def _centroid_dots(vec, lab):
    """Dot products of every pixel with every cluster's renormalised member mean."""
    k = int(lab.max()) + 1
    sums = np.stack([np.bincount(lab, weights=vec[:, c], minlength=k) for c in range(3)], 1)
    cent = sums / np.linalg.norm(sums, axis=1)[:, None]
    return vec @ cent.T


@pytest.mark.parametrize("nside,K,cut", [(4, 5, None), (4, 12, None), (8, 20, 20.0), (8, 40, None)])
def test_labels_are_a_lloyd_fixed_point(nside, K, cut):
    vec = healpix.unit_vectors(nside)
    if cut is not None:
        vec = vec[healpix.galactic_cut(nside, cut)]
    lab = km.spherical_kmeans(vec, K, seed=100 + K)
    # the run converged (the iteration cap did not stop it): more iterations change nothing
    np.testing.assert_array_equal(lab, km.spherical_kmeans(vec, K, seed=100 + K, max_iter=500))
    assert lab.min() == 0 and np.unique(lab).size == lab.max() + 1 <= K
    dots = _centroid_dots(vec, lab)
    own = dots[np.arange(vec.shape[0]), lab]
    assert np.all(own >= dots.max(axis=1) - 1e-12)
    # labels are numbered by first appearance
    _, first = np.unique(lab, return_index=True)
    assert np.all(np.diff(first) > 0)


def _six(order):
    base = {"a": (1.0, 0.1, 0.0), "b": (1.0, -0.1, 0.0), "c": (1.0, 0.0, 0.1),
            "d": (-1.0, 0.1, 0.0), "e": (-1.0, -0.1, 0.0), "f": (-1.0, 0.0, 0.1)}
    v = np.array([base[k] for k in order])
    return v / np.linalg.norm(v, axis=1)[:, None]


def test_six_points_worked_by_hand():
    """K = 2 on three points near +x (a, b, c) and three near -x (d, e, f); the seeded start pixels
    are indices 2 and 0 (init_indices(6, 2, 102)), cluster 0 starting at pixel 2.

    Order a b c d e f: both starts are +x points (c for cluster 0, a for cluster 1). With n = |v|^2 =
    1.01, the first assignment compares (x cx + y cy) + z cz: a -> 1 (1.01 vs 1), b -> 0 (1 vs
    0.99), c -> 0, d -> 1 (-0.99 vs -1), e -> 0 (-1 vs -1.01), f -> 0 (-0.99 vs -1). Member means:
    cluster 0 = {b, c, e, f} along (0, -1, 1), cluster 1 = {a, d} along (0, 1, 0); the next
    assignment repeats (a: -0.07 vs 0.1, b: 0.07 vs -0.1, c: 0.07 vs 0, d: -0.07 vs 0.1, ...), so
    Lloyd stops in this split, relabelled by first appearance: 0 1 1 0 1 1.

    Order a b d e c f: the starts are d (cluster 0) and a (cluster 1), one per side; the +x points
    join a and the -x points join d at once and stay: 1 1 0 0 1 0, relabelled 0 0 1 1 0 1."""
    assert list(km.init_indices(6, 2, 102)) == [2, 0]
    np.testing.assert_array_equal(km.spherical_kmeans(_six("abcdef"), 2, seed=102), [0, 1, 1, 0, 1, 1])
    np.testing.assert_array_equal(km.spherical_kmeans(_six("abdecf"), 2, seed=102), [0, 0, 1, 1, 0, 1])


def test_patch_count_limits():
    vec = _six("abcdef")
    for k in (0, 1):
        np.testing.assert_array_equal(km.spherical_kmeans(vec, k, seed=100 + k), np.zeros(6))
    for k in (6, 7, 50):
        np.testing.assert_array_equal(km.spherical_kmeans(vec, k, seed=100 + k), np.arange(6))
