"""GPU spherical K-means (csx_kmeans) against the input generator (synth.kmeans.spherical_kmeans):
labels bit-exact, for every cluster count at once, including the special counts (K <= 1, K >= n),
a configuration that empties clusters (duplicated points make tied centroids), and the cut-sky
nside-64 pixel set of the scan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import healpix, kmeans  # noqa: E402


@pytest.fixture(scope="module")
def csx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08463_b300 import csx as mod
    mod.lib()
    return mod


def _gpu_labels(csx, vec, ks):
    n = vec.shape[0]
    init = [kmeans.init_indices(n, k, 100 + k) for k in ks if 1 < k < n]
    it = iter(init)
    init_full = [next(it) if 1 < k < n else None for k in ks]
    lab, iters = csx.kmeans(torch.from_numpy(vec).to("cuda"), ks, [x for x in init_full if x is not None])
    torch.cuda.synchronize()
    return lab.cpu().numpy(), iters.cpu().numpy()


def test_kmeans_bit_exact_full_sky_nside16(csx):
    vec = healpix.unit_vectors(16)
    ks = [1, 2, 3, 7, 50, 200, 1000, 3072, 5000]
    lab, iters = _gpu_labels(csx, vec, ks)
    for i, k in enumerate(ks):
        ref = kmeans.spherical_kmeans(vec, k, seed=100 + k)
        assert np.array_equal(lab[i], ref), (k, np.count_nonzero(lab[i] != ref))
    assert iters.max() <= 30


def test_kmeans_bit_exact_emptied_clusters(csx):
    # 64 distinct directions, each repeated 4 times: centroids drawn on repeated points tie, the
    # later cluster loses every pixel and is re-seeded
    rng = np.random.default_rng(3)
    base = rng.normal(size=(64, 3))
    base /= np.linalg.norm(base, axis=1, keepdims=True)
    vec = np.repeat(base, 4, axis=0)
    ks = [20, 63, 100, 180]
    emptied = 0
    for k in ks:  # the generator must actually re-seed for this input to pin that step
        init = kmeans.init_indices(vec.shape[0], k, 100 + k)
        emptied += np.unique(np.argmax(vec @ vec[init].T, axis=1)).size < k
    assert emptied > 0
    lab, _ = _gpu_labels(csx, vec, ks)
    for i, k in enumerate(ks):
        ref = kmeans.spherical_kmeans(vec, k, seed=100 + k)
        assert np.array_equal(lab[i], ref), (k, np.count_nonzero(lab[i] != ref))


def test_kmeans_bit_exact_scan_pixels(csx):
    pix = healpix.galactic_cut(64, 20.0)
    vec = healpix.unit_vectors(64)[pix]
    ks = [5, 100, 500, 1500]
    lab, _ = _gpu_labels(csx, vec, ks)
    for i, k in enumerate(ks):
        ref = kmeans.spherical_kmeans(vec, k, seed=100 + k)
        assert np.array_equal(lab[i], ref), (k, np.count_nonzero(lab[i] != ref))
