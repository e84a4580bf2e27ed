"""Named, seeded synthetic workloads with the shapes of the paper's experiments (Sec. 4):
LiteBIRD-like 15-band Q/U maps at nside 8 .. 128, K-means patch configurations, noise realizations.

Each workload is a plain bundle of arrays. Nothing here evaluates the component-separation method.

Seeds: sky amplitudes 1, truth fields 2 (+10, +20 for T_d and beta_s), K-means 100 + K,
configuration draw 4, noise realization n -> 1000 + n.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import healpix, kmeans, sky as skymod

# Start point and box bounds of the fit (beta_d, T_d [K], beta_s).
BETA0 = (1.5, 19.0, -2.9)
LOWER = (0.5, 5.0, -5.0)
UPPER = (3.0, 60.0, -1.0)


@dataclass
class Workload:
    name: str
    sky: skymod.Sky
    K: np.ndarray               # int32 [C, 3] patches per parameter (beta_d, T_d, beta_s)
    labels: np.ndarray          # int32 [C, 3, npix]
    nreal: int
    noise_kind: str             # "homogeneous" | "separable"
    first_real: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nconf(self):
        return self.K.shape[0]

    @property
    def npix(self):
        return self.sky.npix

    @property
    def P(self):
        return self.K.sum(axis=1)

    def data(self) -> np.ndarray:
        """float32 [nreal, npix, 2, 16]."""
        return self.sky.data_stack(self.nreal, self.first_real)

    def data64(self, r: int) -> np.ndarray:
        """float64 [npix, 2, F] noisy data of realization index r (0-based within the workload)."""
        return self.sky.data(self.first_real + r)

    def foreground_padded(self) -> np.ndarray:
        return self.sky.padded(self.sky.foreground)

    def ninv_band(self) -> np.ndarray:
        return self.sky.ninv_band

    def weights(self) -> np.ndarray:
        return self.sky.w

    def beta0(self, c: int) -> np.ndarray:
        """Start vector of configuration c, packed [beta_d x K_d | T_d x K_T | beta_s x K_s]."""
        k = self.K[c]
        return np.concatenate([np.full(k[j], BETA0[j]) for j in range(3)])


def sample_patch_counts(nconf: int, kmax: int, seed: int = 4) -> np.ndarray:
    """K per parameter drawn log-uniformly in [1, kmax]: round(exp(U[0, ln kmax]))."""
    rng = np.random.default_rng(seed)
    k = np.rint(np.exp(rng.uniform(0.0, np.log(kmax), size=(nconf, 3))))
    return np.clip(k, 1, kmax).astype(np.int64)


def _labels_for(vec, kreq: np.ndarray, key: str):
    table = kmeans.many_patch_labels(vec, kreq.ravel(), key=key)
    C = kreq.shape[0]
    labels = np.empty((C, 3, vec.shape[0]), dtype=np.int32)
    K = np.empty((C, 3), dtype=np.int32)
    for c in range(C):
        for j in range(3):
            lab = table[int(kreq[c, j])]
            labels[c, j] = lab
            K[c, j] = int(lab.max()) + 1
    return K, labels


def plain(nside: int = 8) -> Workload:
    """Uniform truth, homogeneous noise, one patch per parameter, one realization."""
    sk = skymod.make_sky(nside, truth="uniform", hitcount=False)
    labels = np.zeros((1, 3, sk.npix), dtype=np.int32)
    return Workload("plain_nside%d" % nside, sk, np.ones((1, 3), np.int32), labels, 1, "homogeneous")


def fullsky(nside: int = 64, K=(100, 20, 30), nreal: int = 100) -> Workload:
    """Full sky, smooth truth, hit-count noise, one K-means configuration, nreal realizations."""
    sk = skymod.make_sky(nside, truth="smooth", hitcount=True)
    vec = healpix.unit_vectors(nside)
    Kc, labels = _labels_for(vec, np.array([K]), key="full%d" % nside)
    return Workload("fullsky_nside%d" % nside, sk, Kc, labels, nreal, "separable")


def scan(nside: int = 64, nconf: int = 1000, kmax: int = 500, nreal: int = 10,
         b_cut_deg: float = 20.0, seed: int = 4) -> Workload:
    """Galactic cut |b| > b_cut, smooth truth, hit-count noise; nconf configurations with K per
    parameter log-uniform in [1, kmax]; nreal realizations shared by all configurations."""
    pix = healpix.galactic_cut(nside, b_cut_deg)
    sk = skymod.make_sky(nside, pix=pix, truth="smooth", hitcount=True)
    vec = healpix.unit_vectors(nside)[pix]
    kreq = sample_patch_counts(nconf, kmax, seed)
    Kc, labels = _labels_for(vec, kreq, key="cut%d_%g" % (nside, b_cut_deg))
    name = "scan_nside%d_b%g_C%d_K%d_R%d" % (nside, b_cut_deg, nconf, kmax, nreal)
    return Workload(name, sk, Kc, labels, nreal, "separable", meta={"K_requested": kreq})


def scan_subset(configs, nside: int = 64, nconf: int = 4000, kmax: int = 1000, nreal: int = 1,
                b_cut_deg: float = 20.0, seed: int = 4) -> Workload:
    """The configurations `configs` (indices into the K sample of scan(nside, nconf, kmax, seed))
    of that scan, alone: same sky, same K draws and the same K-means labelings, without forming the
    other configurations' labels (the full-pipeline scan has 4000 configurations)."""
    pix = healpix.galactic_cut(nside, b_cut_deg)
    sk = skymod.make_sky(nside, pix=pix, truth="smooth", hitcount=True)
    vec = healpix.unit_vectors(nside)[pix]
    kreq = sample_patch_counts(nconf, kmax, seed)[np.asarray(configs, dtype=np.int64)]
    Kc, labels = _labels_for(vec, kreq, key="cut%d_%g" % (nside, b_cut_deg))
    name = "scan_nside%d_b%g_C%d_K%d_subset%s" % (nside, b_cut_deg, nconf, kmax,
                                                 "-".join(str(int(c)) for c in configs))
    return Workload(name, sk, Kc, labels, nreal, "separable",
                    meta={"K_requested": kreq, "configs": list(configs)})


def gradcheck(nside: int = 128, K=(256, 256, 256), npoints: int = 64) -> Workload:
    """Full sky at nside 128, smooth truth, hit-count noise, K = 256 per parameter; one realization."""
    w = fullsky(nside, K, nreal=1)
    w.name = "gradcheck_nside%d" % nside
    w.meta["npoints"] = npoints
    return w


def random_points(K: np.ndarray, npoints: int, seed: int = 3) -> np.ndarray:
    """Random beta vectors (float64 [npoints, P]): beta_d ~ U[1.3, 1.8], T_d ~ U[15, 30],
    beta_s ~ U[-3.3, -2.7], independently per patch."""
    rng = np.random.default_rng(seed)
    lo = (1.3, 15.0, -3.3)
    hi = (1.8, 30.0, -2.7)
    cols = [rng.uniform(lo[j], hi[j], size=(npoints, int(K[j]))) for j in range(3)]
    return np.concatenate(cols, axis=1)
