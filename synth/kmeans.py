"""Seeded spherical K-means patches (Sec. 2.2): Lloyd iterations on pixel-centre unit vectors.

Assignment is by largest dot product with the centroid directions (smallest angular distance;
ties go to the lowest cluster index); a centroid is the renormalised mean of its members' unit
vectors. An emptied cluster is re-seeded at the pixel farthest from its own centroid. The loop stops
at a fixed point or after `max_iter` iterations; labels are then renumbered 0..K_eff-1 in order of
first appearance (K_eff <= K). K >= number of pixels gives one pixel per patch (the paper's rule when
the requested patch count exceeds the available pixels, Table 1 caption).

Used to generate inputs (cluster labels) only.
"""
from __future__ import annotations

import os

import numpy as np

_CACHE: dict = {}


def _assign(vec, cent, chunk=4096):
    """Label of the largest dot product (first on ties) and its value. The dot product is formed
    element by element as (x cx + y cy) + z cz, each product and sum rounded once in float64 (no
    fused multiply-add, no BLAS reordering), so that any implementation doing the same operations
    in the same order assigns identically."""
    lab = np.empty(vec.shape[0], dtype=np.int64)
    best = np.empty(vec.shape[0])
    for s in range(0, vec.shape[0], chunk):
        v = vec[s:s + chunk]
        dots = (v[:, 0:1] * cent[:, 0] + v[:, 1:2] * cent[:, 1]) + v[:, 2:3] * cent[:, 2]
        lab[s:s + chunk] = np.argmax(dots, axis=1)
        best[s:s + chunk] = dots[np.arange(dots.shape[0]), lab[s:s + chunk]]
    return lab, best


def init_indices(n: int, k: int, seed: int) -> np.ndarray:
    """The K distinct starting pixels of a labeling (seeded), as spherical_kmeans draws them."""
    return np.random.default_rng(seed).choice(n, size=k, replace=False)


def spherical_kmeans(vec: np.ndarray, k: int, seed: int, max_iter: int = 30) -> np.ndarray:
    """Labels (int32, contiguous from 0) of a seeded spherical K-means of unit vectors `vec`."""
    n = vec.shape[0]
    if k >= n:
        return np.arange(n, dtype=np.int32)
    if k <= 1:
        return np.zeros(n, dtype=np.int32)
    cent = vec[init_indices(n, k, seed)].copy()
    labels = None
    for _ in range(max_iter):
        new, best = _assign(vec, cent)
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        counts = np.bincount(labels, minlength=k)
        # member sums in increasing pixel order (bincount accumulates sequentially)
        sums = np.stack([np.bincount(labels, weights=vec[:, c], minlength=k) for c in range(3)], 1)
        empty = np.nonzero(counts == 0)[0]
        if empty.size:
            far = np.argsort(best, kind="stable")[:empty.size]
            sums[empty] = vec[far]
        norm = np.sqrt((sums[:, 0] * sums[:, 0] + sums[:, 1] * sums[:, 1]) + sums[:, 2] * sums[:, 2])
        norm[norm == 0] = 1.0
        cent = sums / norm[:, None]
    _, first = np.unique(labels, return_index=True)
    order = np.argsort(first, kind="stable")
    remap = np.empty(k, dtype=np.int64)
    used = np.unique(labels)[order]
    remap[used] = np.arange(used.size)
    return remap[labels].astype(np.int32)


def _disk_path(key: str, n: int, k: int):
    d = os.environ.get("CSX_KMEANS_CACHE")
    if not d or not key:
        return None
    return os.path.join(d, "km2_%s_%d_%d.npy" % (key, n, k))


def _from_disk(key, n, k):
    p = _disk_path(key, n, k)
    if p and os.path.exists(p):
        lab = np.load(p).astype(np.int32)
        if lab.shape == (n,):
            return lab
    return None


def _to_disk(key, n, k, lab):
    p = _disk_path(key, n, k)
    if p:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".%d.tmp.npy" % os.getpid()
        np.save(tmp, lab.astype(np.int16 if lab.max() < 32767 else np.int32))
        os.replace(tmp, p)


def patch_labels(vec: np.ndarray, k: int, key: str = "") -> np.ndarray:
    """Labels for K patches on the pixel set `vec`, seeded by K (seed 100 + K), memoised.

    Two parameters with the same K share one labeling, as a single K-means seed would give."""
    ck = (key, vec.shape[0], int(k))
    if ck not in _CACHE:
        _CACHE[ck] = spherical_kmeans(vec, int(k), seed=100 + int(k))
    return _CACHE[ck]


def _worker(args):
    vec, k = args
    return k, spherical_kmeans(vec, k, seed=100 + k)


def many_patch_labels(vec: np.ndarray, ks, key: str = "", processes: int | None = None):
    """Labelings for every distinct K in `ks` (dict K -> labels), computed in a spawn pool.

    With CSX_KMEANS_CACHE set to a directory, labelings are also read from / written to disk there
    (keyed by pixel-set name, pixel count and K; the algorithm is deterministic)."""
    n = vec.shape[0]
    for k in {int(k) for k in ks}:
        if (key, n, k) not in _CACHE:
            lab = _from_disk(key, n, k)
            if lab is not None:
                _CACHE[(key, n, k)] = lab
    todo = sorted({int(k) for k in ks if (key, vec.shape[0], int(k)) not in _CACHE}, reverse=True)
    if todo:
        nproc = processes or min(len(todo), len(os.sched_getaffinity(0)))
        work = vec.shape[0] * sum(todo)  # assignment cost ~ pixels x clusters per iteration
        if nproc > 1 and len(todo) > 4 and work > 5e7:
            import multiprocessing as mp
            # one BLAS thread per worker process (the workers read this when they import numpy)
            saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                    "MKL_NUM_THREADS")}
            for v in saved:
                os.environ[v] = "1"
            try:
                pool = mp.get_context("spawn").Pool(nproc)
            finally:
                for v, old in saved.items():
                    if old is None:
                        os.environ.pop(v, None)
                    else:
                        os.environ[v] = old
            with pool:
                for k, lab in pool.imap_unordered(_worker, [(vec, k) for k in todo]):
                    _CACHE[(key, vec.shape[0], k)] = lab
                    _to_disk(key, n, k, lab)
        else:
            for k in todo:
                _CACHE[(key, vec.shape[0], k)] = spherical_kmeans(vec, k, seed=100 + k)
                _to_disk(key, n, k, _CACHE[(key, n, k)])
    return {int(k): _CACHE[(key, vec.shape[0], int(k))] for k in ks}
