"""Writes the stored oracle fits that the full-size GPU fit tests compare against.

    python tests/golden/make_fit_refs.py [name ...]      (all cases when no name is given)

Each case fits sampled (configuration, realization) problems of a seeded synthetic workload with the
FP64 oracle (oracle.fit.fit: L-BFGS-B, then Gauss-Newton and exact-Hessian Newton steps to the
minimiser) and saves, per problem, the fitted parameters, L at them, the interior mask, and a
fingerprint of the inputs (sum of the float64 data and of the labels) that the tests check before
comparing. Only synth/ (input generation) and oracle/ are called. The large problems (P up to
~1300 at nside 64) take minutes each, which is why they are computed once here rather than during
the GPU tests. Problems run in a pool of processes, one BLAS thread each.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
os.environ.setdefault("CSX_KMEANS_CACHE", os.path.join(ROOT, ".cache", "kmeans"))


def _scan64():
    from synth import workloads
    return workloads.scan(nside=64, nconf=1000, kmax=500, nreal=10, b_cut_deg=20.0, seed=4)


def _scan64_picks(wl):
    """Nine problems spread over the scan's P range, six below 200 and three from 600 up."""
    P = np.repeat(wl.P, wl.nreal)
    rng = np.random.default_rng(17)
    picks = []
    for lo, hi in ((3, 20), (20, 50), (50, 80), (80, 120), (120, 160), (160, 200), (600, 800),
                   (800, 1100), (1100, 1400)):
        picks.append(int(rng.choice(np.nonzero((P >= lo) & (P < hi))[0])))
    return picks


def _scan16():
    from synth import workloads
    return workloads.scan(nside=16, nconf=6, kmax=1000, nreal=2, b_cut_deg=20.0, seed=8)


def _scan16_picks(wl):
    """Smallest, median and largest P of the large-K shape."""
    o = np.argsort(np.repeat(wl.P, wl.nreal), kind="stable")
    return [int(o[0]), int(o[len(o) // 2]), int(o[-1])]


def _multires16():
    from synth import healpix, partitions as pt, sky as S, workloads
    nside = 16
    reg = pt.latitude_regions(nside, np.arange(healpix.npix(nside)))
    pix = np.nonzero(reg >= 0)[0]
    sk = S.make_sky(nside, pix=pix, truth="smooth", hitcount=True)
    lab, K = pt.multires_labels(nside, pix, levels=((4, 4, 8), (0, 2, 4), (1, 1, 2)))
    return workloads.Workload("multires16", sk, K[None], lab[None], 2, "separable")


def _pipeline64():
    """The two largest-P configurations of the full-pipeline scan (nside 64, |b| > 20 deg, 4000
    configurations, K log-uniform up to 1000): requested K (872, 874, 843) and (963, 899, 139)."""
    from synth import workloads
    return workloads.scan_subset([937, 1739], nside=64, nconf=4000, kmax=1000, nreal=1)


def _fullsky64():
    """Full sky at nside 64, K = (100, 20, 30), 100 realizations (the fit and W d workload)."""
    from synth import workloads
    return workloads.fullsky(64, (100, 20, 30), nreal=100)


CASES = {
    "scan64": (_scan64, _scan64_picks),
    "scan16_k1000": (_scan16, _scan16_picks),
    "multires16": (_multires16, lambda wl: [0, 1]),
    "pipeline64": (_pipeline64, lambda wl: [0, 1]),
    "fullsky64": (_fullsky64, lambda wl: [0, 57]),
}


def inputs(wl, q):
    """The oracle's float64 inputs of problem q (the float32 values the GPU reads, widened)."""
    c, r = divmod(q, wl.nreal)
    F = wl.sky.nfreq
    nb32 = wl.sky.ninv_band.astype(np.float32).astype(np.float64)
    ninv = wl.sky.w.astype(np.float32).astype(np.float64)[:, None] * nb32[None, :F]
    d64 = wl.data()[r, :, :, :F].astype(np.float64)
    return c, d64, ninv


def fingerprint(wl, q):
    c, d64, _ = inputs(wl, q)
    return np.array([d64.sum(), float(wl.labels[c].astype(np.int64).sum())])


def _job(args):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    name, q = args
    from oracle import fit as ofit
    from synth import workloads
    wl = CASES[name][0]()
    c, d64, ninv = inputs(wl, q)
    t = time.time()
    x, L, info = ofit.fit(wl.sky.nu, d64, ninv, wl.labels[c], wl.K[c], wl.beta0(c), workloads.LOWER,
                          workloads.UPPER)
    print("%s problem %d (P %d): %.0f s, polish %d + %d, max |g_free| %.2e"
          % (name, q, wl.P[c], time.time() - t, info["polished"], info["newton"],
             np.abs(info["grad"][info["interior"]]).max(initial=0.0)), flush=True)
    return q, x, L, info["interior"], fingerprint(wl, q)


def main(names):
    jobs, size = [], {}
    for name in names:
        wl = CASES[name][0]()
        for q in CASES[name][1](wl):
            jobs.append((name, q))
            size[(name, q)] = int(wl.P[q // wl.nreal])
    jobs.sort(key=lambda j: -size[j])  # largest problems first
    with mp.get_context("spawn").Pool(min(len(jobs), len(os.sched_getaffinity(0)))) as pool:
        out = pool.map(_job, jobs, chunksize=1)
    for name in names:
        rows = [o for (n, _), o in zip(jobs, out) if n == name]
        rows.sort(key=lambda o: o[0])
        np.savez(os.path.join(HERE, "fit_refs_%s.npz" % name),
                 picks=np.array([o[0] for o in rows]),
                 **{"x_%d" % o[0]: o[1] for o in rows}, **{"L_%d" % o[0]: o[2] for o in rows},
                 **{"interior_%d" % o[0]: o[3] for o in rows},
                 **{"fingerprint_%d" % o[0]: o[4] for o in rows})
        print("wrote", name, [o[0] for o in rows])


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
