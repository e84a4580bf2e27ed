"""Fixed, seeded cases of the hot kernels, sized for one profiler capture each (a few GB on the
device at most, inputs larger than L2), printed with the unit counts a roofline needs.

    python -m paper_2604_08463_b300.profile_cases fit NCONF KMAX
        the persistent fit (k_fit, moment path, 128 threads) on the first NCONF configurations of
        the nside-64 scan (|b| > 20 deg, K per parameter log-uniform up to KMAX, 10 realizations,
        seed 4), fitted twice from the start point; prints the cell evaluations of one fit
    python -m paper_2604_08463_b300.profile_cases kmeans NCONF KMAX
        the GPU spherical K-means of every distinct K of that scan's first NCONF configurations
        (one launch, twice)
    python -m paper_2604_08463_b300.profile_cases stream NREAL
        the streaming kernel (k_spectral_tma) on the full-sky nside-64 configuration with
        K = (100, 20, 30) and separable noise, NREAL realizations: plan L + grad, plan L,
        L + grad, L (one call each), twice; prints the pixel evaluations of one call

Inputs come from synth/ (seeded generators); every step runs in the library's kernels.
"""
from __future__ import annotations

import sys

import numpy as np


def _device_inputs(wl):
    import torch
    from . import csx
    dev = torch.device("cuda", torch.cuda.current_device())
    nb = np.zeros(16, np.float32)
    nb[:wl.sky.nfreq] = wl.sky.ninv_band.astype(np.float32)
    d = torch.from_numpy(wl.data()).to(dev)
    w = torch.from_numpy(wl.sky.w.astype(np.float32)).to(dev)
    model = csx.Model(wl.sky.nu)
    sky = csx.Sky(d, noise="separable", ninv_band=nb, w=w)
    labels = torch.from_numpy(np.ascontiguousarray(wl.labels, dtype=np.int32)).to(dev)
    return model, sky, labels


def fit_case(nconf: int, kmax: int):
    import torch
    from synth import workloads
    from . import csx
    wl = workloads.scan(nside=64, nconf=nconf, kmax=kmax, nreal=10, b_cut_deg=20.0, seed=4)
    model, sky, labels = _device_inputs(wl)
    beta0 = torch.tensor(np.concatenate([np.tile(wl.beta0(c), wl.nreal) for c in range(wl.nconf)]),
                         dtype=torch.float32, device=labels.device)
    for _ in range(2):
        res = csx.fit_batch(model, sky, labels, wl.K, beta0, path="moment", threads=128)
        torch.cuda.synchronize()
    _, _, nc = csx.build_cells(labels, wl.K)
    nc = nc.cpu().numpy().astype(np.float64)
    nev = res["nevals"].cpu().numpy().astype(np.float64)
    conf = np.repeat(np.arange(wl.nconf), wl.nreal)
    st = res["status"].cpu().numpy()
    print("problems %d converged %d mean P %.1f cell evaluations per fit %.0f"
          % (st.size, int((st == 0).sum()), float(wl.P.mean()), float((nev * nc[conf]).sum())))


def stream_case(nreal: int):
    import torch
    from synth import workloads
    from . import csx
    wl = workloads.fullsky(64, (100, 20, 30), nreal=nreal)
    model, sky, labels = _device_inputs(wl)
    lab, K = labels[0], wl.K[0]
    beta = torch.tensor(np.tile(wl.beta0(0), (wl.nreal, 1)), dtype=torch.float32, device=lab.device)
    plan = csx.SpectralPlan(lab, K)
    for _ in range(2):
        La, ga = plan.grad(model, sky, beta)
        plan.grad(model, sky, beta, want_grad=False)
        Lc, gc = csx.spectral_grad(model, sky, lab, K, beta)
        csx.spectral_like(model, sky, lab, K, beta)
    torch.cuda.synchronize()
    print("cells %d pixel evaluations per call %d; plan vs per-run L max rel %.2e, grad max rel %.2e"
          % (plan.ncell, wl.nreal * wl.npix, float(((La - Lc).abs() / Lc.abs()).max()),
             float((ga - gc).abs().max() / gc.abs().max())))
    plan.close()


def kmeans_case(nconf: int, kmax: int):
    import torch
    from synth import healpix, kmeans as km, workloads
    from . import csx
    pix = healpix.galactic_cut(64, 20.0)
    vec = healpix.unit_vectors(64)[pix]
    n = vec.shape[0]
    ks = sorted({int(k) for k in workloads.sample_patch_counts(nconf, kmax, seed=4).reshape(-1)})
    init = [km.init_indices(n, k, 100 + k) for k in ks if 1 < k < n]
    vd = torch.from_numpy(vec).to(torch.device("cuda", torch.cuda.current_device()))
    for _ in range(2):
        lab, iters = csx.kmeans(vd, ks, init)
        torch.cuda.synchronize()
    print("labelings %d (K %d..%d) pixels %d mean iterations %.1f"
          % (len(ks), ks[0], ks[-1], n, float(iters.float().mean())))


def main(argv):
    if len(argv) >= 1 and argv[0] == "fit":
        fit_case(int(argv[1]) if len(argv) > 1 else 60, int(argv[2]) if len(argv) > 2 else 500)
    elif len(argv) >= 1 and argv[0] == "stream":
        stream_case(int(argv[1]) if len(argv) > 1 else 40)
    elif len(argv) >= 1 and argv[0] == "kmeans":
        kmeans_case(int(argv[1]) if len(argv) > 1 else 1000, int(argv[2]) if len(argv) > 2 else 500)
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
