"""Shared test inputs: one synthetic workload, handed to the CUDA path as device tensors and to the
oracle as float64 copies of the very same float32 values."""
from __future__ import annotations

import numpy as np

from synth import sky as S, workloads


class Case:
    def __init__(self, wl: workloads.Workload, noise: str):
        self.wl = wl
        self.noise = noise
        self.nu = wl.sky.nu
        self.npix = wl.npix
        self.d32 = wl.data()                                   # [R, npix, 2, 16] float32
        self.nb32 = np.zeros(16, np.float32)
        self.nb32[:wl.sky.nfreq] = wl.sky.ninv_band.astype(np.float32)
        self.w32 = wl.sky.w.astype(np.float32)
        self.fg32 = wl.foreground_padded()                     # [npix, 2, 16] float32
        F = wl.sky.nfreq
        if noise == "homogeneous":
            self.ninv64 = np.broadcast_to(self.nb32[:F].astype(np.float64), (self.npix, F)).copy()
        elif noise == "separable":
            self.ninv64 = self.w32.astype(np.float64)[:, None] * self.nb32[:F].astype(np.float64)
        else:
            # per-pixel, not separable: band-dependent modulation
            rng = np.random.default_rng(77)
            mod = 1.0 + 0.3 * rng.random((self.npix, F))
            self.np32 = np.zeros((self.npix, 16), np.float32)
            self.np32[:, :F] = (self.w32[:, None] * self.nb32[:F] * mod).astype(np.float32)
            self.ninv64 = self.np32[:, :F].astype(np.float64)

    def d64(self, r):
        return self.d32[r, :, :, :self.wl.sky.nfreq].astype(np.float64)

    def fg64(self):
        return self.fg32[:, :, :self.wl.sky.nfreq].astype(np.float64)

    def gpu(self, dev="cuda"):
        import torch
        from paper_2604_08463_b300 import csx
        d = torch.from_numpy(self.d32).to(dev)
        kw = {}
        if self.noise == "separable":
            kw["w"] = torch.from_numpy(self.w32).to(dev)
        if self.noise == "perpixel":
            kw["ninv_pix"] = torch.from_numpy(self.np32).to(dev)
        sky = csx.Sky(d, noise=self.noise, ninv_band=self.nb32, **kw)
        model = csx.Model(self.nu)
        labels = torch.from_numpy(np.ascontiguousarray(self.wl.labels)).to(dev)
        return model, sky, labels


def small_case(nside=8, K=(5, 3, 4), nreal=3, noise="separable", truth="smooth", seed=9):
    """Random (not K-means) labels on a small sky, every patch non-empty."""
    sk = S.make_sky(nside, truth=truth, hitcount=noise != "homogeneous")
    rng = np.random.default_rng(seed)
    lab = np.stack([rng.integers(0, K[j], sk.npix) for j in range(3)]).astype(np.int32)
    for j in range(3):
        lab[j, :K[j]] = np.arange(K[j])
    wl = workloads.Workload("small", sk, np.array([K], np.int32), lab[None], nreal, noise)
    return Case(wl, noise)


def scan_case(nside=16, nconf=6, kmax=40, nreal=2, b_cut=20.0, seed=4):
    wl = workloads.scan(nside=nside, nconf=nconf, kmax=kmax, nreal=nreal, b_cut_deg=b_cut, seed=seed)
    return Case(wl, "separable")


def pack(wl, per_problem):
    """Packed parameter vector (problem q = c * nreal + n) from a list of per-problem arrays."""
    return np.concatenate([np.asarray(x, np.float32) for x in per_problem])
