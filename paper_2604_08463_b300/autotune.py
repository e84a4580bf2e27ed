"""Launch-configuration autotuner of the batched fit: for a batch's shape it times the candidate
(likelihood path, CTA size) pairs of csx_fit_batch on the batch with an iteration cap, with CUDA
events, and keeps the fastest, cached per shape bucket in a JSON file.

Candidates: the residual-moment path (per cell; homogeneous or separable noise, adjoint gradient)
with 64, 128 or 256 threads per CTA (64 only for L-BFGS), and the streaming path (per pixel, any
noise) with 256 threads. Per-pixel noise or finite-difference gradients leave the streaming path
as the only candidate: nothing is timed.

Shape bucket: noise model, solver, gradient mode, realizations, and the powers of two nearest to the
pixel count and to the mean and largest parameter counts P of the batch.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

CANDIDATES = (("moment", 128), ("moment", 64), ("moment", 256), ("stream", 256))


def _p2(x: float) -> int:
    return 0 if x <= 0 else int(round(math.log2(x)))


def shape_key(noise: str, npix: int, nreal: int, K, solver: str = "lbfgs",
              grad_mode: str = "adjoint") -> str:
    """Cache key of a batch: K is [nconf][3] (clusters per parameter of every configuration)."""
    P = np.asarray(K).reshape(-1, 3).sum(axis=1)
    return "%s|%s|%s|r%d|n2^%d|Pmean2^%d|Pmax2^%d" % (
        noise, solver, grad_mode, int(nreal), _p2(npix), _p2(float(P.mean())), _p2(float(P.max())))


def candidates(noise: str, solver: str = "lbfgs", grad_mode: str = "adjoint"):
    """Valid (path, threads) pairs for the batch's noise model, solver and gradient mode."""
    out = []
    for path, nt in CANDIDATES:
        if path == "moment" and (noise == "perpixel" or grad_mode != "adjoint"):
            continue
        if path == "moment" and nt == 64 and solver != "lbfgs":
            continue
        out.append((path, nt))
    return out


def sample_configurations(nconf: int, sample: int):
    """Evenly spaced configuration indices (all of them when nconf <= sample)."""
    if nconf <= sample:
        return list(range(nconf))
    return sorted({int(round(x)) for x in np.linspace(0, nconf - 1, sample)})


def _load(cache):
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store(cache, table):
    if not cache:
        return
    d = os.path.dirname(os.path.abspath(cache))
    os.makedirs(d, exist_ok=True)
    tmp = cache + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, cache)


MARGIN = 0.03  # another candidate replaces the first (the library's own rule) only when faster by this


def choose(key: str, cands, timer, cache=None, margin: float = MARGIN):
    """The fastest candidate for `key`: from the cache, else by calling timer(path, threads) -> ms for
    every candidate (a single candidate is returned untimed). The first candidate is the library's
    automatic choice and is kept unless another is faster by more than `margin` (timing noise).
    Returns (dict(path, threads), table entry)."""
    table = _load(cache)
    if key in table:
        e = table[key]
        return {"path": e["path"], "threads": e["threads"]}, e
    if len(cands) == 1:
        path, nt = cands[0]
        e = {"path": path, "threads": nt, "ms": {}}
    else:
        ms = {"%s/%d" % c: float(timer(*c)) for c in cands}
        best = min(cands, key=lambda c: ms["%s/%d" % c])
        first = cands[0]
        if ms["%s/%d" % best] > (1.0 - margin) * ms["%s/%d" % first]:
            best = first
        e = {"path": best[0], "threads": best[1], "ms": ms}
    table[key] = e
    _store(cache, table)
    return {"path": e["path"], "threads": e["threads"]}, e


def tune_fit(csx, model, sky, labels, K, beta0, solver: str = "lbfgs", grad_mode: str = "adjoint",
             sample=None, max_iter: int = 10, cache=None, **opts):
    """Options {path, threads} for csx.fit_batch on this batch (sky: csx.Sky, labels: device
    [nconf][3][npix], K: [nconf][3], beta0: packed device parameters). Times each candidate once,
    after one untimed warm-up, on the whole batch (or `sample` evenly spaced configurations) with
    every problem capped at `max_iter` iterations. The cap keeps tuning short; the whole batch keeps
    the timing a throughput: the persistent fit holds hundreds of problems at once, and a batch of
    only a few problems per resident slot is timed by its slowest problem (a latency), which
    favours larger CTAs than the full batch does."""
    import torch
    K = np.asarray(K, dtype=np.int32).reshape(-1, 3)
    key = shape_key(sky.noise, sky.npix, sky.nreal, K, solver, grad_mode)
    cands = candidates(sky.noise, solver, grad_mode)
    pick = sample_configurations(K.shape[0], sample if sample else K.shape[0])
    offs, P = csx.param_offsets(K, sky.nreal)
    idx = np.concatenate([np.arange(offs[c * sky.nreal], offs[c * sky.nreal] + P[c] * sky.nreal)
                          for c in pick])
    sub_b = beta0[torch.as_tensor(idx, device=beta0.device)].contiguous()
    sub_l = labels[torch.as_tensor(pick, device=labels.device)].contiguous()
    sub_k = K[pick]

    def timer(path, nt):
        kw = dict(opts, path=path, threads=nt, solver=solver, grad_mode=grad_mode,
                  max_iter=max_iter)
        csx.fit_batch(model, sky, sub_l, sub_k, sub_b, **kw)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        csx.fit_batch(model, sky, sub_l, sub_k, sub_b, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    return choose(key, cands, timer, cache)


# ------------------------------------------------------------------ streaming kernel schedule ----
def stream_key(noise: str, npix: int, nprob: int, P: int, grad: bool, plan: bool = False) -> str:
    """Cache key of a streaming call: noise model, gradient or not, cell plan or not, and the
    powers of two nearest to the pixel count, the number of problems and the parameter count."""
    return "stream|%s|%s%s|n2^%d|q2^%d|P2^%d" % (noise, "grad" if grad else "like",
                                                "|plan" if plan else "", _p2(npix), _p2(nprob),
                                                _p2(P))


def choose_schedule(key: str, cands, timer, cache=None, margin: float = MARGIN):
    """The fastest (tile, stages) schedule for `key`: from the cache, else by timer(tile, stages) ->
    ms for every candidate; the first candidate (the library default) is kept unless another is
    faster by more than `margin`. Returns ((tile, stages), table entry)."""
    table = _load(cache)
    if key in table:
        e = table[key]
        return (e["tile"], e["stages"]), e
    ms = {"%d/%d" % c: float(timer(*c)) for c in cands}
    best = min(cands, key=lambda c: ms["%d/%d" % c])
    if ms["%d/%d" % best] > (1.0 - margin) * ms["%d/%d" % cands[0]]:
        best = cands[0]
    e = {"tile": best[0], "stages": best[1], "ms": ms}
    table[key] = e
    _store(cache, table)
    return (e["tile"], e["stages"]), e


def tune_stream(csx, model, sky, labels, K, beta, grad: bool = True, ncall: int = 5, cache=None,
                plan=None):
    """Select the streaming kernel's tile schedule for calls shaped like this one (csx.spectral_grad
    or csx.spectral_like of beta [nprob, P] on sky, or plan.grad of a csx.SpectralPlan): each built
    schedule is timed with CUDA events over `ncall` calls after one untimed call; the chosen
    schedule is left in force (csx.stream_schedule). Returns ((tile, stages), table entry)."""
    import torch
    if plan is not None:
        def fn(model, sky, labels, K, beta):
            plan.grad(model, sky, beta, want_grad=grad)
    else:
        fn = csx.spectral_grad if grad else csx.spectral_like
    key = stream_key(sky.noise, sky.npix, beta.shape[0], beta.shape[1], grad, plan is not None)

    def timer(tile, stages):
        csx.stream_schedule(tile, stages)
        fn(model, sky, labels, K, beta)
        stream = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ncall):
            fn(model, sky, labels, K, beta)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / ncall

    sched, e = choose_schedule(key, list(csx.STREAM_SCHEDULES), timer, cache)
    csx.stream_schedule(*sched)
    return sched, e
