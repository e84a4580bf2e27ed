"""Oracle fits run in worker processes (spawned, one BLAS thread each) for the full-size tests."""
from __future__ import annotations

import os


def fit_job(args):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    from oracle import fit as ofit
    nu, d64, ninv64, labels, K, beta0, lower, upper = args
    x, L, info = ofit.fit(nu, d64, ninv64, labels, K, beta0, lower, upper)
    return x, L, info["interior"]


def grad_job(args):
    """(L, dL/dbeta, term scale S, data-scale term scale Sd) of the oracle at one point."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    from oracle import likelihood as lk
    nu, d64, ninv64, labels, K, beta = args
    L, g = lk.spectral_gradient(nu, d64, ninv64, labels, K, beta)
    return (L, g, lk.gradient_term_scale(nu, d64, ninv64, labels, K, beta),
            lk.gradient_term_scale(nu, d64, ninv64, labels, K, beta, data_scale=True))


def oracle_pool(n):
    import multiprocessing as mp
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                            "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(n)
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
