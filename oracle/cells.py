"""Oracle: intersection cells of the three patch labelings (Sec. 2.2-2.3).

The three labelings (beta_d, T_d, beta_s) are independent and need not align (Sec. 2.3), so the
pixels that share all three parameters form "cells": the distinct (l_d, l_T, l_s) triples. The
cell structure is the stable ordering of pixels by (l_d, l_T, l_s) (lexicographic, ties kept in pixel
order), the start offset of every run of equal triples, and the triple of every run.

Also the per-cell weighted second moment used by the moment form of the likelihood: for separable
noise N_p^-1 = w_p diag(n), every pixel of a cell has the same A, so
  L = - sum_p sum_s w_p (A^T n d)^T (A^T n A)^-1 (A^T n d) = - sum_c tr[(A_c^T n A_c)^-1 A_c^T n S_c n A_c],
  S_c = sum_{p in c} w_p sum_s d_{p,s} d_{p,s}^T.

Parity pins: a pure-Python grouping of the triples (brute force), and the moment-form likelihood
against the per-pixel definition.
"""
from __future__ import annotations

import numpy as np


def cells(labels):
    """(perm int64 [npix], offsets int64 [ncell + 1], triples int64 [3, ncell])."""
    labels = np.asarray(labels)
    npix = labels.shape[1]
    perm = np.lexsort((labels[2], labels[1], labels[0]))
    keys = labels[:, perm]
    if npix == 0:
        return perm, np.zeros(1, np.int64), np.zeros((3, 0), np.int64)
    change = np.any(keys[:, 1:] != keys[:, :-1], axis=0)
    starts = np.concatenate([[0], np.nonzero(change)[0] + 1])
    return perm, np.append(starts, npix).astype(np.int64), keys[:, starts].astype(np.int64)


def cells_bruteforce(labels):
    """Same result built with a dictionary of Python lists (small inputs only)."""
    groups = {}
    for p in range(labels.shape[1]):
        groups.setdefault(tuple(int(v) for v in labels[:, p]), []).append(p)
    triples = sorted(groups)
    perm, offs = [], [0]
    for t in triples:
        perm.extend(groups[t])
        offs.append(len(perm))
    return (np.array(perm, np.int64), np.array(offs, np.int64),
            np.array(triples, np.int64).T.reshape(3, -1))


def cell_moments(d, w, labels):
    """S_c [ncell, F, F] = sum_{p in c} w_p sum_s d_{p,s} d_{p,s}^T, with the cell structure."""
    perm, offs, trip = cells(labels)
    F = d.shape[-1]
    S = np.zeros((offs.size - 1, F, F))
    for c in range(offs.size - 1):
        idx = perm[offs[c]:offs[c + 1]]
        x = d[idx] * np.sqrt(w[idx])[:, None, None]
        S[c] = np.einsum("psf,psg->fg", x, x)
    return S, trip


def moment_likelihood(nu, S, trip, ninv_band, K, beta):
    """L = - sum_c tr[(A_c^T n A_c)^-1 A_c^T n S_c n A_c] for separable noise."""
    from .likelihood import split_params
    from .mixing import mixing_matrix
    bd, td, bs = split_params(beta, K)
    A = mixing_matrix(nu, bd[trip[0]], td[trip[1]], bs[trip[2]])  # [ncell, F, 3]
    na = ninv_band[None, :, None] * A
    M = np.einsum("cfi,cfj->cij", A, na)
    G = np.einsum("cfi,cfg,cgj->cij", na, S, na)
    return -float(np.sum(np.linalg.inv(M) * G))
