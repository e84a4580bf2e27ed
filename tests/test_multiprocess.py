"""Host-side logic of the multi-process path, on CPU with the gloo backend (world size 2):
the contiguous chunking of problems (Sec. 3.1) and the one exchange of the path, the all-gather of
every rank's per-problem metric rows for the global selection (which csx_select then makes on the
device); the gathered rows are checked against the full list and the oracle's selection over them.
No GPU is used."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rows(nconf, nreal):
    """Metric rows of nconf configurations x nreal problems: SYS_SQ and STAT slots set, a tie
    between configurations 2 and 7 at the smallest total."""
    rng = np.random.default_rng(5)
    m = np.zeros((nconf * nreal, 8))
    m[:, 0] = rng.random(nconf * nreal)
    m[:, 1] = rng.random(nconf * nreal)
    m[7 * nreal:8 * nreal] = m[2 * nreal:3 * nreal] = 0.0
    return m


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2604_08463_b300 import csx
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nconf, nreal = 11, 3
        lo, hi = csx.chunk(nconf, world, rank)  # whole configurations per rank
        m = _rows(nconf, nreal)
        allm = csx.gather_metrics(torch.tensor(m[lo * nreal:hi * nreal]))
        q.put((rank, lo, hi, allm.numpy().tolist()))
    finally:
        dist.destroy_process_group()


def test_chunk_covers_every_problem_once():
    from paper_2604_08463_b300 import csx
    for n in (0, 1, 7, 10000):
        for world in (1, 2, 3, 8):
            spans = [csx.chunk(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
    with pytest.raises(ValueError):
        csx.chunk(5, 2, 2)


def test_gather_metrics_gloo_two_ranks():
    import multiprocessing as mp
    from oracle import reconstruct as rc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nconf, nreal, npix = 11, 3, 1
    full = _rows(nconf, nreal)
    spans = sorted((lo, hi) for _, lo, hi, _ in out)
    assert spans == [(0, 5), (5, 11)]
    for _, _, _, allm in out:
        np.testing.assert_array_equal(np.array(allm), full)  # every row, in rank order
    # the oracle's selection over the gathered rows: argmin, ties to the lowest index
    metrics = [[{"sys_sq": full[c * nreal + n, 0], "stat": full[c * nreal + n, 1]}
                for n in range(nreal)] for c in range(nconf)]
    vref, bref = rc.total_residual_variance(metrics, npix)
    assert bref == 2 and vref[7] == vref[2]
