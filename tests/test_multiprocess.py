"""Host-side logic of the multi-process path, on CPU with the gloo backend (world size 2):
the contiguous chunking of problems (Sec. 3.1) and the one exchange of the path, the all-gather of
per-configuration V_tot for the global selection; checked against the oracle's selection over the
concatenated values. No GPU is used."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2604_08463_b300 import csx
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 11
        lo, hi = csx.chunk(n, world, rank)
        rng = np.random.default_rng(5)
        v = rng.random(n)
        v[7] = v[2] = v.min() - 0.5  # a tie: the lower index must win
        allv, best = csx.gather_select(torch.tensor(v[lo:hi]))
        q.put((rank, lo, hi, allv.numpy().tolist(), best))
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


def test_gather_select_gloo_two_ranks():
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
    rng = np.random.default_rng(5)
    v = rng.random(11)
    v[7] = v[2] = v.min() - 0.5
    # the oracle's selection on the same values: argmin, ties to the lowest index
    metrics = [[{"sys_sq": 2.0 * x, "stat": 0.0}] for x in v]
    vref, bref = rc.total_residual_variance(metrics, 1)
    assert bref == 2
    spans = sorted((lo, hi) for _, lo, hi, _, _ in out)
    assert spans == [(0, 5), (5, 11)]
    for _, _, _, allv, best in out:
        np.testing.assert_array_equal(np.array(allv), vref)
        assert best == bref
