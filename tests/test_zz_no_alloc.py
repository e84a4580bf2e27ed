"""csx_spectral_grad_noalloc, the entry point for callers that cannot let the library allocate
device memory (their device memory belongs to their own pool allocator, or they run a fixed memory
budget): it must give the results of csx_spectral_grad, call after call, from its static buffer.

Kept in a file of its own that pytest collects last; it passes alone and after the other tests.
Tolerances are those of the parity tests: L relative 1e-5, dL/dbeta max-norm relative 1e-4.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import workloads  # noqa: E402
from tests._inputs import small_case  # noqa: E402


@pytest.fixture(scope="module")
def csx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08463_b300 import csx as mod
    mod.lib()
    return mod


def _noalloc(csx, model, sky, labels, K, beta):
    """Call the C entry point directly through ctypes with caller-owned outputs."""
    nprob, P = beta.shape
    L = torch.full((nprob,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((nprob, P), float("nan"), dtype=torch.float32, device="cuda")
    Kh = np.ascontiguousarray(K, dtype=np.int32)
    rc = csx.lib().csx_spectral_grad_noalloc(
        ctypes.byref(model.c), ctypes.byref(sky.c), ctypes.c_void_p(labels.data_ptr()),
        Kh.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), nprob, ctypes.c_void_p(beta.data_ptr()),
        ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, csx.lib().csx_last_error()
    return L, g


def _close(L, g, Lr, gr):
    L, g, Lr, gr = (x.cpu().numpy().astype(np.float64) for x in (L, g, Lr, gr))
    assert np.all(np.abs(L - Lr) <= 1e-5 * np.abs(Lr))
    for q in range(g.shape[0]):
        assert np.abs(g[q] - gr[q]).max() <= 1e-4 * np.abs(gr[q]).max()


def test_noalloc_matches_spectral_grad_twice(csx):
    K = (9, 4, 5)
    case = small_case(nside=16, K=K, nreal=3, noise="separable")
    model, sky, labels = case.gpu()
    lab = labels[0].contiguous()
    for seed in (21, 22):  # two calls in a row, different parameters each time
        beta = torch.tensor(workloads.random_points(np.array(K), 3, seed=seed), dtype=torch.float32,
                            device="cuda")
        L, g = _noalloc(csx, model, sky, lab, K, beta)
        Lr, gr = csx.spectral_grad(model, sky, lab, K, beta)
        torch.cuda.synchronize()
        _close(L, g, Lr, gr)


def test_noalloc_second_configuration_and_size_limit(csx):
    # a different configuration after the first test's calls: the static buffer's leftovers
    # must not matter
    K = (30, 2, 7)
    case = small_case(nside=8, K=K, nreal=2, noise="perpixel")
    model, sky, labels = case.gpu()
    lab = labels[0].contiguous()
    beta = torch.tensor(workloads.random_points(np.array(K), 2, seed=5), dtype=torch.float32,
                        device="cuda")
    L, g = _noalloc(csx, model, sky, lab, K, beta)
    Lr, gr = csx.spectral_grad(model, sky, lab, K, beta)
    torch.cuda.synchronize()
    _close(L, g, Lr, gr)
    # a request larger than the static buffer is refused on the host, before any launch
    Kbig = np.array([40000, 20000, 5000], dtype=np.int32)  # 85000 rows x 16 > 2^20 floats
    Lb = torch.zeros(1, dtype=torch.float64, device="cuda")
    gb = torch.zeros(1, dtype=torch.float32, device="cuda")
    rc = csx.lib().csx_spectral_grad_noalloc(
        ctypes.byref(model.c), ctypes.byref(sky.c), ctypes.c_void_p(lab.data_ptr()),
        Kbig.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1, ctypes.c_void_p(beta.data_ptr()),
        ctypes.c_void_p(Lb.data_ptr()), ctypes.c_void_p(gb.data_ptr()), None)
    assert rc == -1
    assert b"static buffer" in csx.lib().csx_last_error()


def test_noalloc_python_wrapper_and_host_refusals(csx):
    # the Python wrapper passes caller-owned outputs straight through: same results as the
    # allocating call
    K = (7, 3, 5)
    case = small_case(nside=8, K=K, nreal=2, noise="separable")
    model, sky, labels = case.gpu()
    lab = labels[0].contiguous()
    beta = torch.tensor(workloads.random_points(np.array(K), 2, seed=11), dtype=torch.float32,
                        device="cuda")
    L = torch.empty(2, dtype=torch.float64, device="cuda")
    g = torch.empty((2, sum(K)), dtype=torch.float32, device="cuda")
    out = csx.spectral_grad_noalloc(model, sky, lab, K, beta, L, g)
    assert out[0] is L and out[1] is g
    Lr, gr = csx.spectral_grad(model, sky, lab, K, beta)
    torch.cuda.synchronize()
    _close(L, g, Lr, gr)
    # outputs of the wrong type or shape, or an input that would need converting, are refused
    # before anything reaches the device
    with pytest.raises(ValueError, match="L must be"):
        csx.spectral_grad_noalloc(model, sky, lab, K, beta, L.to(torch.float32), g)
    with pytest.raises(ValueError, match="grad must be"):
        csx.spectral_grad_noalloc(model, sky, lab, K, beta, L, g[:, :-1].contiguous())
    with pytest.raises(ValueError, match="beta must be"):
        csx.spectral_grad_noalloc(model, sky, lab, K, beta.double(), L, g)
    # a patch count above CSX_MAX_K is refused by the C entry point
    Kbad = np.array([1 << 25, 2, 2], dtype=np.int32)
    rc = csx.lib().csx_spectral_grad_noalloc(
        ctypes.byref(model.c), ctypes.byref(sky.c), ctypes.c_void_p(lab.data_ptr()),
        Kbad.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1, ctypes.c_void_p(beta.data_ptr()),
        ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(g.data_ptr()), None)
    assert rc == -1 and b"K_j" in csx.lib().csx_last_error()
