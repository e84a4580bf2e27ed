"""The C ABI library (no GPU needed): it loads, exports every symbol include/csx.h declares, and
the binding's ctypes structures have the C layout."""
import ctypes
import numpy as np
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "csx.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csx_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_08463_b300 import build, csx
    build.build()
    return csx.lib()


def test_exports_every_declared_symbol(lib):
    from paper_2604_08463_b300 import csx
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(csx.EXPORTS) == names
    so = os.path.join(ROOT, "paper_2604_08463_b300", "libcsx.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True,
                         check=True).stdout
    for n in names:
        assert re.search(r"\bT %s$" % n, out, re.M), n


def test_struct_layouts_match_c(lib):
    from paper_2604_08463_b300 import csx
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "csx.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(csx_model), sizeof(csx_sky), sizeof(csx_fit_opts),
         offsetof(csx_sky, ninv_band), offsetof(csx_sky, w), offsetof(csx_fit_opts, fd_step));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as t:
        c = os.path.join(t, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(t, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(csx.CModel), ctypes.sizeof(csx.CSky), ctypes.sizeof(csx.CFitOpts),
                    csx.CSky.ninv_band.offset, csx.CSky.w.offset, csx.CFitOpts.fd_step.offset]


def test_host_only_calls(lib):
    from paper_2604_08463_b300 import csx
    assert csx.version().startswith("csx")
    o = csx.fit_options(max_iter=7, path="moment")
    assert o.max_iter == 7 and o.path == 2 and o.history == 8
    # argument errors are reported before touching a device
    rc = lib.csx_mixing(None, 1, None, None, None, None)
    assert rc == -1 and b"model" in lib.csx_last_error()


def test_misaligned_pointers_are_rejected_on_the_host(lib):
    """Pixel rows are read as 16-byte vectors and staged by tensor copies: a data pointer that is
    not 16-byte aligned (or an int / float / double array off its natural alignment) is refused with
    CSX_EINVAL before anything touches a device. The pointers below are never dereferenced."""
    import ctypes
    from paper_2604_08463_b300 import csx
    model = csx.Model(np.array([40.0, 100.0, 402.0]))
    sky = csx.CSky()
    sky.npix, sky.nreal, sky.noise_kind = 10, 1, 0
    for f in range(3):
        sky.ninv_band[f] = 1.0
    K = (ctypes.c_int32 * 3)(1, 1, 1)
    ok16, off4 = 0x10000, 0x10004
    sky.d = off4
    rc = lib.csx_spectral_like(ctypes.byref(model.c), ctypes.byref(sky), ctypes.c_void_p(ok16), K, 1,
                               ctypes.c_void_p(ok16), ctypes.c_void_p(ok16), None)
    assert rc == -1 and b"sky->d must be 16-byte aligned" in lib.csx_last_error()
    sky.d = ok16
    rc = lib.csx_spectral_grad(ctypes.byref(model.c), ctypes.byref(sky), ctypes.c_void_p(ok16 + 2),
                               K, 1, ctypes.c_void_p(ok16), ctypes.c_void_p(ok16),
                               ctypes.c_void_p(ok16), None)
    assert rc == -1 and b"labels must be 4-byte aligned" in lib.csx_last_error()
    rc = lib.csx_spectral_grad(ctypes.byref(model.c), ctypes.byref(sky), ctypes.c_void_p(ok16), K,
                               1, ctypes.c_void_p(ok16), ctypes.c_void_p(off4), ctypes.c_void_p(ok16),
                               None)
    assert rc == -1 and b"L must be 8-byte aligned" in lib.csx_last_error()
    rc = lib.csx_spectral_grad_noalloc(ctypes.byref(model.c), ctypes.byref(sky), ctypes.c_void_p(ok16),
                                       K, 1, ctypes.c_void_p(ok16 + 1), ctypes.c_void_p(ok16),
                                       ctypes.c_void_p(ok16), None)
    assert rc == -1 and b"beta must be 4-byte aligned" in lib.csx_last_error()


def test_spectra_arguments_are_refused_on_the_host(lib):
    """The pseudo-C_ell entry points check sizes and the pixel list before touching a device."""
    import ctypes
    plan = ctypes.c_void_p()
    pix = (ctypes.c_int32 * 4)(0, 5, 5, 9)
    rc = lib.csx_sht_plan_create(4, 11, pix, 4, ctypes.byref(plan), None)
    assert rc == -1 and b"strictly increasing" in lib.csx_last_error() and not plan.value
    pix = (ctypes.c_int32 * 2)(0, 192)
    rc = lib.csx_sht_plan_create(4, 11, pix, 2, ctypes.byref(plan), None)
    assert rc == -1 and b"pix out of range" in lib.csx_last_error()
    rc = lib.csx_sht_plan_create(4, 16, pix, 1, ctypes.byref(plan), None)
    assert rc == -1 and b"lmax" in lib.csx_last_error()
    rc = lib.csx_sht_plan_create(0, 0, pix, 1, ctypes.byref(plan), None)
    assert rc == -1 and b"nside" in lib.csx_last_error()
    rc = lib.csx_sht_plan_create(4, 11, pix, 1, None, None)
    assert rc == -1 and b"plan is NULL" in lib.csx_last_error()
    rc = lib.csx_pseudo_cl(None, 1, ctypes.c_void_p(0x10000), 2, 2, 1, None, None, 1,
                           ctypes.c_void_p(0x10000), None)
    assert rc == -1 and b"plan is NULL" in lib.csx_last_error()
    assert lib.csx_sht_plan_destroy(None) == 0


def test_residual_spectra_arguments_are_refused_on_the_host(lib):
    import ctypes
    ok = ctypes.c_void_p(0x10000)
    rc = lib.csx_residual_cl(None, 2, ok, 12, 6, 3, None, ok, 1, ok, ok, ok, None)
    assert rc == -1 and b"plan is NULL" in lib.csx_last_error()


def test_patch_counts_are_bounded_on_the_host(lib):
    """K_j above CSX_MAX_K (where sizes such as P = K_d + K_T + K_s would leave 32-bit range) are
    refused before anything touches a device; so is per-pixel noise for the cell-moment call. The
    pointers below are never dereferenced."""
    import ctypes
    from paper_2604_08463_b300 import csx
    model = csx.Model(np.array([40.0, 100.0, 402.0]))
    sky = csx.CSky()
    sky.npix, sky.nreal, sky.noise_kind = 10, 1, 0
    for f in range(3):
        sky.ninv_band[f] = 1.0
    ok = ctypes.c_void_p(0x10000)
    sky.d = 0x10000
    big = (ctypes.c_int32 * 3)(2 ** 31 - 1, 2 ** 30, 2)
    rc = lib.csx_spectral_grad(ctypes.byref(model.c), ctypes.byref(sky), ok, big, 1, ok, ok, ok, None)
    assert rc == -1 and b"K_j" in lib.csx_last_error()
    rc = lib.csx_spectral_grad_noalloc(ctypes.byref(model.c), ctypes.byref(sky), ok, big, 1, ok, ok,
                                       ok, None)
    assert rc == -1 and b"K_j" in lib.csx_last_error()
    rc = lib.csx_cell_like_grad(ctypes.byref(model.c), ctypes.byref(sky), ok, big, 1, ok, ok, ok,
                                ok, None)
    assert rc == -1 and b"K_j" in lib.csx_last_error()
    opts = csx.fit_options()
    rc = lib.csx_fit_batch(ctypes.byref(model.c), ctypes.byref(sky), 1, ok, big, ctypes.byref(opts),
                           ok, ok, ok, ok, ok, None, None)
    assert rc == -1 and b"K_j" in lib.csx_last_error()
    small = (ctypes.c_int32 * 3)(2, 2, 2)
    sky.noise_kind = 2
    sky.ninv_pix = 0x10000
    rc = lib.csx_cell_like_grad(ctypes.byref(model.c), ctypes.byref(sky), ok, small, 1, ok, ok, ok,
                                ok, None)
    assert rc == -1 and b"homogeneous or separable" in lib.csx_last_error()


def test_spectral_plan_arguments_are_refused_on_the_host(lib):
    """The cell plan's entry points check their arguments before touching a device; destroying
    NULL is a no-op. The pointers below are never dereferenced."""
    import ctypes
    plan = ctypes.c_void_p()
    ok = ctypes.c_void_p(0x10000)
    K = (ctypes.c_int32 * 3)(4, 2, 3)
    rc = lib.csx_spectral_plan_create(-1, ok, K, None, ctypes.byref(plan))
    assert rc == -1 and b"npix" in lib.csx_last_error() and not plan.value
    big = (ctypes.c_int32 * 3)(2 ** 31 - 1, 2 ** 30, 2)
    rc = lib.csx_spectral_plan_create(10, ok, big, None, ctypes.byref(plan))
    assert rc == -1 and b"K_j" in lib.csx_last_error() and not plan.value
    rc = lib.csx_spectral_plan_create(10, None, K, None, ctypes.byref(plan))
    assert rc == -1 and b"labels is NULL" in lib.csx_last_error()
    rc = lib.csx_spectral_plan_create(10, ok, K, None, None)
    assert rc == -1 and b"plan is NULL" in lib.csx_last_error()
    n = ctypes.c_int32()
    assert lib.csx_spectral_plan_ncell(None, ctypes.byref(n)) == -1
    rc = lib.csx_spectral_grad_plan(None, None, None, 1, ok, ok, ok, None)
    assert rc == -1 and b"plan is NULL" in lib.csx_last_error()
    assert lib.csx_spectral_plan_destroy(None) == 0
