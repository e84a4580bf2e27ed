"""ctypes binding of libcsx (include/csx.h). Argument marshalling only: every step of the method
runs in the CUDA library. Device buffers are torch CUDA tensors; work is enqueued on torch's
current CUDA stream. There is no CPU fallback: a missing library raises."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int32, c_void_p

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcsx.so")

NB = 16
NMETRIC = 8
NOISE = {"homogeneous": 0, "separable": 1, "perpixel": 2}
PATH = {"auto": 0, "stream": 1, "moment": 2}
GRAD = {"adjoint": 0, "fd": 1}
SOLVER = {"lbfgs": 0, "adatopk": 1}
STATUS = {0: "converged", 1: "max_iter", 2: "nonphysical", 3: "line_search", 4: "bad_label"}
M_SYS_SQ, M_STAT, M_CMB_Q, M_CMB_Q2, M_CMB_U, M_CMB_U2, M_NPIX = range(7)

EXPORTS = ["csx_version", "csx_last_error", "csx_release", "csx_device_status",
           "csx_stream_schedule", "csx_fit_defaults", "csx_mixing",
           "csx_spectral_like", "csx_spectral_grad", "csx_spectral_grad_f64",
           "csx_spectral_grad_noalloc", "csx_spectral_plan_create", "csx_spectral_plan_destroy",
           "csx_spectral_plan_ncell", "csx_spectral_grad_plan",
           "csx_cell_like_grad", "csx_build_cells", "csx_fit_batch", "csx_reconstruct",
           "csx_select", "csx_kmeans", "csx_sht_plan_create", "csx_sht_plan_destroy",
           "csx_pseudo_cl", "csx_residual_cl"]


class CsxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("csx error %d: %s" % (code, msg))
        self.code = code


class CModel(ctypes.Structure):
    _fields_ = [("nfreq", c_int32), ("units", c_int32), ("nu_ghz", c_double * NB),
                ("nu0_dust_ghz", c_double), ("nu0_sync_ghz", c_double), ("t_cmb", c_double)]


class CSky(ctypes.Structure):
    _fields_ = [("npix", c_int32), ("nreal", c_int32), ("noise_kind", c_int32),
                ("reserved", c_int32), ("d", c_void_p), ("ninv_band", c_float * NB),
                ("w", c_void_p), ("ninv_pix", c_void_p)]


class CFitOpts(ctypes.Structure):
    _fields_ = [("max_iter", c_int32), ("history", c_int32), ("max_ls", c_int32),
                ("path", c_int32), ("grad_mode", c_int32), ("threads", c_int32),
                ("lower", c_float * 3), ("upper", c_float * 3), ("xtol", c_float * 3),
                ("fd_step", c_float), ("solver", c_int32), ("topk", c_float)]


_lib = None


def lib():
    """Load libcsx.so (raises if it is missing: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcsx.so not built (run paper_2604_08463_b300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, pi32 = c_void_p, c_int32, POINTER(c_int32)
        L.csx_version.restype = ctypes.c_char_p
        L.csx_last_error.restype = ctypes.c_char_p
        L.csx_release.restype = i32
        L.csx_device_status.argtypes = [vp]
        L.csx_stream_schedule.argtypes = [i32, i32, pi32]
        L.csx_fit_defaults.argtypes = [POINTER(CFitOpts)]
        L.csx_mixing.argtypes = [POINTER(CModel), i32, vp, vp, vp, vp]
        L.csx_spectral_like.argtypes = [POINTER(CModel), POINTER(CSky), vp, pi32, i32, vp, vp, vp]
        L.csx_spectral_grad.argtypes = [POINTER(CModel), POINTER(CSky), vp, pi32, i32, vp, vp, vp, vp]
        L.csx_spectral_grad_f64.argtypes = [POINTER(CModel), POINTER(CSky), vp, pi32, i32, vp, vp,
                                            vp, vp]
        L.csx_spectral_grad_noalloc.argtypes = [POINTER(CModel), POINTER(CSky), vp, pi32, i32, vp,
                                                vp, vp, vp]
        L.csx_spectral_plan_create.argtypes = [i32, vp, pi32, vp, POINTER(c_void_p)]
        L.csx_spectral_plan_destroy.argtypes = [vp]
        L.csx_spectral_plan_ncell.argtypes = [vp, pi32]
        L.csx_spectral_grad_plan.argtypes = [vp, POINTER(CModel), POINTER(CSky), i32, vp, vp, vp, vp]
        L.csx_cell_like_grad.argtypes = [POINTER(CModel), POINTER(CSky), vp, pi32, i32, vp, vp,
                                         vp, vp, vp]
        L.csx_build_cells.argtypes = [i32, i32, vp, pi32, vp, vp, vp, vp]
        L.csx_fit_batch.argtypes = [POINTER(CModel), POINTER(CSky), i32, vp, pi32,
                                    POINTER(CFitOpts), vp, vp, vp, vp, vp, vp, vp]
        L.csx_reconstruct.argtypes = [POINTER(CModel), POINTER(CSky), i32, vp, pi32, vp, vp, vp,
                                      vp, vp, vp, vp]
        L.csx_select.argtypes = [i32, i32, vp, vp, vp, vp]
        L.csx_kmeans.argtypes = [vp, i32, i32, pi32, vp, i32, vp, vp, vp]
        L.csx_sht_plan_create.argtypes = [i32, i32, pi32, i32, POINTER(c_void_p), vp]
        L.csx_sht_plan_destroy.argtypes = [vp]
        L.csx_pseudo_cl.argtypes = [vp, i32, vp, ctypes.c_int64, i32, i32, vp, vp, i32, vp, vp]
        L.csx_residual_cl.argtypes = [vp, i32, vp, ctypes.c_int64, i32, i32, vp, vp, i32, vp, vp,
                                      vp, vp]
        for name in EXPORTS:
            if name not in ("csx_version", "csx_last_error"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise CsxError(rc, lib().csx_last_error().decode())


def _stream():
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return c_void_p(t.data_ptr())


def _host_i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(POINTER(c_int32))


class Model:
    """Spectral model of Eq. 5: band centres (GHz), reference frequencies, units."""

    def __init__(self, nu_ghz, nu0_dust=353.0, nu0_sync=23.0, t_cmb=2.7255, units="K_CMB"):
        nu = np.asarray(nu_ghz, dtype=np.float64)
        self.c = CModel()
        self.c.nfreq = nu.size
        self.c.units = 0 if units == "K_CMB" else 1
        for f in range(nu.size):
            self.c.nu_ghz[f] = nu[f]
        self.c.nu0_dust_ghz = nu0_dust
        self.c.nu0_sync_ghz = nu0_sync
        self.c.t_cmb = t_cmb
        self.nfreq = nu.size


class Sky:
    """Device-resident data and noise (Eq. 1).

    d: float32 [nreal, npix, 2, 16] CUDA tensor; noise "homogeneous" (ninv_band),
    "separable" (ninv_band, w [npix]) or "perpixel" (ninv_pix [npix, 16])."""

    def __init__(self, d, noise="homogeneous", ninv_band=None, w=None, ninv_pix=None):
        assert d.dtype == torch.float32 and d.dim() == 4 and d.shape[2] == 2 and d.shape[3] == NB
        self.d = d.contiguous()
        self.w = None if w is None else w.to(torch.float32).contiguous()
        self.ninv_pix = None if ninv_pix is None else ninv_pix.to(torch.float32).contiguous()
        self.noise = noise
        self.c = CSky()
        self.c.npix = d.shape[1]
        self.c.nreal = d.shape[0]
        self.c.noise_kind = NOISE[noise]
        self.c.d = self.d.data_ptr() if d.numel() else None
        if ninv_band is not None:
            nb = np.asarray(ninv_band, dtype=np.float32)
            for f in range(nb.size):
                self.c.ninv_band[f] = float(nb[f])
        self.c.w = self.w.data_ptr() if self.w is not None and self.w.numel() else None
        self.c.ninv_pix = (self.ninv_pix.data_ptr() if self.ninv_pix is not None and
                           self.ninv_pix.numel() else None)

    @property
    def npix(self):
        return self.c.npix

    @property
    def nreal(self):
        return self.c.nreal

    def subset(self, nreal):
        """A view on the first nreal realizations."""
        s = Sky.__new__(Sky)
        s.__dict__.update(self.__dict__)
        s.c = CSky.from_buffer_copy(self.c)
        s.c.nreal = nreal
        return s


def version():
    return lib().csx_version().decode()


def release():
    _check(lib().csx_release())


STREAM_SCHEDULES = ((128, 2), (64, 2), (64, 3), (128, 3), (128, 4), (256, 2))


def stream_schedule(tile=None, stages=None):
    """Select the streaming kernel's (pixels per tile, stages) for the calls that follow (None: keep
    the current one; (0, 0): the default); returns the schedule in force as a tuple."""
    cur = (c_int32 * 2)()
    t = -1 if tile is None else int(tile)
    st = -1 if stages is None else int(stages)
    _check(lib().csx_stream_schedule(t, st, cur))
    return int(cur[0]), int(cur[1])


def device_status():
    """Raise CsxError (CSX_ETIMEOUT) if a bounded device wait gave up since the last check;
    synchronises torch's current stream."""
    _check(lib().csx_device_status(_stream()))


def mixing(model: Model, beta: torch.Tensor, want_derivatives=True):
    """A [n, 16, 3] and dA [n, 3, 16] for beta [n, 3] = (beta_d, T_d, beta_s)."""
    beta = beta.to(torch.float32).contiguous()
    n = beta.shape[0]
    A = torch.empty((n, NB, 3), device=beta.device, dtype=torch.float32)
    dA = torch.empty((n, 3, NB), device=beta.device, dtype=torch.float32) if want_derivatives else None
    _check(lib().csx_mixing(ctypes.byref(model.c), n, _ptr(beta), _ptr(A), _ptr(dA), _stream()))
    return A, dA


def spectral_like(model: Model, sky: Sky, labels, K, beta):
    """L [nprob] (float64) for one configuration; beta [nprob, P], problem i uses realization i."""
    K, Kp = _host_i32(K)
    beta = beta.to(torch.float32).contiguous()
    L = torch.empty(beta.shape[0], device=beta.device, dtype=torch.float64)
    _check(lib().csx_spectral_like(ctypes.byref(model.c), ctypes.byref(sky.c), _ptr(labels), Kp,
                                   beta.shape[0], _ptr(beta), _ptr(L), _stream()))
    return L


def spectral_grad(model: Model, sky: Sky, labels, K, beta):
    """(L [nprob] float64, grad [nprob, P] float32)."""
    K, Kp = _host_i32(K)
    beta = beta.to(torch.float32).contiguous()
    L = torch.empty(beta.shape[0], device=beta.device, dtype=torch.float64)
    g = torch.empty_like(beta)
    _check(lib().csx_spectral_grad(ctypes.byref(model.c), ctypes.byref(sky.c), _ptr(labels), Kp,
                                   beta.shape[0], _ptr(beta), _ptr(L), _ptr(g), _stream()))
    return L, g


class SpectralPlan:
    """Cell plan of one patch configuration (labels [3, npix] int32 on the device, K) for repeated
    streaming evaluations at changing beta (csx_spectral_plan_create; freed with the object)."""

    def __init__(self, labels: torch.Tensor, K):
        K, Kp = _host_i32(K)
        self.K = K
        self.npix = int(labels.shape[-1])
        self._labels = labels  # kept alive while the plan is built
        h = c_void_p()
        _check(lib().csx_spectral_plan_create(self.npix, _ptr(labels), Kp, _stream(), ctypes.byref(h)))
        self._h = h
        n = c_int32()
        _check(lib().csx_spectral_plan_ncell(self._h, ctypes.byref(n)))
        self.ncell = int(n.value)

    def grad(self, model: "Model", sky: "Sky", beta, want_grad=True):
        """(L [nprob] float64, grad [nprob, P] float32 or None) of csx_spectral_grad_plan."""
        beta = beta.to(torch.float32).contiguous()
        L = torch.empty(beta.shape[0], device=beta.device, dtype=torch.float64)
        g = torch.empty_like(beta) if want_grad else None
        _check(lib().csx_spectral_grad_plan(self._h, ctypes.byref(model.c), ctypes.byref(sky.c),
                                            beta.shape[0], _ptr(beta), _ptr(L), _ptr(g), _stream()))
        return L, g

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().csx_spectral_plan_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spectral_grad_f64(model: Model, sky: Sky, labels, K, beta, want_grad=True):
    """(L [nprob] float64, grad [nprob, P] float64 or None) with every operation in FP64."""
    K, Kp = _host_i32(K)
    beta = beta.to(torch.float64).contiguous()
    L = torch.empty(beta.shape[0], device=beta.device, dtype=torch.float64)
    g = torch.empty_like(beta) if want_grad else None
    _check(lib().csx_spectral_grad_f64(ctypes.byref(model.c), ctypes.byref(sky.c), _ptr(labels), Kp,
                                       beta.shape[0], _ptr(beta), _ptr(L), _ptr(g), _stream()))
    return L, g


def spectral_grad_noalloc(model: Model, sky: Sky, labels, K, beta, L, grad):
    """csx_spectral_grad_noalloc into caller-provided outputs: the library allocates no device
    memory for this call (for callers whose device memory is owned by their own allocator or
    budget). Every tensor must already have the layout the C entry point reads, on the data's
    device: beta float32 [nprob, P], L float64 [nprob], grad float32 [nprob, P], labels int32
    [3, npix], all contiguous; nothing is converted or copied here (a conversion would allocate),
    and anything else is refused before the call."""
    K, Kp = _host_i32(K)
    if K.shape != (3,):
        raise ValueError("K must hold three patch counts")
    P = int(K.astype(np.int64).sum())
    dev = sky.d.device
    want = (("beta", beta, torch.float32), ("L", L, torch.float64), ("grad", grad, torch.float32),
            ("labels", labels, torch.int32))
    for name, t, dt in want:
        if not isinstance(t, torch.Tensor) or t.device != dev or t.dtype != dt or \
                not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor on %s" % (name, dt, dev))
    if beta.dim() != 2 or beta.shape[1] != P:
        raise ValueError("beta must be [nprob, %d]" % P)
    nprob = beta.shape[0]
    if L.shape != (nprob,):
        raise ValueError("L must be [%d]" % nprob)
    if grad.shape != (nprob, P):
        raise ValueError("grad must be [%d, %d]" % (nprob, P))
    if labels.shape != (3, sky.npix):
        raise ValueError("labels must be [3, %d]" % sky.npix)
    _check(lib().csx_spectral_grad_noalloc(ctypes.byref(model.c), ctypes.byref(sky.c), _ptr(labels),
                                           Kp, nprob, _ptr(beta), _ptr(L), _ptr(grad), _stream()))
    return L, grad


def cell_like_grad(model: Model, sky: Sky, labels, K, beta_ref, beta):
    """(L [nprob] float64, grad [nprob, P] float32) at beta [nprob, P] by the fit's cell-moment
    evaluation, the moments formed about beta_ref [nprob, P] (homogeneous or separable noise)."""
    K, Kp = _host_i32(K)
    beta_ref = beta_ref.to(torch.float32).contiguous()
    beta = beta.to(torch.float32).contiguous()
    if beta.shape != beta_ref.shape:
        raise ValueError("beta and beta_ref must have the same shape")
    L = torch.empty(beta.shape[0], device=beta.device, dtype=torch.float64)
    g = torch.empty_like(beta)
    _check(lib().csx_cell_like_grad(ctypes.byref(model.c), ctypes.byref(sky.c), _ptr(labels), Kp,
                                    beta.shape[0], _ptr(beta_ref), _ptr(beta), _ptr(L), _ptr(g),
                                    _stream()))
    return L, g


def build_cells(labels: torch.Tensor, K):
    """(perm [C, npix], cell_off [C, npix+1], ncell [C]) int32 for labels [C, 3, npix]."""
    C, _, npix = labels.shape
    K, Kp = _host_i32(K)
    dev = labels.device
    perm = torch.empty((C, npix), dtype=torch.int32, device=dev)
    off = torch.empty((C, npix + 1), dtype=torch.int32, device=dev)
    nc = torch.empty(C, dtype=torch.int32, device=dev)
    _check(lib().csx_build_cells(npix, C, _ptr(labels), Kp, _ptr(perm), _ptr(off), _ptr(nc),
                                 _stream()))
    return perm, off, nc


def fit_options(**kw) -> CFitOpts:
    o = CFitOpts()
    _check(lib().csx_fit_defaults(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "path":
            v = PATH[v] if isinstance(v, str) else v
        if k == "grad_mode":
            v = GRAD[v] if isinstance(v, str) else v
        if k == "solver":
            v = SOLVER[v] if isinstance(v, str) else v
        if k in ("lower", "upper", "xtol"):
            arr = getattr(o, k)
            for j in range(3):
                arr[j] = float(v[j])
            continue
        setattr(o, k, v)
    return o


def param_offsets(K, nreal):
    """Start of each problem's parameters in the packed layout (problem q = c * nreal + n)."""
    K = np.asarray(K, dtype=np.int64)
    P = K.sum(axis=1)
    coff = np.concatenate([[0], np.cumsum(P)[:-1]])
    q = []
    for c in range(K.shape[0]):
        for n in range(nreal):
            q.append(nreal * coff[c] + n * P[c])
    return np.array(q, dtype=np.int64), P


def fit_batch(model: Model, sky: Sky, labels, K, beta0, **opts):
    """Fit every (configuration, realization) problem. Returns dict of device tensors."""
    K, Kp = _host_i32(K)
    nconf = K.shape[0]
    nprob = nconf * sky.nreal
    dev = sky.d.device
    beta0 = beta0.to(torch.float32).contiguous()
    out = torch.empty_like(beta0)
    L = torch.empty(nprob, dtype=torch.float64, device=dev)
    st = torch.empty(nprob, dtype=torch.int32, device=dev)
    it = torch.empty(nprob, dtype=torch.int32, device=dev)
    ne = torch.empty(nprob, dtype=torch.int32, device=dev)
    o = fit_options(**opts)
    _check(lib().csx_fit_batch(ctypes.byref(model.c), ctypes.byref(sky.c), nconf, _ptr(labels),
                               Kp, ctypes.byref(o), _ptr(beta0), _ptr(out), _ptr(L), _ptr(st),
                               _ptr(it), _ptr(ne), _stream()))
    return {"beta": out, "L": L, "status": st, "iters": it, "nevals": ne}


def reconstruct(model: Model, sky: Sky, labels, K, beta, d_fg=None, s_hat=False, sigma2=False,
                r_sys=False, metrics=True):
    """s_hat, sigma2, r_sys and per-problem metric sums at beta (packed per problem, the layout
    of fit_batch: problem q = c * nreal + n)."""
    K, Kp = _host_i32(K)
    nprob = K.shape[0] * sky.nreal
    dev = sky.d.device
    npix = sky.npix
    sh = torch.empty((nprob, npix, 2, 3), dtype=torch.float32, device=dev) if s_hat else None
    sv = torch.empty((nprob, npix), dtype=torch.float32, device=dev) if sigma2 else None
    rs = torch.empty((nprob, npix, 2), dtype=torch.float32, device=dev) if r_sys else None
    me = torch.empty((nprob, NMETRIC), dtype=torch.float64, device=dev) if metrics else None
    beta = beta.to(torch.float32).contiguous()
    _check(lib().csx_reconstruct(ctypes.byref(model.c), ctypes.byref(sky.c), K.shape[0],
                                 _ptr(labels), Kp, _ptr(beta), _ptr(d_fg), _ptr(sh), _ptr(sv),
                                 _ptr(rs), _ptr(me), _stream()))
    return {"s_hat": sh, "sigma2": sv, "r_sys": rs, "metrics": me}


def select(metrics: torch.Tensor, nconf: int, nreal: int):
    """(vtot [nconf] float64, best [1] int32) by total residual variance."""
    v = torch.empty(nconf, dtype=torch.float64, device=metrics.device)
    b = torch.empty(1, dtype=torch.int32, device=metrics.device)
    _check(lib().csx_select(nconf, nreal, _ptr(metrics.contiguous()), _ptr(v), _ptr(b), _stream()))
    return v, b


def kmeans(vec: torch.Tensor, K, init, max_iter: int = 30):
    """Seeded spherical K-means labels (Sec. 2.2) for every cluster count in K at once.

    vec: [n, 3] float64 CUDA unit vectors; K: sequence of cluster counts; init: for each K with
    1 < K < n, its K distinct starting pixels (the seeded draw is the caller's). Returns
    (labels [len(K), n] int32, iters [len(K)] int32) as device tensors."""
    vec = vec.to(torch.float64).contiguous()
    n = vec.shape[0]
    Kh, Kp = _host_i32(np.asarray(K).reshape(-1))
    nvalid = int(((Kh > 1) & (Kh < n)).sum())
    if len(init) != nvalid:
        raise ValueError("init needs one array per cluster count with 1 < K < n (%d)" % nvalid)
    parts = [np.asarray(x, dtype=np.int32) for x in init]
    flat = np.concatenate(parts) if parts else np.zeros(1, np.int32)
    init_d = torch.from_numpy(flat).to(vec.device)
    labels = torch.empty((Kh.size, n), dtype=torch.int32, device=vec.device)
    iters = torch.empty(Kh.size, dtype=torch.int32, device=vec.device)
    _check(lib().csx_kmeans(_ptr(vec), n, int(Kh.size), Kp, _ptr(init_d), int(max_iter),
                            _ptr(labels), _ptr(iters), _stream()))
    return labels, iters


class ShtPlan:
    """Ring geometry and spin-2 harmonic tables of the observed pixels `pix` (RING, nside) up to
    lmax, on the current CUDA device (csx_sht_plan_create; freed with the object)."""

    def __init__(self, nside: int, lmax: int, pix):
        pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32).reshape(-1))
        self.nside, self.lmax, self.npix = int(nside), int(lmax), int(pix.size)
        self._pix = pix
        h = c_void_p()
        _check(lib().csx_sht_plan_create(self.nside, self.lmax,
                                         pix.ctypes.data_as(POINTER(c_int32)), self.npix,
                                         ctypes.byref(h), _stream()))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().csx_sht_plan_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pseudo_cl(plan: ShtPlan, maps: torch.Tensor, sub_common=None, sub_each=None, navg: int = 1):
    """(EE, BB) pseudo-spectra [nmaps // navg, 2, lmax + 1] (float64) of the Q, U maps
    maps[b, p, k] (k = 0 Q, 1 U; any strides in the last two dims, e.g. s_hat[..., 0] of
    `reconstruct`), minus sub_common [npix, 2] and sub_each [nmaps, npix, 2] when given, averaged
    over consecutive groups of navg maps."""
    if maps.dim() != 3 or maps.shape[1] != plan.npix or maps.shape[2] != 2:
        raise ValueError("maps must be [nmaps, npix, 2]")
    if maps.dtype != torch.float32:
        raise ValueError("maps must be float32")
    nmaps = maps.shape[0]
    if sub_common is not None:
        sub_common = sub_common.to(torch.float32).contiguous()
    if sub_each is not None:
        sub_each = sub_each.to(torch.float32).contiguous()
    if not maps.is_cuda:
        raise ValueError("maps must be a CUDA tensor")
    st = maps.stride()
    cl = torch.empty((nmaps // max(navg, 1), 2, plan.lmax + 1), dtype=torch.float64,
                     device=maps.device)
    _check(lib().csx_pseudo_cl(plan._h, nmaps, c_void_p(maps.data_ptr()), st[0], st[1], st[2],
                               _ptr(sub_common),
                               _ptr(sub_each), int(navg), _ptr(cl), _stream()))
    return cl


def residual_spectra(plan: ShtPlan, s_hat: torch.Tensor, s_true: torch.Tensor, r_sys, nreal: int):
    """The residual spectra of Sec. 2.5 for every configuration, averaged over its nreal noise
    realizations: s_hat [nprob, npix, 2, 3] and r_sys [nprob, npix, 2] of `reconstruct` (problem
    q = c * nreal + n), s_true [npix, 2] the input CMB. Returns {'tot', 'syst', 'stat'}, each
    [nconf, 2, lmax + 1] (EE, BB). One pass: the ring coefficients of s_hat - s_true and of r_sys
    are taken once and a_lm of their difference is the difference of theirs."""
    if s_hat.dim() != 4 or s_hat.shape[1] != plan.npix or s_hat.shape[2:] != (2, 3):
        raise ValueError("s_hat must be [nprob, npix, 2, 3]")
    if s_hat.dtype != torch.float32 or not s_hat.is_cuda:
        raise ValueError("s_hat must be a float32 CUDA tensor")
    nprob = s_hat.shape[0]
    r_sys = r_sys.to(torch.float32).contiguous()
    s_true = s_true.to(torch.float32).contiguous() if s_true is not None else None
    st = s_hat.stride()
    out = {k: torch.empty((nprob // max(nreal, 1), 2, plan.lmax + 1), dtype=torch.float64,
                          device=s_hat.device) for k in ("tot", "syst", "stat")}
    _check(lib().csx_residual_cl(plan._h, nprob, c_void_p(s_hat.data_ptr()), st[0], st[1], st[2],
                                 _ptr(s_true), _ptr(r_sys), int(nreal), _ptr(out["tot"]),
                                 _ptr(out["syst"]), _ptr(out["stat"]), _stream()))
    return out


def chunk(n: int, world: int, rank: int):
    """Contiguous share [lo, hi) of n independent problems (or configurations) for `rank` of
    `world` processes: [floor(k n / W), floor((k + 1) n / W)) (Sec. 3.1)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need n >= 0 and 0 <= rank < world")
    return (rank * n) // world, ((rank + 1) * n) // world


def gather_metrics(metrics: torch.Tensor, group=None):
    """The path's one exchange across processes: every rank holds the metric rows
    [n_r, CSX_NMETRIC] (float64) of its own problems, numbered in rank order in the global problem
    list; every rank receives all rows, concatenated in rank order (one all-gather of the sizes,
    one of the padded rows; nccl for CUDA tensors, gloo for host tensors)."""
    import torch.distributed as dist
    if metrics.dim() != 2 or metrics.shape[1] != NMETRIC or metrics.dtype != torch.float64:
        raise ValueError("metrics must be float64 [n, %d]" % NMETRIC)
    world = dist.get_world_size(group)
    n = torch.tensor([metrics.shape[0]], dtype=torch.int64, device=metrics.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    pad = torch.zeros((max(sizes), NMETRIC), dtype=torch.float64, device=metrics.device)
    pad[: metrics.shape[0]] = metrics
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad.contiguous(), group=group)
    return torch.cat([p[:k] for p, k in zip(parts, sizes)]).contiguous()


def gather_select(metrics: torch.Tensor, nreal: int, group=None):
    """Selection across processes: gather_metrics, then csx_select over all configurations (each
    rank holds whole configurations, nreal problems each) on this rank's device. Returns (V_tot of
    every configuration [nconf_total] float64, index of the best [1] int32), as csx_select."""
    allm = gather_metrics(metrics, group)
    if allm.shape[0] % nreal:
        raise ValueError("every rank must hold whole configurations")
    return select(allm, allm.shape[0] // nreal, nreal)


class SpectralLikelihood(torch.autograd.Function):
    """L(beta) for one configuration as a differentiable torch op (Sec. 3.3.1).

    forward: csx_spectral_grad (one streaming pass gives L and dL/dbeta; FP32 arithmetic with FP64
    sums) or, with precision="fp64", csx_spectral_grad_f64 (every operation in FP64); only the
    gradient [nprob, P] is saved, no per-pixel intermediate. backward: grad_output[:, None] *
    dL/dbeta, in beta's dtype."""

    @staticmethod
    def forward(ctx, beta, model, sky, labels, K, precision="fp32"):
        if precision == "fp64":
            L, g = spectral_grad_f64(model, sky, labels, K, beta.detach())
        elif precision == "fp32":
            L, g = spectral_grad(model, sky, labels, K, beta.detach())
        else:
            raise ValueError("precision must be 'fp32' or 'fp64'")
        ctx.save_for_backward(g)
        ctx.beta_dtype = beta.dtype
        return L

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        gb = grad_out.to(torch.float64)[:, None] * g.to(torch.float64)
        return gb.to(ctx.beta_dtype), None, None, None, None, None
