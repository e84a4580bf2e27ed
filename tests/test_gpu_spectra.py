"""Parity of the pseudo-C_ell kernels (residual spectra of Sec. 2.5) with the oracle: ragged
masked rings, strided inputs with subtraction and group averages, the aliasing edge lmax = 4 nside
- 1, degenerate plans, rotated pure-E / pure-B patterns, the scan's cut sky at nside 64 to
l = 150 (chunked launches), and the residual spectra of reconstructed maps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import spectra as osp  # noqa: E402
from synth import healpix  # noqa: E402
from tests._inputs import pack, scan_case  # noqa: E402
from tests.test_oracle_spectra import _quadrupole  # noqa: E402

# FP32 ring sums and harmonic sums: C_l to 1e-4 relative, plus an absolute floor of 1e-6 of the
# largest multipole's power (a_lm accumulated from terms of that size in float32)
RTOL, ATOL_REL = 1e-4, 1e-6


@pytest.fixture(scope="module")
def csx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08463_b300 import csx as mod
    mod.lib()
    return mod


def _close(got, ref):
    ref = np.asarray(ref)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=ATOL_REL * np.abs(ref).max())


def _masked(nside, frac, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(healpix.npix(nside), int(frac * healpix.npix(nside)), replace=False))


def test_pseudo_cl_ragged_masked_rings(csx):
    nside = 8
    pix = _masked(nside, 0.7, 1)
    rng = np.random.default_rng(2)
    maps = rng.normal(size=(11, pix.size, 2)).astype(np.float32)
    for lmax in (3 * nside - 1, 4 * nside - 1):  # the second aliases m >= ring length near the poles
        plan = csx.ShtPlan(nside, lmax, pix)
        got = csx.pseudo_cl(plan, torch.from_numpy(maps).cuda()).cpu().numpy()
        ref = osp.pseudo_cl(nside, pix, maps.astype(np.float64), lmax)
        _close(got, ref)
        assert np.all(got[:, :, :2] == 0.0)


def test_strided_input_subtraction_and_group_average(csx):
    """maps read through s_hat-like strides [nmaps][npix][2][3], minus a common and a per-map
    map, averaged over groups of 3."""
    nside, lmax = 8, 20
    pix = _masked(nside, 0.55, 3)
    rng = np.random.default_rng(4)
    s_hat = rng.normal(size=(9, pix.size, 2, 3)).astype(np.float32)
    s_true = rng.normal(size=(pix.size, 2)).astype(np.float32)
    r_sys = (0.3 * rng.normal(size=(9, pix.size, 2))).astype(np.float32)
    plan = csx.ShtPlan(nside, lmax, pix)
    t = torch.from_numpy(s_hat).cuda()
    got = csx.residual_spectra(plan, t, torch.from_numpy(s_true).cuda(),
                               torch.from_numpy(r_sys).cuda(), nreal=3)
    for c in range(3):
        sl = slice(3 * c, 3 * c + 3)
        ref = osp.residual_spectra(nside, pix, s_hat[sl, :, :, 0].astype(np.float64), s_true,
                                   r_sys[sl], lmax)
        for k in ("tot", "syst", "stat"):
            _close(got[k][c].cpu().numpy(), ref[k])


def test_degenerate_plans(csx):
    rng = np.random.default_rng(5)
    # lmax < 2: no spin-2 power at all
    plan = csx.ShtPlan(4, 1, np.arange(healpix.npix(4)))
    m = torch.from_numpy(rng.normal(size=(2, healpix.npix(4), 2)).astype(np.float32)).cuda()
    assert not csx.pseudo_cl(plan, m).cpu().numpy().any()
    # no observed pixel
    plan = csx.ShtPlan(4, 8, np.zeros(0, np.int32))
    assert not csx.pseudo_cl(plan, torch.zeros((3, 0, 2), device="cuda")).cpu().numpy().any()
    # one pixel, the last of the sky (south polar ring)
    nside, lmax = 4, 15
    pix = np.array([healpix.npix(nside) - 1])
    mp = rng.normal(size=(1, 1, 2)).astype(np.float32)
    plan = csx.ShtPlan(nside, lmax, pix)
    _close(csx.pseudo_cl(plan, torch.from_numpy(mp).cuda()).cpu().numpy(),
           osp.pseudo_cl(nside, pix, mp.astype(np.float64), lmax))
    # no maps
    assert csx.pseudo_cl(plan, torch.zeros((0, 1, 2), device="cuda")).shape == (0, 2, lmax + 1)


def test_rotated_quadrupoles_pure_e_and_b(csx):
    nside, lmax = 16, 10
    pix = np.arange(healpix.npix(nside))
    n0 = np.array([0.3, -0.5, 0.81])
    n0 /= np.linalg.norm(n0)
    maps = np.stack([_quadrupole(nside, n0, "E"), _quadrupole(nside, n0, "B")]).astype(np.float32)
    plan = csx.ShtPlan(nside, lmax, pix)
    got = csx.pseudo_cl(plan, torch.from_numpy(maps).cuda()).cpu().numpy()
    c2 = 128.0 * np.pi / 75.0
    for k in (0, 1):
        assert abs(got[k, k, 2] / c2 - 1.0) < 1e-3
        assert got[k, 1 - k, 2] < 1e-6 * c2   # float32 floor: no quadrupole in the other mode
        assert got[k].max() <= got[k, k, 2]


def test_scan_cut_sky_nside64_to_l150(csx):
    """The scan's |b| > 20 deg pixels at nside 64, l <= 150 (the multipole range of the paper's
    r-likelihood), 700 maps: two chunks of ring coefficients, groups of 7 straddling the chunk
    boundary; sampled maps against the oracle, groups against the mean of their maps."""
    nside, lmax = 64, 150
    z, _ = healpix.pixel_centres(nside)
    pix = np.nonzero(np.abs(z) > np.sin(np.deg2rad(20.0)))[0]
    rng = np.random.default_rng(6)
    maps = torch.from_numpy(rng.normal(size=(700, pix.size, 2)).astype(np.float32)).cuda()
    plan = csx.ShtPlan(nside, lmax, pix)
    one = csx.pseudo_cl(plan, maps).cpu().numpy()
    grp = csx.pseudo_cl(plan, maps, navg=7).cpu().numpy()
    np.testing.assert_allclose(grp, one.reshape(100, 7, 2, lmax + 1).mean(axis=1), rtol=1e-6)
    picks = [0, 353, 699]
    ref = osp.pseudo_cl(nside, pix, maps[picks].cpu().numpy().astype(np.float64), lmax)
    _close(one[picks], ref)


def test_residual_spectra_of_reconstructed_maps(csx):
    """s_hat and r_sys from the reconstruction kernel at given parameters, then the three spectra;
    the oracle takes the same float32 maps."""
    case = scan_case(nside=16, nconf=2, kmax=10, nreal=3)
    wl = case.wl
    model, sky, labels = case.gpu()
    beta = pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)])
    fg = torch.tensor(case.fg32, device="cuda")
    out = csx.reconstruct(model, sky, labels, wl.K, torch.tensor(beta, device="cuda"), d_fg=fg,
                          s_hat=True, r_sys=True, metrics=False)
    s_true = torch.tensor(np.asarray(wl.sky.cmb, dtype=np.float32), device="cuda")
    lmax = 3 * 16 - 1
    plan = csx.ShtPlan(16, lmax, wl.sky.pix)
    got = csx.residual_spectra(plan, out["s_hat"], s_true, out["r_sys"], wl.nreal)
    sh = out["s_hat"].cpu().numpy()[..., 0].astype(np.float64)
    rs = out["r_sys"].cpu().numpy().astype(np.float64)
    st = s_true.cpu().numpy().astype(np.float64)
    for c in range(wl.nconf):
        sl = slice(c * wl.nreal, (c + 1) * wl.nreal)
        ref = osp.residual_spectra(16, wl.sky.pix, sh[sl], st, rs[sl], lmax)
        for k in ("tot", "syst", "stat"):
            _close(got[k][c].cpu().numpy(), ref[k])


def test_fused_residual_spectra_equal_three_pseudo_cl_calls(csx):
    """One pass (ring coefficients of s_hat - s_true and of r_sys, a_lm of the difference as the
    difference) against three separate spectra calls, 10 problems in groups of 5, nside 16."""
    nside, lmax = 16, 40
    pix = _masked(nside, 0.8, 7)
    rng = np.random.default_rng(8)
    s_hat = torch.from_numpy(rng.normal(size=(10, pix.size, 2, 3)).astype(np.float32)).cuda()
    s_true = torch.from_numpy(rng.normal(size=(pix.size, 2)).astype(np.float32)).cuda()
    r_sys = torch.from_numpy((0.2 * rng.normal(size=(10, pix.size, 2))).astype(np.float32)).cuda()
    plan = csx.ShtPlan(nside, lmax, pix)
    got = csx.residual_spectra(plan, s_hat, s_true, r_sys, nreal=5)
    cmb = s_hat[..., 0]
    ref = {"tot": csx.pseudo_cl(plan, cmb, sub_common=s_true, navg=5),
           "syst": csx.pseudo_cl(plan, r_sys, navg=5),
           "stat": csx.pseudo_cl(plan, cmb, sub_common=s_true, sub_each=r_sys, navg=5)}
    for k in ref:
        _close(got[k].cpu().numpy(), ref[k].cpu().numpy())
