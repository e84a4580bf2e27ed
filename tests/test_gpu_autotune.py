"""The fit autotuner on the device: it times every valid launch configuration on a small scan,
returns one of them, the fit converges with it, and a second call is served from the cache."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests._inputs import pack, scan_case  # noqa: E402


def test_autotune_small_scan(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08463_b300 import autotune, csx
    case = scan_case(nside=16, nconf=6, kmax=30, nreal=2)
    wl = case.wl
    model, sky, labels = case.gpu()
    beta0 = torch.tensor(pack(wl, [wl.beta0(c) for c in range(wl.nconf) for _ in range(wl.nreal)]),
                         device="cuda")
    cache = str(tmp_path / "tune.json")
    opts, entry = autotune.tune_fit(csx, model, sky, labels, wl.K, beta0, sample=4, cache=cache)
    assert (opts["path"], opts["threads"]) in autotune.candidates(sky.noise)
    assert set(entry["ms"]) == {"%s/%d" % c for c in autotune.candidates(sky.noise)}
    assert all(v > 0 for v in entry["ms"].values())
    res = csx.fit_batch(model, sky, labels, wl.K, beta0, **opts)
    torch.cuda.synchronize()
    assert np.all(res["status"].cpu().numpy() == 0)
    again, entry2 = autotune.tune_fit(csx, model, sky, labels, wl.K, beta0, sample=4, cache=cache)
    assert again == opts and entry2 == entry
