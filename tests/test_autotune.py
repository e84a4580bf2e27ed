"""Host logic of the fit autotuner: shape buckets, candidate sets, sampling and the JSON cache."""
import numpy as np

from paper_2604_08463_b300 import autotune as at


def test_shape_key_buckets():
    K = np.array([[10, 2, 3], [100, 20, 30]])
    k1 = at.shape_key("separable", 32512, 10, K)
    assert k1 == at.shape_key("separable", 32000, 10, K + 1)  # same powers of two
    assert k1 != at.shape_key("separable", 32512, 10, K * 4)
    assert k1 != at.shape_key("homogeneous", 32512, 10, K)
    assert k1 != at.shape_key("separable", 32512, 10, K, solver="adatopk")


def test_candidates_follow_noise_solver_and_gradient():
    assert at.candidates("perpixel") == [("stream", 256)]
    assert at.candidates("separable", grad_mode="fd") == [("stream", 256)]
    assert ("moment", 64) not in at.candidates("separable", solver="adatopk")
    assert set(at.candidates("homogeneous")) == set(at.CANDIDATES)


def test_sample_configurations():
    assert at.sample_configurations(5, 32) == [0, 1, 2, 3, 4]
    s = at.sample_configurations(1000, 32)
    assert len(s) == 32 and s[0] == 0 and s[-1] == 999 and s == sorted(set(s))


def test_choose_times_once_then_reads_the_cache(tmp_path):
    cache = str(tmp_path / "tune.json")
    calls = []

    def timer(path, nt):
        calls.append((path, nt))
        return {"moment/128": 3.0, "moment/64": 2.0, "moment/256": 5.0, "stream/256": 9.0}["%s/%d" % (path, nt)]

    opts, entry = at.choose("k", at.candidates("separable"), timer, cache)
    assert opts == {"path": "moment", "threads": 64} and len(calls) == 4
    assert entry["ms"]["stream/256"] == 9.0
    opts2, _ = at.choose("k", at.candidates("separable"), timer, cache)
    assert opts2 == opts and len(calls) == 4  # served from the file
    opts3, e3 = at.choose("p", at.candidates("perpixel"), timer, cache)
    assert opts3 == {"path": "stream", "threads": 256} and e3["ms"] == {} and len(calls) == 4


def test_first_candidate_kept_within_the_margin():
    t = {"moment/128": 100.0, "moment/64": 98.0, "moment/256": 150.0, "stream/256": 300.0}
    opts, _ = at.choose("m", at.candidates("separable"), lambda p, n: t["%s/%d" % (p, n)])
    assert opts == {"path": "moment", "threads": 128}  # 2% faster is within the noise margin
    t["moment/64"] = 90.0
    opts, _ = at.choose("m", at.candidates("separable"), lambda p, n: t["%s/%d" % (p, n)])
    assert opts == {"path": "moment", "threads": 64}
