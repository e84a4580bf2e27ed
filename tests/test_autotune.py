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


def test_stream_schedule_choice_and_cache(tmp_path):
    from paper_2604_08463_b300 import csx
    cache = str(tmp_path / "tune.json")
    key = at.stream_key("separable", 49152, 100, 150, True)
    assert key != at.stream_key("separable", 49152, 100, 150, False)
    assert key == at.stream_key("separable", 50000, 100, 160, True)
    t = {"128/2": 10.0, "64/2": 9.8, "64/3": 12.0, "128/3": 9.0, "128/4": 9.5, "256/2": 11.0}
    calls = []

    def timer(tile, stages):
        calls.append((tile, stages))
        return t["%d/%d" % (tile, stages)]

    sched, e = at.choose_schedule(key, list(csx.STREAM_SCHEDULES), timer, cache)
    assert sched == (128, 3) and len(calls) == 6 and e["ms"]["256/2"] == 11.0
    sched2, _ = at.choose_schedule(key, list(csx.STREAM_SCHEDULES), timer, cache)
    assert sched2 == (128, 3) and len(calls) == 6
    t["128/3"], t["128/4"] = 9.9, 9.75  # all within the 3% margin of the default
    sched3, _ = at.choose_schedule("other", list(csx.STREAM_SCHEDULES), timer, None)
    assert sched3 == (128, 2)


def test_stream_schedule_setter_is_host_only():
    from paper_2604_08463_b300 import build, csx
    build.build()
    assert csx.stream_schedule() == (128, 2)
    assert csx.stream_schedule(256, 2) == (256, 2)
    assert csx.stream_schedule() == (256, 2)
    assert csx.stream_schedule(0, 0) == (128, 2)
    import pytest
    with pytest.raises(csx.CsxError):
        csx.stream_schedule(96, 2)
    assert csx.stream_schedule() == (128, 2)
