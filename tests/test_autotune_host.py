"""The autotuner's search and cache (no GPU: a deterministic cost stands in for timing)."""
import json

from paper_2112_10223_gb300 import autotune

DEV = {"device": "GB300-test", "sms": 152, "cuda": "13.0", "library": 100}
WORK = autotune.workload_key([4, 32], [1024, 4096], [10000, 50000], ["torch.float64"])


def fake_cost(values):
    # minimum at warp_max 256, cta_max 2048, window_max 2048, accumulator 2
    return (abs(values["warp_max"] - 256) / 64 + abs(values["cta_max"] - 2048) / 512
            + (values["window_max"] != 2048) * 1.5 + (values["block_accumulator"] != 2) * 0.7 + 1.0)


def test_coordinate_sweep_finds_the_minimum_and_caches_it(tmp_path):
    calls = []

    def timer(run, values):
        calls.append(values)
        return fake_cost(values)

    path = str(tmp_path / "tune.json")
    t = autotune.Autotuner(cache_path=path)
    best = t.tune(lambda v: None, DEV, WORK, timer=timer)
    assert best == {"warp_max": 256, "cta_max": 2048, "window_max": 2048, "block_accumulator": 2}
    assert not t.last["cached"] and t.last["timed"] == len(calls)
    assert all(autotune.valid(c) for c in calls)
    assert len(calls) <= sum(len(v) for v in autotune.SPACE.values())  # one sweep, each point timed once
    # a fresh tuner on the same file answers from the cache without timing
    calls.clear()
    t2 = autotune.Autotuner(cache_path=path)
    assert t2.tune(lambda v: None, DEV, WORK, timer=timer) == best
    assert calls == [] and t2.last["cached"]
    # the record is plain JSON keyed by device and workload
    with open(path) as f:
        d = json.load(f)
    (key,) = d.keys()
    assert json.loads(key) == {"dev": DEV, "work": WORK}


def test_another_device_or_workload_tunes_again(tmp_path):
    n = {"calls": 0}

    def timer(run, values):
        n["calls"] += 1
        return fake_cost(values)

    t = autotune.Autotuner(cache_path=str(tmp_path / "c.json"))
    t.tune(lambda v: None, DEV, WORK, timer=timer)
    first = n["calls"]
    t.tune(lambda v: None, dict(DEV, sms=148), WORK, timer=timer)
    assert n["calls"] == 2 * first
    other = autotune.workload_key([200, 256], [1024, 65536], [10 ** 8, 10 ** 9], ["torch.float32"])
    t.tune(lambda v: None, DEV, other, timer=timer)
    assert n["calls"] == 3 * first
    assert t.tune(lambda v: None, DEV, WORK, timer=timer, force=True) is not None and n["calls"] == 4 * first


def test_candidates_respect_the_option_ranges():
    assert autotune.valid({"warp_max": 512, "cta_max": 4096})
    assert not autotune.valid({"warp_max": 512, "cta_max": 256})
    for knob, values in autotune.SPACE.items():
        assert autotune.DEFAULTS[knob] in values


def test_gains_within_the_margin_keep_the_defaults(tmp_path):
    """A candidate 1 % faster than the defaults is noise under a 3 % margin; 10 % faster is taken."""
    def timer_small(run, values):
        return 0.99 if values["block_accumulator"] == 2 else 1.0

    t = autotune.Autotuner(cache_path=str(tmp_path / "m.json"))
    assert t.tune(lambda v: None, DEV, WORK, timer=timer_small) == autotune.DEFAULTS

    def timer_big(run, values):
        return 0.9 if values["block_accumulator"] == 2 else 1.0

    assert t.tune(lambda v: None, DEV, WORK, timer=timer_big, force=True) == dict(autotune.DEFAULTS,
                                                                                 block_accumulator=2)
