"""The autotuner's host logic on the CPU, with the library calls replaced by fakes: candidates are
grouped by (r,s), every (heavy threshold, dense buckets) pair is timed, the fastest is kept and set
on the context, and a stored choice round-trips through its JSON file and is applied as stored."""
import json

import numpy as np
import pytest

import paper_2111_10980_gb300 as nd
from paper_2111_10980_gb300 import autotune


class FakeLib:
    """Records nd_ctx_set_tuning calls; nd_batch_run 'takes' a time that depends on the current
    setting, so that one candidate per (r,s) is fastest."""

    def __init__(self, best):
        self.best = best  # (r, s) -> (heavy_work, dense)
        self.setting = {}
        self.calls = []
        self.clock = 0.0

    def set_tuning(self, ctx, r, s, heavy, flags):
        self.setting[(r, s)] = (heavy, bool(flags & nd.ND_DENSE_BUCKETS))
        self.calls.append((r, s, heavy, flags))

    def batch_run(self, ctx, items, outs=None):
        r, s = int(items[0][2]), int(items[0][3])
        cost = 1.0 if self.setting.get((r, s)) == self.best[(r, s)] else 2.0
        self.clock += cost
        n = len(items)
        return [None] * n, [3] * n, [0] * n, None

    def perf_counter(self):
        return self.clock


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib({(2, 3): (256, False), (2, 4): (64, True), (3, 4): (0, True)})
    monkeypatch.setattr(autotune, "nd_ctx_set_tuning", f.set_tuning)
    monkeypatch.setattr(autotune, "nd_batch_run", f.batch_run)
    monkeypatch.setattr(autotune, "device_key", lambda: "FakeGPU_sm103_152sms")
    monkeypatch.setattr(autotune.time, "perf_counter", f.perf_counter)
    return f


def _graphs(rs_list):
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    return [(rp, col, r, s) for r, s in rs_list]


def test_tune_picks_the_fastest_candidate_per_rs(fake):
    res = autotune.tune("ctx", _graphs([(2, 3), (3, 4), (2, 4), (2, 3)]), reps=2)
    assert res["device"] == "FakeGPU_sm103_152sms"
    assert set(res["rs"]) == {"2,3", "2,4", "3,4"}
    for key, (h, dense) in [("2,3", (256, False)), ("2,4", (64, True)), ("3,4", (0, True))]:
        c = res["rs"][key]
        assert (c["heavy_work"], c["dense_buckets"]) == (h, dense)
    assert res["rs"]["2,3"]["graphs"] == 2
    # every candidate was timed: (2,4) over its staged thresholds, the others over the general ones
    assert len(res["rs"]["2,4"]["tried"]) == 2 * len(autotune.HEAVY_CANDIDATES_STAGED)
    assert len(res["rs"]["3,4"]["tried"]) == 2 * len(autotune.HEAVY_CANDIDATES)
    # the context is left with the winners
    assert fake.setting == {(2, 3): (256, False), (2, 4): (64, True), (3, 4): (0, True)}


def test_save_load_apply_round_trip(fake, tmp_path, monkeypatch):
    monkeypatch.setenv("ND_TUNING_DIR", str(tmp_path))
    res = autotune.tune("ctx", _graphs([(2, 3), (3, 4)]), reps=1)
    path = autotune.save(res)
    assert path.startswith(str(tmp_path)) and path.endswith("tuning_FakeGPU_sm103_152sms.json")
    assert json.load(open(path)) == res
    loaded = autotune.load()
    assert loaded == res
    fake.calls.clear()
    assert autotune.apply("ctx", loaded) == 2
    got = {(r, s): (h, fl) for r, s, h, fl in fake.calls}
    assert got == {(2, 3): (256, 0), (3, 4): (0, nd.ND_DENSE_BUCKETS)}


def test_missing_file_and_empty_result(tmp_path):
    assert autotune.load(str(tmp_path / "none.json")) is None
    assert autotune.apply("ctx", None) == 0


def test_failed_request_stops_tuning(fake, monkeypatch):
    def failing(ctx, items, outs=None):
        n = len(items)
        return [None] * n, [3] * n, [nd.ND_EINVAL] + [0] * (n - 1), None

    monkeypatch.setattr(autotune, "nd_batch_run", failing)
    with pytest.raises(RuntimeError):
        autotune.tune("ctx", _graphs([(2, 3)]), reps=1)
