"""The JSON cache of tuning choices (host logic, no GPU): a miss tunes and stores, a hit
applies the stored choice (and the multi handle's tile costs) without timing, keys separate GPU, process, precision, k and
batch composition, and an unreadable file counts as empty."""
import json

from paper_2510_05100_b300 import tune_cache


class FakeProcess:
    def __init__(self, name="gg_ttxg", precision=1, best=4, nvar=9):
        self.name, self.precision, self.variant = name, precision, 0
        self.best, self.nvar, self.tuned = best, nvar, 0

    def autotune(self, momenta, w_in, points, w_out, stream=None):
        self.tuned += 1
        self.variant = self.best
        return [10.0 - (v == self.best) for v in range(self.nvar)]


class FakeBatch:
    def __init__(self, n):
        self.shape = (n, 5, 4)


class FakeMulti:
    def __init__(self, precision=1, best=2):
        self.precision, self.slot_groups, self.best, self.tuned = precision, 1, best, 0
        self.costs = {}

    def autotune(self, batches, points, stream=None):
        self.tuned += 1
        self.slot_groups = self.best
        for i, b in enumerate(batches):
            self.costs[b[0].name] = 10.0 * (i + 1) + self.best
        return [3.0, 2.0, 2.5]

    def tile_cost(self, proc):
        return self.costs.get(proc.name, 0.0)

    def set_tile_cost(self, proc, us):
        self.costs[proc.name] = us


def test_miss_tunes_and_stores_then_hit_applies_without_timing(tmp_path):
    path = str(tmp_path / "tune.json")
    pts = [{}] * 16
    p = FakeProcess(best=4)
    e = tune_cache.autotune_process(p, None, None, pts, None, path, gpu="B300")
    assert (e["choice"], e["cached"], p.tuned, p.variant) == (4, False, 1, 4)
    stored = json.load(open(path))
    assert stored[tune_cache.variant_key("B300", "gg_ttxg", 1, 16)]["choice"] == 4
    q = FakeProcess(best=7)                 # a new handle: the stored choice wins, no timing
    e = tune_cache.autotune_process(q, None, None, pts, None, path, gpu="B300")
    assert (e["choice"], e["cached"], q.tuned, q.variant) == (4, True, 0, 4)


def test_keys_separate_gpu_process_precision_and_points(tmp_path):
    path = str(tmp_path / "tune.json")
    base = dict(gpu="B300")
    tune_cache.autotune_process(FakeProcess(best=4), None, None, [{}] * 16, None, path, **base)
    for proc, pts, gpu in ((FakeProcess(best=2), [{}] * 8, "B300"),
                           (FakeProcess(name="gg_ttx", best=3), [{}] * 16, "B300"),
                           (FakeProcess(precision=0, best=1), [{}] * 16, "B300"),
                           (FakeProcess(best=5), [{}] * 16, "other GPU")):
        e = tune_cache.autotune_process(proc, None, None, pts, None, path, gpu=gpu)
        assert not e["cached"] and proc.tuned == 1
    assert len(json.load(open(path))) == 5


def test_slot_groups_keyed_by_batch_composition(tmp_path):
    path = str(tmp_path / "tune.json")
    batches = [(FakeProcess("gg_ttx"), FakeBatch(8000), None, None), (FakeProcess("qq_ttx"), FakeBatch(3000), None, None)]
    m = FakeMulti(best=2)
    assert tune_cache.autotune_multi(m, batches, [{}] * 64, path, gpu="B300")["choice"] == 2
    assert m.costs == {"gg_ttx": 12.0, "qq_ttx": 22.0}
    m2 = FakeMulti(best=6)
    e = tune_cache.autotune_multi(m2, batches, [{}] * 64, path, gpu="B300")
    assert e["cached"] and m2.slot_groups == 2 and m2.tuned == 0
    assert m2.costs == {"gg_ttx": 12.0, "qq_ttx": 22.0}     # the stored tile costs, restored
    other = [(FakeProcess("gg_ttx"), FakeBatch(8001), None, None)] + batches[1:]
    m3 = FakeMulti(best=3)
    assert not tune_cache.autotune_multi(m3, other, [{}] * 64, path, gpu="B300")["cached"]


def test_unreadable_file_counts_as_empty(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    p = FakeProcess(best=4)
    e = tune_cache.autotune_process(p, None, None, [{}] * 16, None, str(path), gpu="B300")
    assert not e["cached"] and p.variant == 4
    assert json.load(open(path))[tune_cache.variant_key("B300", "gg_ttxg", 1, 16)]["choice"] == 4
