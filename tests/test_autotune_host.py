"""Autotuner host logic with fake handles (no GPU).

The fastest candidate wins; a candidate whose handle cannot be made or
whose probe fails is skipped and its handle closed; a search in which no
candidate ran raises instead of caching nothing; choices round-trip through
the cache file without probing again.
"""
import pytest

from paper_1704_05132_gb300 import autotune, gen


class FakeBatch:
    rates = {}      # (lanes, threads[, runs per CTA]) -> moves per ms; "ctor" / None: fails
    made = []

    def __init__(self, insts, lanes=0, threads=0, cluster=0, runs_per_cta=0):
        self.key = (lanes, threads, runs_per_cta)
        if self.key not in FakeBatch.rates and runs_per_cta == 1:
            self.key = (lanes, threads)
        if FakeBatch.rates.get(self.key) == "ctor":
            raise RuntimeError("refused at create")
        self.closed = False
        self.iters = 0
        FakeBatch.made.append(self)

    def run(self, seeds, iters, kmax, mode):
        if FakeBatch.rates.get(self.key) is None:
            raise RuntimeError("launch failed")
        self.iters = iters

    def results(self):
        return [{"moves_evaluated": FakeBatch.rates[self.key] * self.iters}]

    def close(self):
        self.closed = True


class FakeSolver:
    rates = {}      # (lanes, cluster) -> moves per ms; None: fails
    made = []

    def __init__(self, inst, lanes=0, cluster=0, speculation=0):
        self.key = (lanes, cluster)
        self.closed = False
        self.iters = 0
        FakeSolver.made.append(self)

    def vns(self, seed, iters, kmax, mode, **kw):
        if FakeSolver.rates.get(self.key) is None:
            raise RuntimeError("run refused")

    def vns_run(self, seed, iters, kmax, mode):
        self.iters = iters

    def result(self, **kw):
        return {"moves_evaluated": FakeSolver.rates[self.key] * self.iters}

    def close(self):
        self.closed = True


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(autotune, "Batch", FakeBatch)
    monkeypatch.setattr(autotune, "Solver", FakeSolver)
    monkeypatch.setattr(autotune, "_timed", lambda fn: (1.0, fn()))
    monkeypatch.setattr(autotune, "_cache", {})
    FakeBatch.rates, FakeBatch.made = {}, []
    FakeSolver.rates, FakeSolver.made = {}, []
    return [gen.plain_small(), gen.make_instance(3, 1, K=9, T=20)]


def test_batch_fastest_wins_and_failures_are_skipped(fakes):
    FakeBatch.rates = {(0, 512): 5.0, (0, 1024): "ctor", (8, 512): None, (16, 1024): 9.0,
                       (32, 512): 7.0}
    shape = autotune.tune_batch(fakes, probe_iters=4)
    assert shape == dict(lanes=16, threads=1024, cluster=1, runs_per_cta=1)
    FakeBatch.rates[(16, 1024, 2)] = 9.5                # two runs per CTA, faster still
    autotune._cache.clear()
    assert autotune.tune_batch(fakes, probe_iters=4)["runs_per_cta"] == 2
    assert FakeBatch.made and all(b.closed for b in FakeBatch.made)


def test_batch_nothing_ran_raises_and_caches_nothing(fakes):
    FakeBatch.rates = {(l, t): None for l in (0, 8, 16, 32) for t in (512, 1024)}
    FakeBatch.rates.update({(l, t, p): None for l in (0, 8, 16) for t in (512, 1024)
                            for p in (2, 4)})
    with pytest.raises(RuntimeError, match="no candidate") as ei:
        autotune.tune_batch(fakes)
    assert isinstance(ei.value.__cause__, RuntimeError)     # the last failure
    assert autotune._cache == {}
    assert all(b.closed for b in FakeBatch.made)


def test_batch_choice_cached_in_file(fakes, tmp_path, monkeypatch):
    cache = str(tmp_path / "tune.json")
    FakeBatch.rates = {(8, 1024): 3.0, (0, 512): 1.0}
    first = autotune.tune_batch(fakes, cache_file=cache)
    assert first == dict(lanes=8, threads=1024, cluster=1, runs_per_cta=1)
    monkeypatch.setattr(autotune, "_cache", {})     # a new process
    FakeBatch.rates, FakeBatch.made = {}, []        # any probe would now fail
    assert autotune.tune_batch(fakes, cache_file=cache) == first
    assert FakeBatch.made == []


def test_single_fastest_wins_and_nothing_ran_raises(fakes):
    inst = fakes[1]
    FakeSolver.rates = {(32, 8): 2.0, (64, 8): 6.0, (64, 16): 4.0}
    shape = autotune.tune_single(inst, probe_iters=10)
    assert shape == dict(lanes=64, cluster=8, teams=0)
    assert all(s.closed for s in FakeSolver.made)
    FakeSolver.rates, FakeSolver.made = {}, []
    with pytest.raises(RuntimeError, match="no candidate"):
        autotune.tune_single(gen.make_instance(4, 2, K=300, T=52))
    assert all(s.closed for s in FakeSolver.made)


def test_batch_lookup_takes_the_cached_shape_without_probing(fakes, tmp_path, monkeypatch):
    """lookup_batch (what a Batch created with every knob at 0 consults)
    returns the cached choice, from memory or from the file named by
    ELSR_AUTOTUNE_CACHE, and None when nothing is cached."""
    assert autotune.lookup_batch(fakes) is None
    cache = str(tmp_path / "tune.json")
    monkeypatch.setenv("ELSR_AUTOTUNE_CACHE", cache)
    FakeBatch.rates = {(16, 512, 2): 4.0}
    chosen = autotune.tune_batch(fakes)
    monkeypatch.setattr(autotune, "_cache", {})     # a new process, same file
    FakeBatch.made = []
    assert autotune.lookup_batch(fakes) == chosen == dict(lanes=16, threads=512, cluster=1,
                                                          runs_per_cta=2)
    assert FakeBatch.made == []
