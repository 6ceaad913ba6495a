"""Host logic of the autotuner (paper_2104_00537_gb300/autotune.py) on CPU,
with a fake engine whose step time is a known function of the launch choices:
the search takes the fastest (cell size, pair loop), then the fastest block
size of its list walk, restores the cases' cell size, and caches the result
per (GPU, case-count bucket, particle-count bucket)."""
import json

from paper_2104_00537_gb300 import autotune


class FakeCase:
    def __init__(self, n):
        self.n = n
        self.params = {"cell_mode": 0}


def cost(cm, var, block):
    base = {(1, 5): 10.0, (1, 4): 12.0, (2, 5): 11.0}.get((cm, var), 20.0 + cm + var)
    return base * {0: 1.0, 128: 1.0, 256: 0.9, 512: 0.95}[block]


class FakeEngine:
    made = []

    def __init__(self, cases):
        self.cm = cases[0].params["cell_mode"]
        self.var, self.block, self.ms = 0, 0, 0.0
        FakeEngine.made.append((self.cm,))

    def set_options(self, pi_variant=-1, pi_block=0, timing=0, **kw):
        self.var, self.block = pi_variant, pi_block

    def step(self, n):
        self.ms += n * cost(self.cm, self.var, self.block)

    def timing(self, reset=False):
        t = {"step_ms": self.ms}
        if reset:
            self.ms = 0.0
        return t

    def destroy(self):
        pass


def test_tune_picks_fastest_configuration_and_block(tmp_path, monkeypatch):
    monkeypatch.setenv("SPH_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    cases = [FakeCase(5000), FakeCase(70000)]
    best, times = autotune.tune(cases, FakeEngine, "GB300")
    assert best == (1, 5, 256)
    assert times["1,5,128"] == 10.0 and abs(times["1,5,256"] - 9.0) < 1e-12
    assert all(c.params["cell_mode"] == 0 for c in cases)  # restored
    cached = json.load(open(tmp_path / "cache.json"))
    key = autotune.bucket_key("GB300", cases)
    assert cached[key]["best"] == [1, 5, 256]
    # a second call is served from the cache without building an engine
    FakeEngine.made.clear()
    best2, _ = autotune.tune(cases, FakeEngine, "GB300")
    assert best2 == (1, 5, 256) and FakeEngine.made == []


def test_tune_without_list_skips_block_search(tmp_path, monkeypatch):
    monkeypatch.setenv("SPH_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    cases = [FakeCase(1000)]
    best, times = autotune.tune(cases, FakeEngine, "GB300", candidates=[(1, 0), (2, 0)],
                                use_cache=False)
    assert best == (1, 0, 128)
    assert set(times) == {"1,0,128", "2,0,128"}


class FailingEngine(FakeEngine):
    def __init__(self, cases):
        if cases[0].params["cell_mode"] == 2:
            raise RuntimeError("list overflow")
        super().__init__(cases)


def test_configuration_that_cannot_run_is_skipped(tmp_path, monkeypatch):
    monkeypatch.setenv("SPH_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    best, times = autotune.tune([FakeCase(1000)], FailingEngine, "GB300",
                                candidates=[(2, 5), (1, 4)], use_cache=False)
    assert times["2,5,128"] == float("inf")
    assert best[:2] == (1, 4)
