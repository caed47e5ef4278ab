"""Host logic of the launch-shape autotuner: cache keys, the JSON file and
the choice between a cached tile and a fresh search (a fake context stands
in for the GPU)."""
import json

import pytest

from paper_2410_20441_gb300 import autotune


class FakeCtx:
    def __init__(self, shape=(40, 30, 20), prec="fp32", bc="kubc"):
        self.shape, self.prec, self.bc = shape, prec, bc
        self.tuned = 0
        self.tile = (0, 0, 0, 0)

    def autotune(self, sweeps, solves="auto"):
        self.tuned += 1
        self.solves = solves
        self.tile = (3, 16, 24, 2) if solves != "plain" else (3, 16, 48, 1)
        return self.tile, 0.5

    def set_tile(self, t):
        self.tile = tuple(t)


@pytest.fixture
def cache(tmp_path, monkeypatch):
    p = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("CE_TUNE_CACHE", str(p))
    monkeypatch.setattr(autotune, "_library_tag", lambda: "libX")
    monkeypatch.setattr(autotune, "gpu_tag", lambda: "GPU|sm152")
    return p


def test_key_separates_shape_precision_cases_bc_gpu_and_build():
    k = autotune.key((3, 4, 5), "fp32", 6, "kubc", gpu="G", lib="L")
    assert k == "3x4x5|fp32|6|kubc|G|L"
    others = [autotune.key((3, 4, 6), "fp32", 6, "kubc", gpu="G", lib="L"),
              autotune.key((3, 4, 5), "fp64", 6, "kubc", gpu="G", lib="L"),
              autotune.key((3, 4, 5), "fp32", 3, "kubc", gpu="G", lib="L"),
              autotune.key((3, 4, 5), "fp32", 6, "roller", gpu="G", lib="L"),
              autotune.key((3, 4, 5), "fp32", 6, "kubc", gpu="H", lib="L"),
              autotune.key((3, 4, 5), "fp32", 6, "kubc", gpu="G", lib="M")]
    assert len({k, *others}) == 7


def test_first_call_searches_and_caches_then_reuses(cache):
    c = FakeCtx()
    t, ms = autotune.tune_context(c)
    assert (t, ms, c.tuned) == ((3, 16, 24, 2), 0.5, 1)
    d = json.loads(cache.read_text())
    (k, e), = d.items()
    assert k.startswith("40x30x20|fp32|6|kubc|GPU|sm152|libX") and e["tile"] == [3, 16, 24, 2]
    c2 = FakeCtx()
    t2, ms2 = autotune.tune_context(c2)
    assert (t2, ms2, c2.tuned, c2.tile) == ((3, 16, 24, 2), None, 0, (3, 16, 24, 2))
    c3 = FakeCtx(shape=(41, 30, 20))
    autotune.tune_context(c3)
    assert c3.tuned == 1 and len(json.loads(cache.read_text())) == 2
    autotune.tune_context(c2, force=True)
    assert c2.tuned == 1


def test_unreadable_or_malformed_cache_is_ignored(cache):
    cache.parent.mkdir(parents=True)
    cache.write_text("{not json")
    assert autotune.load_cache() == {}
    c = FakeCtx()
    autotune.tune_context(c)
    assert c.tuned == 1 and json.loads(cache.read_text())
    cache.write_text(json.dumps({autotune.key(c.shape, "fp32", 6, "kubc"): {"tile": [1, 2, 3]}}))
    c2 = FakeCtx()
    autotune.tune_context(c2)
    assert c2.tuned == 1


def test_plain_tuning_has_its_own_entry(cache):
    """A tile tuned for the double-word sweep (batches, unrefined solves) is
    cached apart from the one tuned for the context's own solves."""
    c = FakeCtx()
    assert autotune.tune_context(c) == ((3, 16, 24, 2), 0.5) and c.solves == "auto"
    c2 = FakeCtx()
    assert autotune.tune_context(c2, solves="plain") == ((3, 16, 48, 1), 0.5) and c2.solves == "plain"
    d = json.loads(cache.read_text())
    assert len(d) == 2 and any(k.endswith("|plain") for k in d)
    c3 = FakeCtx()
    assert autotune.tune_context(c3, solves="plain") == ((3, 16, 48, 1), None) and c3.tuned == 0
