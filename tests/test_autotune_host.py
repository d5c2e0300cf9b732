"""Host logic of the batched-curvature autotuner on CPU: the workload shape
classes, the JSON cache (atomic save, reload) and the cache-hit path, which
answers without launching anything; and every candidate shape is one that the
batched entry point accepts (4 warps per block, one or eight lanes per cell)."""
import json
import os

from paper_2006_12838_gb300 import autotune


class _Field(tuple):
    """Stands in for a (phi, idx, n_iface, kappa) tuple; only n_iface is read."""


def _fields(counts):
    return [_Field((None, None, k, None)) for k in counts]


def test_shape_class_rounds_up_to_powers_of_two():
    assert autotune.shape_class(_fields([5, 10, 17])) == "f4-k32"
    assert autotune.shape_class(_fields([1 << 20] * 64)) == "f64-k%d" % (1 << 26)
    assert autotune.shape_class(_fields([1 << 20] * 65)) == "f128-k%d" % (1 << 27)
    assert autotune.shape_class(_fields([0])) == "f1-k1"
    assert autotune.shape_class(_fields([])) == "f1-k1"
    # one more interface cell than a power of two moves to the next class
    assert autotune.shape_class(_fields([1024])) == "f1-k1024"
    assert autotune.shape_class(_fields([1025])) == "f1-k2048"


def test_cache_round_trip_is_atomic(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setenv("PLIC_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}                      # missing file: empty cache
    d = {"gpu|batched-v2|sz_opt|0|f4-k32": {"shape": [128, 64, 2, 1], "ms": 0.25}}
    autotune._save(d)
    assert json.loads(path.read_text()) == d
    assert autotune._load() == d
    assert sorted(os.listdir(path.parent)) == ["autotune.json"]   # no temporary left
    path.write_text("{not json")
    assert autotune._load() == {}                      # a damaged cache is ignored


def test_cache_hit_returns_the_stored_shape_without_timing(tmp_path, monkeypatch):
    monkeypatch.setenv("PLIC_AUTOTUNE_CACHE", str(tmp_path / "autotune.json"))
    fields = _fields([100, 200])
    monkeypatch.setattr(autotune, "key", lambda f, m, fl: "fake-gpu|%s|%d|%s" % (m, fl, autotune.shape_class(f)))
    k = autotune.key(fields, "sz_opt", 0)
    autotune._save({k: {"shape": [128, 256, 3, 8], "ms": 0.1}})

    def no_launch(*a, **kw):
        raise AssertionError("a cache hit must not launch")
    monkeypatch.setattr(autotune.plic, "curvature_batched", no_launch)
    shape, times = autotune.tune(fields, method="sz_opt", flags=0)
    assert shape == (128, 256, 3, 8) and times == {}


def test_candidates_are_accepted_shapes():
    assert len(set(autotune.CANDIDATES)) == len(autotune.CANDIDATES)
    for threads, chunk, bps, lanes in autotune.CANDIDATES:
        assert threads == 128            # the batched kernels are built for 4 warps per block
        assert chunk >= 1 and bps >= 0
        assert lanes in (1, 8)
    assert {c[3] for c in autotune.CANDIDATES} == {1, 8}
