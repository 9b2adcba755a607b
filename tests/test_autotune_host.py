"""Host-side logic of the uneven-batch autotuner (Sec. 8's fusion study
tunes the fused launch): the cache key separates every GPU model, SM count
and batch shape, and the cache file round-trips a choice."""
import pytest

pytest.importorskip("torch")


def test_cache_key_names_gpu_sms_and_batch_shape():
    from paper_2606_15437_gb300 import engine as E
    base = E.tune_cache_key("NVIDIA GB300", 152, 64, [5, 3, 4, 3])
    assert base == E.tune_cache_key("NVIDIA GB300", 152, 64, (3, 4, 5))     # a set of n_max values
    assert "NVIDIA GB300" in base and "|152|" in base
    others = [E.tune_cache_key("NVIDIA B200", 152, 64, [3, 4, 5]),        # another GPU model
              E.tune_cache_key("NVIDIA GB300", 148, 64, [3, 4, 5]),       # fewer SMs (another part)
              E.tune_cache_key("NVIDIA GB300", 152, 256, [3, 4, 5]),      # other sampled valuations
              E.tune_cache_key("NVIDIA GB300", 152, 64, [3, 4])]          # other layers
    assert len({base, *others}) == 5


def test_cache_file_round_trip(tmp_path):
    from paper_2606_15437_gb300 import engine as E
    p = str(tmp_path / "autotune.json")
    assert E._load_cache(p) == {}
    k = E.tune_cache_key("G", 1, 64, [3])
    E._store_cache(p, {k: {"units": 4, "block": 128, "tiles": [8, 8, 4, 4]}})
    assert E._load_cache(p)[k]["tiles"] == [8, 8, 4, 4]


def test_grid_is_the_documented_one():
    from paper_2606_15437_gb300 import engine as E
    assert E.TUNE_UNITS == (4, 8) and E.TUNE_BLOCKS == (128, 256)
    assert E.TUNE_TILES == (4, 8, 16, 32, 64)
