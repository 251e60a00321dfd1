"""Host side of the autotuner: the selection rules, the JSON cache and the library's tuning ABI
(no GPU needed: the tuning table is process-wide host state)."""
import numpy as np
import pytest

from paper_1407_5609_gb300 import autotune


@pytest.fixture
def capi(libpath):
    from paper_1407_5609_gb300 import capi
    before = {k: capi.cpp_get_tuning(k) for k in (capi.TUNE_BATCH_PATH, capi.TUNE_DENSE_BAND)}
    yield capi
    capi.cpp_set_tuning(capi.TUNE_BATCH_PATH, before[capi.TUNE_BATCH_PATH])
    if before[capi.TUNE_DENSE_BAND][0] > 0:
        capi.cpp_set_tuning(capi.TUNE_DENSE_BAND, before[capi.TUNE_DENSE_BAND])


def test_choose_batch_table_picks_the_faster_path():
    ms = {(0, 0): {1: 1.0, 2: 2.0, 3: 2.5}, (3, 1): {1: 5.0, 2: 4.0, 3: 4.5}, (2, 2): {1: 3.0, 2: 3.0, 3: 3.0},
          (1, 5): {1: 3.0, 2: 2.0, 3: 1.0}}
    t = autotune.choose_batch_table(ms)
    assert len(t) == 4 and all(len(r) == 6 for r in t)
    assert t[0][0] == 1 and t[3][1] == 2 and t[1][5] == 3
    assert t[2][2] == 3                                     # ties go to the higher path
    assert t[1][3] == 2                                     # unmeasured cells keep the default


def test_path_for_matches_the_library_buckets():
    table = [[10 * nb + dc for dc in range(6)] for nb in range(4)]
    assert autotune.path_for(table, 256, 8) == 0 and autotune.path_for(table, 256, 16) == 0
    assert autotune.path_for(table, 256, 17) == 1 and autotune.path_for(table, 1000, 32) == 1
    assert autotune.path_for(table, 1023, 64) == 2 and autotune.path_for(table, 1024, 65) == 13
    assert autotune.path_for(table, 4095, 128) == 13 and autotune.path_for(table, 4096, 129) == 24
    assert autotune.path_for(table, 16384, 256) == 35 and autotune.path_for(table, 10 ** 6, 192) == 34


def test_choose_band():
    assert autotune.choose_band({8: 3.0, 16: 2.0, 32: 2.5}) == 16
    assert autotune.choose_band({8: 2.0, 16: 2.0}) == 8


def test_choose_dense_shape_and_band():
    assert autotune.choose_dense({(1, 8): 3.0, (1, 16): 2.0, (2, 8): 1.5, (2, 16): 2.5}) == (2, 8)
    assert autotune.choose_dense({(1, 16): 2.0, (2, 8): 2.0}) == (1, 16)   # ties: the smaller shape


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(p) == {"version": autotune.CACHE_VERSION, "entries": {}}
    data = autotune.load_cache(p)
    data["entries"]["GPU|sm152|abc"] = {"batch_path": [[1, 2, 1, 2, 2, 2]] * 4, "dense_band": 32}
    autotune.save_cache(data, p)
    assert autotune.load_cache(p) == data
    (tmp_path / "bad.json").write_text("{not json")
    assert autotune.load_cache(str(tmp_path / "bad.json"))["entries"] == {}


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("CPPGB_TUNE_CACHE", str(tmp_path / "x.json"))
    assert autotune.cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("CPPGB_TUNE_CACHE")
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    assert autotune.cache_path() == str(tmp_path / "cppgb" / "tune.json")


def test_install_reaches_the_library(capi):
    table = [[1, 2, 1, 2, 3, 3], [2, 2, 2, 2, 3, 1], [1, 1, 1, 1, 1, 1], [2, 1, 2, 1, 3, 2]]
    autotune.install({"batch_path": table, "dense_band": 32, "dense_shape": 2})
    assert capi.cpp_get_tuning(capi.TUNE_BATCH_PATH) == list(np.asarray(table).reshape(-1))
    assert capi.cpp_get_tuning(capi.TUNE_DENSE_BAND) == [32]
    assert capi.cpp_get_tuning(capi.TUNE_DENSE_SHAPE) == [2]
    autotune.install({"dense_shape": 1})
    assert capi.cpp_get_tuning(capi.TUNE_DENSE_SHAPE) == [1]


def test_tuning_argument_errors(capi):
    for kind, vals in [(capi.TUNE_BATCH_PATH, [2] * 23), (capi.TUNE_BATCH_PATH, [2] * 23 + [4]),
                       (capi.TUNE_BATCH_PATH, [0] + [2] * 23),
                       (capi.TUNE_DENSE_BAND, [0]), (capi.TUNE_DENSE_BAND, [5000]), (capi.TUNE_DENSE_SHAPE, [0]),
                       (capi.TUNE_DENSE_SHAPE, [3]), (7, [1])]:
        with pytest.raises(capi.CppgbError) as e:
            capi.cpp_set_tuning(kind, vals)
        assert e.value.status == capi.ERR_ARG
