"""The autotuner on the device: it measures every (n-bucket, d-class) cell and the dense bands,
installs a valid policy, and the tuned library still returns the oracle's answers."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import autotune, synth

pytestmark = pytest.mark.gpu


def test_tune_installs_a_valid_policy(tmp_path):
    from paper_1407_5609_gb300 import capi
    before = capi.cpp_get_tuning(capi.TUNE_BATCH_PATH)
    try:
        entry = autotune.load_or_tune(path=str(tmp_path / "tune.json"), target_pairs=5e7, reps=1)
        table = np.asarray(entry["batch_path"])
        assert table.shape == (4, 6) and set(table.reshape(-1)) <= {1, 2, 3}
        assert len(entry["batch_ms"]) == 24
        assert capi.cpp_get_tuning(capi.TUNE_BATCH_PATH) == list(table.reshape(-1))
        if capi.filters_available():
            assert entry["dense_band"] in autotune.BANDS and entry["dense_shape"] in autotune.SHAPES
            assert len(entry["dense_ms"]) == len(autotune.BANDS) * len(autotune.SHAPES)
            assert capi.cpp_get_tuning(capi.TUNE_DENSE_SHAPE) == [entry["dense_shape"]]
        again = autotune.load_or_tune(path=str(tmp_path / "tune.json"))  # served from the cache
        assert again["when"] == entry["when"]
        # the tuned default path gives the oracle's closest pairs
        g = synth.rng_for(81)
        xs = [g.random((n, d)).astype(np.float32) for n, d in [(300, 8), (1500, 64), (5000, 100), (700, 200)]]
        res, _, _ = capi.cpp_batch([to_dev(x, device()) for x in xs], [-1.0] * len(xs))
        for x, r in zip(xs, res):
            oi, oj, od2 = oracle.cpp(x.astype(np.float64))
            assert (r["i"], r["j"], r["dist2"]) == (oi, oj, od2)
    finally:
        capi.cpp_set_tuning(capi.TUNE_BATCH_PATH, before)
        capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [1])


@pytest.mark.parametrize("band", [1, 8, 64])
def test_dense_band_does_not_change_the_answer(band):
    from paper_1407_5609_gb300 import capi
    if not capi.filters_available():
        pytest.skip("no tensor-core filter in this build")
    before = capi.cpp_get_tuning(capi.TUNE_DENSE_BAND)
    x, _ = synth.make_cpp(n=3000, d=48, seed=82)
    try:
        capi.cpp_set_tuning(capi.TUNE_DENSE_BAND, [band])
        r = capi.cpp_closest_pair(to_dev(x, device()), mode="filter_bf16")
    finally:
        capi.cpp_set_tuning(capi.TUNE_DENSE_BAND, before if before[0] > 0 else [16])
    oi, oj, od2 = oracle.cpp(np.asarray(x, dtype=np.float64))
    assert (r["i"], r["j"], r["dist2"]) == (oi, oj, od2)
