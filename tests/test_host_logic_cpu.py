"""Host logic around the C ABI that needs no GPU: the tuning structure and cache of the autotuner
and the storage of calibrations."""
import json

import numpy as np
import pytest

from paper_1712_09434_gb300 import capi, synth


def test_tuning_struct_and_cache_round_trip(tmp_path):
    tune = pytest.importorskip("paper_1712_09434_gb300.tune")
    shapes = {"links": (64, 6, 0), "follow": (96, 12, 2), "refit_grad": (128, 4, 0)}
    t = tune.to_struct(shapes)
    assert isinstance(t, capi.tpc_tuning)
    for k, name in enumerate(tune.KERNELS):
        b, c, h = shapes.get(name, (0, 0, 0))
        assert (t.block[k], t.ctas_per_sm[k], t.chunk[k]) == (b, c, h)
    path = str(tmp_path / "cache.json")
    tune.store("gpuA|sm152|ev64|cl2^19", {"best": {k: list(v) for k, v in shapes.items()}}, path=path)
    tune.store("gpuB|sm132|ev1|cl2^20", {"best": {}}, path=path)
    got = tune.load("gpuA|sm152|ev64|cl2^19", path=path)
    assert got["best"]["follow"] == [96, 12, 2]
    assert tune.load("missing", path=path) is None
    assert sorted(json.load(open(path))) == ["gpuA|sm152|ev64|cl2^19", "gpuB|sm132|ev1|cl2^20"]


def test_candidates_respect_the_kernels_block_limits():
    tune = pytest.importorskip("paper_1712_09434_gb300.tune")
    limits = {"grid": 256, "links": 128, "chains": 256, "follow": 128, "select": 1024, "merge": 512,
              "refit": 128, "refit_grad": 128}       # tpc_tuning bounds declared in include/tpc.h
    for name, cand in tune.CANDIDATES.items():
        for b in cand["block"]:
            assert b % 32 == 0 and 0 < b <= limits[name], (name, b)
        assert all(0 <= c <= 64 for c in cand["ctas"])
        assert all(0 <= h <= 64 for h in cand["chunk"])


def test_calibration_save_load_round_trip(tmp_path):
    from paper_1712_09434_gb300 import calib
    th = synth.calib_theta(1005)
    path = str(tmp_path / "theta.json")
    calib.save_theta(path, th, meta={"event": "calibration", "steps": 20})
    back = calib.load_theta(path)
    np.testing.assert_array_equal(back, th)
    doc = json.load(open(path))
    assert doc["s_vd"] == th[0] and len(doc["d"]) == 36 and len(doc["a"]) == 36
