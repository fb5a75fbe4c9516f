"""The bench's JSON line (host logic only, no GPU): every key of the measurement contract is
present and the derived figures follow from the timings they are computed from."""
import argparse

import pytest

import bench

STAGES = ["grid", "links", "chains", "follow", "select", "merge", "refit", "pack", "refit_grad", "reduce"]


def fake_result():
    ms = dict(zip(STAGES, [0.3, 2.1, 0.9, 2.8, 1.6, 1.4, 0.6, 0.4, 2.2, 0.2]))
    n_calls = 5
    return {
        "ms_step": 11.6, "ms_single": 12.6, "n_clusters": 33_000_000, "n_clusters_all": 33_000_000,
        "n_tracks": 218_000, "n_hits": 26_000_000, "weighted_hits": 25_000_000, "n_chains": 790_000,
        "cand_hits": 68_000_000, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5},
        "tuning": {"key": "k", "source": "cache"}, "prof": ({k: v * n_calls for k, v in ms.items()}, n_calls),
        "ms_plain": 114.0, "ms_grad_event": 1.2, "ms_grad_event_stored": 1.0, "ms_grad_copies": 2.0, "ms_grad_copies_stored": 1.8, "n_tracks_c5": 25_779, "calib": {}, "single": {},
        "frame": {"value": 1.5e9}, "h2d": 134_324_888, "d2h": 365_388_892, "ms_e2e": 12.7, "ms_e2e_seq": 15.4,
    }


def test_bench_line_has_every_contract_key_and_consistent_figures():
    args = argparse.Namespace(steps=40, warmup=3, events=64)
    res = fake_result()
    line = bench.finish_native(args, res, 1)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "single_stream",
              "time_frame"):
        assert k in line, k
    assert line["value"] == pytest.approx(33e6 / 11.6e-3)
    assert line["ms_per_step"] == 11.6 and line["steps"] == 40 and line["warmup"] == 3
    assert line["single_stream"]["value"] == pytest.approx(33e6 / 12.6e-3)
    assert line["config"]["workload"] and "l2" in line["config"]
    r = line["roofline"]
    assert r["kernel"] == "follow" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["achieved"] == pytest.approx(bench.stage_bytes(res)["follow"] / 2.8e-3 / 1e9)
    assert "traffic" in r
    e = line["e2e"]
    assert e["value"] == pytest.approx(33e6 / 12.7e-3) and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    a = line["adjoint"]
    assert a["value"] == pytest.approx(1200.0) and a["stored_states"]["value"] == pytest.approx(1000.0)
    assert a["batched"]["events"] == bench.CENTRAL_COPIES
    assert a["batched"]["value"] == pytest.approx(2000.0 / bench.CENTRAL_COPIES)
    assert a["batched"]["stored_states"] == pytest.approx(1800.0 / bench.CENTRAL_COPIES)
    # no tuned shapes: the library default adjoint (states recomputed from checkpoints)
    assert line["adjoint_form_in_step"] == "checkpoints"
    assert line["gpu_launches"] == (bench.LAUNCHES_TRACKING + bench.LAUNCHES_REFIT_GRAD["checkpoints"]) * 40
    assert line["stage_tflops"]["refit_grad"] == pytest.approx(
        (2 * bench.FLOP_FWD + bench.FLOP_ADJ) * 25e6 / 2.2e-3 / 1e12)
    # with the stored-state form tuned in: fewer flop per hit, four more launches
    res2 = fake_result()
    res2["tuning"] = {"key": "k", "source": "cache", "best": {"refit_grad": [64, 8, 1]}}
    line2 = bench.finish_native(args, res2, 1)
    assert line2["gpu_launches"] == (bench.LAUNCHES_TRACKING + bench.LAUNCHES_REFIT_GRAD["stored states"]) * 40
    assert line2["stage_tflops"]["refit_grad"] == pytest.approx((bench.FLOP_FWD + bench.FLOP_ADJ) * 25e6 / 2.2e-3 / 1e12)


def test_alu_roofline_when_the_gradient_stage_dominates():
    args = argparse.Namespace(steps=10, warmup=3, events=64)
    res = fake_result()
    ms, n = res["prof"]
    ms = dict(ms)
    ms["refit_grad"] = 5.0 * n
    res["prof"] = (ms, n)
    r = bench.finish_native(args, res, 1)["roofline"]
    assert r["bound"] == "alu" and r["kernel"] == "refit_grad" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS)
    # a measured FMA peak replaces the derived one
    res["fp32_peak"] = {"tflops": 70.0, "config": "c", "clocks": None}
    r = bench.finish_native(args, res, 1)["roofline"]
    assert r["peak"] == 70.0 and r["frac"] == pytest.approx(r["achieved"] / 70.0) and "measured" in r["peak_kind"]
