"""The full 64-event batch of the bench (33 M clusters, multiplicities log-uniform in [100, 20000]
tracks), tracked in the bench's launch configuration (CUDA graph, autotuned launch shapes from
the cache): properties that hold at any size on the whole batch, and bit-exact tracks, FP32 refit
parameters and per-track chi2 against the FP64 oracle on sampled events (the largest, a median
and a small one)."""
import numpy as np
import pytest
import torch

import bench
from oracle import oracle as O
from paper_1712_09434_gb300 import capi, synth, tune
from tests import _gpu

pytestmark = pytest.mark.gpu

N_MIN = 10


@pytest.fixture(scope="module")
def batch():
    d = bench.make_batch(64, 2000)
    n = int(d["pad"].shape[0])
    ctx = _gpu.make_context(n, 64)
    cached = tune.load(tune.workload_key(64, n))
    if cached:
        ctx.tpc_set_tuning(tune.to_struct({k: tuple(v) for k, v in cached["best"].items()}))
    cl = capi.Clusters.from_numpy(d["pad"], d["tim"], d["bin_off"], 64)
    g = _gpu.run(ctx, cl, n_events=64, batch=True)
    yield d, ctx, cl, g
    ctx.close()


def test_whole_batch_properties(batch):
    d, ctx, cl, g = batch
    n = int(d["pad"].shape[0])
    off, hits, lab, evo = g["trk_off"], g["trk_hits"], g["label"], g["ev_trk_off"]
    nt = g["n_tracks"]
    assert nt > 150000
    assert np.all(np.diff(off) >= N_MIN)
    # partition: a cluster is in at most one track, and its label names that track
    assert len(np.unique(hits)) == len(hits)
    owner = np.repeat(np.arange(nt), np.diff(off))
    np.testing.assert_array_equal(lab[hits], owner)
    assert (lab >= 0).sum() == len(hits)
    # every track's hits lie in its event's cluster range, events in order
    assert evo[0] == 0 and evo[-1] == nt and np.all(np.diff(evo) >= 0)
    ev_of_track = np.repeat(np.arange(64), np.diff(evo))
    ev_off = d["ev_off"]
    assert np.all(hits >= ev_off[ev_of_track[owner]]) and np.all(hits < ev_off[ev_of_track[owner] + 1])


def _sample_events(d):
    sizes = np.diff(d["ev_off"])
    order = np.argsort(sizes)
    return [int(order[-1]), int(order[len(order) // 2]), int(order[len(order) // 8])]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_sampled_events_match_the_oracle(batch, k):
    d, ctx, cl, g = batch
    e = _sample_events(d)[k]
    a, b = int(d["ev_off"][e]), int(d["ev_off"][e + 1])
    pad, tim, bo = d["pad"][a:b], d["tim"][a:b], d["ev_bin_off"][e]
    o = O.track_event(pad, tim, bo)
    t0, t1 = int(g["ev_trk_off"][e]), int(g["ev_trk_off"][e + 1])
    goff = g["trk_off"][t0:t1 + 1]
    np.testing.assert_array_equal(goff - goff[0], o["trk_off"])
    np.testing.assert_array_equal(g["trk_hits"][goff[0]:goff[-1]] - a, o["trk_hits"])
    # FP32 square-root refit against the FP64 oracle (consistent tracks)
    f = O.fit(pad, tim, bo, o["trk_off"], o["trk_hits"])
    gp, gc = g["par"][t0:t1], g["chi2"][t0:t1]
    both = (f["ndf"] > 0) & (g["ndf"][t0:t1] > 0)
    good = both & (f["chi2"] < 5 * np.maximum(f["ndf"], 1))
    sig = np.sqrt(np.maximum(f["cov"][:, [0, 2, 5, 9, 14]], 0.0))
    scale = np.maximum(np.maximum(np.abs(f["par"]), [1.0, 1.0, 0.1, 0.1, 0.1]), sig)
    err = np.abs(gp - f["par"]) / scale
    print("event %d: %d clusters, %d tracks, max par err %s" % (e, b - a, t1 - t0, err[good].max(axis=0)))
    assert np.all(err[good].max(axis=0) < 1e-4)
    tight = good & (f["chi2"] < 2 * np.maximum(f["ndf"], 1))
    assert np.all(np.abs(gc[tight] - f["chi2"][tight]) / np.maximum(f["chi2"][tight], 1.0) < 2e-4)


def test_batch_refit_records_match_the_oracle_on_a_sampled_event(batch):
    """tpc_refit_grad over the whole batch (the bench's second half of a step): the per-track chi2
    records of a sampled event equal the oracle's refit chi2 (weights 1, nominal calibration)."""
    d, ctx, cl, g = batch
    nt = g["n_tracks"]
    th = torch.tensor(synth.theta_nominal(), dtype=torch.float64, device="cuda")
    s = torch.empty(1, dtype=torch.float64, device="cuda")
    gr = torch.empty(73, dtype=torch.float64, device="cuda")
    ctx.tpc_refit_grad(cl, g["tracks_obj"], th, s, gr)
    rec = torch.empty(nt * 26, dtype=torch.float32, device="cuda")
    ctx.tpc_debug_copy(11, rec)
    assert ctx.tpc_sync_status() == 0
    chi = rec.view(nt, 26)[:, 0].cpu().numpy()
    e = _sample_events(d)[1]
    a, b = int(d["ev_off"][e]), int(d["ev_off"][e + 1])
    pad, tim, bo = d["pad"][a:b], d["tim"][a:b], d["ev_bin_off"][e]
    t0, t1 = int(g["ev_trk_off"][e]), int(g["ev_trk_off"][e + 1])
    goff = g["trk_off"][t0:t1 + 1]
    f = O.fit(pad, tim, bo, goff - goff[0], g["trk_hits"][goff[0]:goff[-1]] - a)
    ok = (f["ndf"] > 0) & (f["chi2"] < 2 * np.maximum(f["ndf"], 1))
    rel = np.abs(chi[t0:t1][ok] - f["chi2"][ok]) / np.maximum(f["chi2"][ok], 1.0)
    assert rel.max() < 2e-4, rel.max()
    assert np.isfinite(s.item()) and np.all(np.isfinite(gr.cpu().numpy()))
