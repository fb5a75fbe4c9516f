"""TPC-ITS matching on the GPU (tpc_its_match) against the oracle's, and the drift calibration with
the references it produces in place of references assigned by generator truth: the calibration of
sections 2.1 and 6 of the paper, matching TPC tracks to inner-tracker tracks."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1712_09434_gb300 import calib, capi, synth
from tests import _events, _gpu
from tests.test_gpu_calibration import BLOCKS

pytestmark = pytest.mark.gpu


def _gpu_match(ctx, cl, g, its32):
    nt = g["n_tracks"]
    its_d = torch.tensor(its32, dtype=torch.float32, device="cuda")
    mt = torch.full((max(nt, 1),), -7, dtype=torch.int32, device="cuda")
    mi = torch.full((max(len(its32), 1),), -7, dtype=torch.int32, device="cuda")
    anchor = torch.zeros((max(nt, 1), 8), dtype=torch.float32, device="cuda")
    ctx.tpc_its_match(cl, g["tracks_obj"], its_d, mt, mi, anchor)
    assert ctx.tpc_sync_status() == 0
    return mt.cpu().numpy()[:nt], mi.cpu().numpy()[:len(its32)], anchor.cpu().numpy()[:nt]


@pytest.mark.parametrize("name", ["c2", "c5"])
def test_its_match_equals_the_oracle(name):
    """The GPU matches (its FP32 fit, FP64 extrapolation and chi2) equal the oracle's (FP64 fit) for
    at least 99.9 % of the tracks: a match decided by floating point can differ only where two
    candidates or the gate are within rounding; the references written for matched tracks of the
    reference selection are the ITS track's values."""
    ev = _events.event(name)
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    g = _gpu.run(ctx, cl)
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    np.testing.assert_array_equal(g["trk_hits"], o["trk_hits"])
    its, part = synth.its_tracks(ev)
    its32 = its.astype(np.float32)
    mt, mi, anchor = _gpu_match(ctx, cl, g, its32)
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    sec = ev.sector[o["trk_hits"][o["trk_off"][:-1]]].astype(np.int32)
    omt, omi, _ = O.its_match(f, sec, its32.astype(np.float64))
    same = (mt == omt).mean()
    print("%s: %d tracks, %d matched on the GPU, %d by the oracle, identical for %.5f" % (
        name, len(mt), (mt >= 0).sum(), (omt >= 0).sum(), same))
    assert same > 0.999
    m = mt >= 0
    assert np.all(mi[mt[m]] == np.nonzero(m)[0])
    # references only for matched tracks that start within the first 8 rows, have >= 30 hits and
    # |sin phi| < 0.9 at the vertex (from the oracle's own fit and extrapolation)
    first_row = ev.row[o["trk_hits"][o["trk_off"][:-1]]]
    nh = np.diff(o["trk_off"])
    snp = np.array([O.propagate(f["xref"][t], f["par"][t], 0.0)[1][2] if m[t] else 0.0 for t in range(len(mt))])
    ref = m & (first_row <= 8) & (nh >= 30) & (np.abs(snp) < 0.9)
    has = anchor[:, 0] > 0
    assert (has != ref).sum() <= max(2, len(mt) // 2000), (has != ref).sum()
    both = has & ref
    np.testing.assert_array_equal(anchor[both][:, [1, 2, 3, 4, 5, 6]], its32[mt[both]][:, [1, 5, 2, 6, 3, 7]])
    assert np.all(anchor[both][:, 0] == np.float32(0.01)) and np.all(anchor[~has] == 0)
    ctx.close()


def test_calibration_with_matched_its_references():
    """The 20-step recovery of the injected calibration with references from tpc_its_match (ITS
    tracks with 95 % efficiency and 2 % fakes; references for matched tracks starting at the inner
    wall, >= 30 hits, |sin phi| < 0.9 at the vertex) instead of references assigned by truth: every
    parameter within 5 standard errors of its injected value, each block's remaining distortion
    within 3 times its statistical expectation."""
    ev = _events.event("c5")
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    g = _gpu.run(ctx, cl)
    its, part = synth.its_tracks(ev)
    mt, _, anchor = _gpu_match(ctx, cl, g, its.astype(np.float32))
    ok = (g["ndf"] > 0) & (g["chi2"] < 5.0 * np.maximum(g["ndf"], 1))
    w = torch.tensor(ok.astype(np.float32), device="cuda")
    th_star = synth.calib_theta(1005)
    th0 = synth.theta_nominal()
    res, n_drop, n_calls = calib.calibrate(ctx, cl, g["tracks_obj"], w, anchor.astype(np.float64), th0, steps=20)
    pull = (res.theta - th_star) / res.sigma
    frac = [np.linalg.norm(res.theta[b] - th_star[b]) / np.linalg.norm(th0[b] - th_star[b]) for b in BLOCKS]
    expect = [np.sqrt(np.sum(res.sigma[b] ** 2)) / np.linalg.norm(th0[b] - th_star[b]) for b in BLOCKS]
    lead = np.array([np.bincount(np.maximum(ev.mc_track[g["trk_hits"][a:b]], 0)).argmax()
                     for a, b in zip(g["trk_off"][:-1], g["trk_off"][1:])])
    m = mt >= 0
    print("matched %d of %d tracks (%.4f to the right particle, %d to fakes), %d with references, %d dropped" % (
        m.sum(), len(mt), (part[mt[m]] == lead[m]).mean(), (part[mt[m]] < 0).sum(), int((anchor[:, 0] > 0).sum()),
        n_drop))
    print("remaining distortion per block:", np.round(frac, 5), "expectation", np.round(expect, 5))
    print("max |pull| per block:", [float(np.abs(pull[b]).max()) for b in BLOCKS])
    assert np.all(np.array(frac) < 3.0 * np.array(expect)), (frac, expect)
    assert np.all(np.abs(pull) < 5.0), pull
    ctx.close()


def test_its_match_arguments():
    ev = _events.event("c1")
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    g = _gpu.run(ctx, cl)
    too_many = torch.zeros((ev.n_clusters // 5 + 2, 8), dtype=torch.float32, device="cuda")
    mt = torch.empty(g["n_tracks"], dtype=torch.int32, device="cuda")
    mi = torch.empty(too_many.shape[0], dtype=torch.int32, device="cuda")
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_its_match(cl, g["tracks_obj"], too_many, mt, mi)
    assert e.value.code == capi.TPC_ERR_CAPACITY
    misaligned = torch.zeros(8 * g["n_tracks"] + 1, dtype=torch.float32, device="cuda")[1:]
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_its_match(cl, g["tracks_obj"], too_many[:10], mt, mi, misaligned)
    assert e.value.code == capi.TPC_ERR_INVALID_ARG
    ctx.close()
