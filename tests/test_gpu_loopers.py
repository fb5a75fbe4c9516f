"""Looper-leg pairing on the GPU (tpc_looper_pairs) against the oracle's (or_looper_pairs): section 3
of the paper merges track segments after the sector tracking; the two legs of a low-pT looper leave
the tracking as two tracks and are joined here."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1712_09434_gb300 import capi, synth
from tests import _events, _gpu
from tests import test_oracle_loopers as L

pytestmark = pytest.mark.gpu


def _gpu_pairs(ctx, cl, tr, nt):
    pair = torch.full((max(nt, 1),), -7, dtype=torch.int32, device="cuda")
    leg = torch.full((max(nt, 1),), -7, dtype=torch.int32, device="cuda")
    ctx.tpc_looper_pairs(cl, tr, pair, leg)
    assert ctx.tpc_sync_status() == 0
    return pair.cpu().numpy()[:nt], leg.cpu().numpy()[:nt]


def _looper_rich(seed=1011):
    return synth.make_event(synth.EventConfig(n_tracks=3000, noise_frac=0.1, looper_frac=0.3, seed=seed))


@pytest.mark.parametrize("name", ["rich", "c3"])
def test_looper_pairs_equal_the_oracle(name):
    """The GPU pairs (FP64 decisions from its FP32 fit) equal the oracle's (FP64 fit) for at least
    99.9 % of the tracks: a decision can differ only where a gate or the order of two candidates is
    within the rounding of the two fits."""
    ev = _looper_rich() if name == "rich" else _events.event(name)
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    g = _gpu.run(ctx, cl)
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    np.testing.assert_array_equal(g["trk_hits"], o["trk_hits"])
    pair, leg = _gpu_pairs(ctx, cl, g["tracks_obj"], g["n_tracks"])
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    sec = ev.sector[o["trk_hits"][o["trk_off"][:-1]]].astype(np.int32)
    opair, oleg, _ = O.looper_pairs(f, sec)
    same = (pair == opair).mean()
    print("%s: %d tracks, %d pairs on the GPU, %d by the oracle, identical for %.5f" % (
        name, len(pair), (pair >= 0).sum() // 2, (opair >= 0).sum() // 2, same))
    assert same > 0.999
    m = pair >= 0
    assert np.all(pair[pair[m]] == np.nonzero(m)[0])
    both = m & (pair == opair)
    assert np.all(leg[both] == oleg[both]) and np.all(leg[~m] == 0)
    ctx.close()


def _constructed(legs, events=None, n_events=1):
    """Clusters and a track object for hand-made fitted states: one cluster per track, in row 0 of
    the track's sector (and event), the track's first and only hit; par and xref rounded to FP32,
    and the oracle given the same rounded values."""
    nt = len(legs)
    ev_of = np.zeros(nt, np.int64) if events is None else np.asarray(events, np.int64)
    nb = n_events * synth.N_SECTORS * synth.N_ROWS
    bins = np.array([ev_of[t] * synth.N_SECTORS * synth.N_ROWS + legs[t][2] * synth.N_ROWS for t in range(nt)])
    order = np.argsort(bins, kind="stable")
    cl_of_trk = np.empty(nt, np.int64)
    cl_of_trk[order] = np.arange(nt)
    bin_off = np.zeros(nb + 1, np.int32)
    np.add.at(bin_off, bins + 1, 1)
    bin_off = np.cumsum(bin_off).astype(np.int32)
    cl = capi.Clusters.from_numpy(np.zeros(nt, np.int16), np.zeros(nt, np.uint16), bin_off, n_events)
    tr = capi.Tracks(nt, n_events, nt, nt)
    par = np.array([l[0] for l in legs], np.float32)
    xref = np.array([l[1] for l in legs], np.float32)
    tr.par[:5 * nt] = torch.from_numpy(par.reshape(-1)).cuda()
    tr.xref[:nt] = torch.from_numpy(xref).cuda()
    tr.ndf[:nt] = 20
    tr.trk_off[:nt + 1] = torch.arange(nt + 1, dtype=torch.int32, device="cuda")
    tr.trk_hits[:nt] = torch.from_numpy(cl_of_trk.astype(np.int32)).cuda()
    tr.n_tracks[0] = nt
    f = dict(par=par.astype(np.float64), xref=xref.astype(np.float64), ndf=np.full(nt, 20, np.int32))
    sec = np.array([l[2] for l in legs], np.int32)
    ref = O.looper_pairs(f, sec, None if events is None else np.asarray(events, np.int32))
    return cl, tr, ref


def _edge_cases():
    cx, cy, R, tl, zf = L._base()
    A = L._legs(cx, cy, R, tl, zf)[0]
    u = (-cy / math.hypot(cx, cy), cx / math.hypot(cx, cy))
    cases = [("two legs", [A, L._legs(cx, cy, R, tl, zf)[1]], [1, 0])]
    for shift, ok in ((4.99, True), (5.01, False)):
        cases.append(("centre %.2f" % shift, [A, L._legs(cx + shift * u[0], cy + shift * u[1], R, tl, zf)[1]], ok))
    for dR, ok in ((4.99, True), (5.01, False), (-4.99, True), (-5.01, False)):
        cases.append(("radius %.2f" % dR, [A, L._legs(cx, cy, R + dR, tl, zf)[1]], ok))
    for dz, ok in ((7.99, True), (8.01, False), (-7.99, True), (-8.01, False)):
        cases.append(("far z %.2f" % dz, [A, L._legs(cx, cy, R, tl, zf + dz)[1]], ok))
    for dtl, ok in ((0.0499, True), (0.0501, False)):
        cases.append(("tan lambda %.4f" % dtl, [A, L._legs(cx, cy, R, tl + dtl, zf)[1]], ok))
    B = L._legs(cx, cy, R + 1.0, tl, zf)[1]
    Cl = L._legs(cx, cy, R + 2.0, tl, zf)[1]
    Dl = L._legs(cx, cy, R + 1.0, tl, zf)[0]
    cases.append(("mutual best", [A, B, Cl, Dl], [-1, 3, -1, 1]))
    near = L._legs(cx, cy, R, tl, zf + 1.0)[1]
    far = L._legs(cx, cy, R, tl, zf + 2.0)[1]
    cases.append(("score order", [A, far, near], [2, -1, 0]))
    for R2, ok in ((129.9, True), (130.1, False)):
        c2 = L._base(R=R2, phi_c=0.7, tl=0.2, z_far=100.0)
        cases.append(("radius limit %.1f" % R2, L._legs(*c2), ok))
    for rc, ok in ((40.1, True), (39.9, False)):
        cases.append(("centre limit %.1f" % rc, L._legs(rc * math.cos(2.0), rc * math.sin(2.0), 60.0, 0.3, 50.0,
                                                         dpsi=0.5), ok))
    # a circle whose centre lies on the edge of an azimuth bin of the GPU's grid (10 degrees), the
    # other leg's centre 4 cm away across it
    for deg in (40.0, 0.0):     # 0: the bins 35 and 0 of the wrap-around
        phi_e = math.radians(deg)
        ce = (80.0 * math.cos(phi_e), 80.0 * math.sin(phi_e))
        ue = (-math.sin(phi_e), math.cos(phi_e))
        cases.append(("across the bin edge at %g deg" % deg,
                      [L._legs(ce[0] - 2.0 * ue[0], ce[1] - 2.0 * ue[1], 80.0, 0.3, 70.0)[0],
                       L._legs(ce[0] + 2.0 * ue[0], ce[1] + 2.0 * ue[1], 80.0, 0.3, 70.0)[1]], [1, 0]))
    return cases


@pytest.mark.parametrize("case", _edge_cases(), ids=lambda c: c[0])
def test_constructed_cases_equal_the_oracle(case):
    """Hand-made fitted states at every gate edge, the limits of a candidate, mutual best, the score
    order and centres on either side of an azimuth bin edge: the GPU gives the oracle's pairs and legs
    on the same FP32 inputs, and the expected ones."""
    name, legs, expect = case
    ctx = _gpu.make_context(1000, 1)
    cl, tr, (opair, oleg, _) = _constructed(legs)
    pair, leg = _gpu_pairs(ctx, cl, tr, len(legs))
    np.testing.assert_array_equal(pair, opair)
    np.testing.assert_array_equal(leg, oleg)
    if isinstance(expect, bool):
        assert (pair[0] == 1) == expect
    else:
        assert list(pair) == expect
    ctx.close()


def test_pairs_stay_inside_their_event():
    """The same two legs in events 0 and 1 of a batch, the returning legs swapped between the events'
    track lists: each outgoing leg pairs with the returning leg of its own event only."""
    cx, cy, R, tl, zf = L._base()
    a, b = L._legs(cx, cy, R, tl, zf)
    legs, events = [a, b, a, b], [0, 1, 1, 0]
    ctx = _gpu.make_context(1000, 2)
    cl, tr, (opair, oleg, _) = _constructed(legs, events, n_events=2)
    pair, leg = _gpu_pairs(ctx, cl, tr, 4)
    np.testing.assert_array_equal(pair, opair)
    assert list(pair) == [3, 2, 1, 0]
    ctx.close()


def test_looper_pairs_arguments():
    ev = _events.event("c1")
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    g = _gpu.run(ctx, cl)
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_looper_pairs(cl, g["tracks_obj"], None)
    assert e.value.code == capi.TPC_ERR_INVALID_ARG
    ctx.close()
