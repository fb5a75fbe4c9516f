"""Time frames on the GPU: the slices tracked as one batch (tpc_track_batch) and joined by
tpc_merge_slices, bit-exact against the oracle's track_frame (slice tracks, links, frame tracks),
and at the bench's full size (64 collisions, 33 M clusters) on a sampled pair of slices plus the
properties of the whole frame."""
import numpy as np
import pytest
import torch

import bench
from oracle import oracle as O
from paper_1712_09434_gb300 import capi, synth
from tests import _gpu
from tests.test_frame_oracle import line_frame

pytestmark = pytest.mark.gpu


def run_frame(ctx, pad, tim, bin_off, n_slices, slice_len):
    n = int(pad.shape[0])
    cl = capi.Clusters.from_numpy(pad, tim, bin_off, n_slices)
    st = capi.Tracks(n, n_slices, max(n // 10 + 16, 64), max(n, 1))
    ctx.tpc_track_batch(cl, st)
    fr = capi.Tracks(n, 1, max(n // 10 + 16, 64), max(n, 1))
    ctx.tpc_merge_slices(cl, st, slice_len, fr)
    s = ctx.tpc_sync_status()
    assert s == 0, capi.lib().tpc_strerror(s)
    a, b = st.to_host(), fr.to_host()
    nxt = torch.empty(max(a["n_tracks"], 1), dtype=torch.int32, device="cuda")
    ctx.tpc_debug_copy(9, nxt)
    return dict(trk_off=a["trk_off"], trk_hits=a["trk_hits"], ev_trk_off=a["ev_trk_off"], label=a["label"],
                next=nxt.cpu().numpy()[:a["n_tracks"]], ftrk_off=b["trk_off"], ftrk_hits=b["trk_hits"],
                flabel=b["label"], fevo=b["ev_trk_off"])


def compare(g, o):
    for k in ("trk_off", "trk_hits", "ev_trk_off", "next", "ftrk_off", "ftrk_hits", "flabel"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    assert list(g["fevo"][:2]) == [0, len(o["ftrk_off"]) - 1]


@pytest.fixture(scope="module")
def ctx():
    c = _gpu.make_context(6_000_000, 64)
    yield c
    c.close()


def test_constructed_line_is_one_frame_track(ctx):
    (pad, tim, bin_off, o), sl = line_frame()
    g = run_frame(ctx, pad, tim, bin_off, 2, 32000)
    compare(g, O.track_frame(pad, tim, bin_off, 2, 32000))
    assert len(g["ftrk_off"]) == 2 and list(g["next"]) == [-1, 0]


@pytest.mark.parametrize("n_col,per_drift,slice_len", [(6, 5.0, 32000), (4, 3.0, 6000), (3, 8.0, 1000)])
def test_frame_matches_oracle(ctx, n_col, per_drift, slice_len):
    evs = [synth.make_event(c) for c in synth.batch_configs(n_col, seed0=2000 + 10 * n_col)]
    tf = synth.time_frame(evs, per_drift=per_drift, slice_len=slice_len, seed=3000 + n_col)
    o = O.track_frame(tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices, tf.slice_len)
    g = run_frame(ctx, tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices, tf.slice_len)
    compare(g, o)
    print("%d collisions, %d slices of %d LSB: %d slice tracks, %d links, %d frame tracks" % (
        n_col, tf.n_slices, slice_len, len(o["trk_off"]) - 1, (o["next"] >= 0).sum(), len(o["ftrk_off"]) - 1))
    assert (o["next"] >= 0).sum() > 0


def test_full_size_frame_sampled_slices():
    tf = bench.make_frame(64, 2000)
    n = tf["pad"].shape[0]
    ns = int(tf["n_slices"])
    c = _gpu.make_context(n, ns)
    try:
        g = run_frame(c, tf["pad"], tf["tim"], tf["bin_off"], ns, int(tf["slice_len"]))
    finally:
        c.close()
    # whole frame: frame tracks partition the slice tracks, links go from slice j+1 to slice j
    assert np.array_equal(np.sort(g["ftrk_hits"]), np.sort(g["trk_hits"]))
    owner = np.repeat(np.arange(len(g["ftrk_off"]) - 1), np.diff(g["ftrk_off"]))
    np.testing.assert_array_equal(g["flabel"][g["ftrk_hits"]], owner)
    sl = np.searchsorted(g["ev_trk_off"], np.arange(len(g["trk_off"]) - 1), side="right") - 1
    s = np.nonzero(g["next"] >= 0)[0]
    assert np.all(sl[s] == sl[g["next"][s]] + 1) and len(np.unique(g["next"][s])) == len(s)
    assert len(s) > 10000
    # a sampled pair of consecutive slices in the middle: the oracle's tracks of both slices and
    # its links from the later one
    nbe = synth.N_SECTORS * synth.N_ROWS
    j = ns // 2
    ev_off = tf["bin_off"][::nbe].astype(np.int64)
    a, b = int(ev_off[j]), int(ev_off[j + 2])
    sub_bin = (tf["bin_off"][j * nbe:(j + 2) * nbe + 1].astype(np.int64) - a).astype(np.int32)
    o = O.track_frame(tf["pad"][a:b], tf["tim"][a:b], sub_bin, 2, int(tf["slice_len"]))
    t0, t2 = int(g["ev_trk_off"][j]), int(g["ev_trk_off"][j + 2])
    off = g["trk_off"][t0:t2 + 1]
    np.testing.assert_array_equal(off - off[0], o["trk_off"])
    np.testing.assert_array_equal(g["trk_hits"][off[0]:off[-1]] - a, o["trk_hits"])
    t1 = int(g["ev_trk_off"][j + 1])
    gn = g["next"][t1:t2]
    on = o["next"][t1 - t0:]
    np.testing.assert_array_equal(np.where(gn >= 0, gn - t0, -1), on)


def test_frames_with_empty_slices(ctx):
    """Collisions far apart leave whole slices empty; an empty frame has no tracks at all."""
    evs = [synth.make_event(synth.EventConfig(n_tracks=300, noise_frac=0.1, seed=s)) for s in (41, 42)]
    tf = synth.time_frame(evs, slice_len=16000, t0=[0, 96000])
    o = O.track_frame(tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices, tf.slice_len)
    assert np.any(np.diff(tf.ev_off) == 0)                      # some slices hold no cluster
    g = run_frame(ctx, tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices, tf.slice_len)
    compare(g, o)
    n_sl = 5
    empty_bo = np.zeros(n_sl * synth.N_SECTORS * synth.N_ROWS + 1, np.int32)
    e = run_frame(ctx, np.zeros(0, np.int16), np.zeros(0, np.uint16), empty_bo, n_sl, 32000)
    assert len(e["ftrk_off"]) == 1 and len(e["ftrk_hits"]) == 0 and list(e["fevo"][:2]) == [0, 0]
