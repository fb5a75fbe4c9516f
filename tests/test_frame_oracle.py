"""Pins of the oracle's time-frame slice merge (S11; section 3 of arxiv 1712.09434, its outlook
for continuous readout: slices of a time frame tracked one by one, segments merged afterwards)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_09434_gb300 import synth

NBE = synth.N_SECTORS * synth.N_ROWS


def frame_arrays(sl, sec, row, pad, tim, n_slices):
    """Clusters given by (slice, sector, row, pad, slice-local time) in the frame layout."""
    gb = np.asarray(sl) * NBE + np.asarray(sec) * synth.N_ROWS + np.asarray(row)
    o = np.lexsort((tim, pad, gb))
    gb = gb[o]
    bin_off = np.searchsorted(gb, np.arange(n_slices * NBE + 1)).astype(np.int32)
    return np.asarray(pad)[o].astype(np.int16), np.asarray(tim)[o].astype(np.uint16), bin_off, o


def line_frame(kink=0):
    """One track on all 159 rows of sector 0: Y a parabola in the row, readout time 40000 - 100 r
    (falling outwards, as for a particle from the vertex), plus kink after row 80.  Slices of
    32000 LSB: rows 0-80 fall in slice 1, rows 81-158 in slice 0."""
    r = np.arange(159)
    y = -1500 + 20 * r + (r * r) // 8
    tau = 40000 - 100 * r + np.where(r > 80, kink, 0)
    sl = tau // 32000
    return frame_arrays(sl, np.zeros(159, int), r, y, tau - sl * 32000, 2), sl


def test_line_split_by_the_slice_boundary_is_one_frame_track():
    (pad, tim, bin_off, o), sl = line_frame()
    f = O.track_frame(pad, tim, bin_off, 2, 32000)
    assert list(f["ev_trk_off"]) == [0, 1, 2]
    assert list(np.diff(f["trk_off"])) == [78, 81]            # slice 0: rows 81-158; slice 1: rows 0-80
    assert list(f["next"]) == [-1, 0]                          # the slice-1 piece continues in slice 0
    assert len(f["ftrk_off"]) == 2
    np.testing.assert_array_equal(o[f["ftrk_hits"]], np.arange(159))   # generation index = row
    assert np.all(f["flabel"] == 0)


def test_pieces_that_do_not_meet_stay_apart():
    """A 300 LSB jump in time across the boundary exceeds the 192 LSB merge window."""
    (pad, tim, bin_off, o), sl = line_frame(kink=-300)
    f = O.track_frame(pad, tim, bin_off, 2, 32000)
    assert list(np.diff(f["trk_off"])) == [78, 81]
    assert list(f["next"]) == [-1, -1]
    assert len(f["ftrk_off"]) == 3


def test_single_slice_frame_is_plain_tracking():
    ev = synth.make_event(synth.EventConfig(n_tracks=400, noise_frac=0.1, seed=11))
    tf = synth.time_frame([ev], t0=[0], slice_len=32001)     # drift times reach 32000
    assert tf.n_slices == 1
    np.testing.assert_array_equal(tf.pad_fp, ev.pad_fp)
    f = O.track_frame(tf.pad_fp, tf.time_fp, tf.bin_off, 1, tf.slice_len)
    np.testing.assert_array_equal(tf.time_fp, ev.time_fp)
    e = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    np.testing.assert_array_equal(f["ftrk_off"], e["trk_off"])
    np.testing.assert_array_equal(f["ftrk_hits"], e["trk_hits"])
    assert np.all(f["next"] < 0)


def test_a_whole_slice_of_delay_changes_nothing():
    """Delaying every collision by exactly one slice only prepends an empty slice."""
    evs = [synth.make_event(synth.EventConfig(n_tracks=300, noise_frac=0.1, seed=s)) for s in (21, 22)]
    t = np.array([0, 9000])
    a = synth.time_frame(evs, slice_len=16000, t0=t)
    b = synth.time_frame(evs, slice_len=16000, t0=t + 16000)
    assert b.n_slices == a.n_slices + 1
    np.testing.assert_array_equal(a.pad_fp, b.pad_fp)
    np.testing.assert_array_equal(a.time_fp, b.time_fp)
    fa = O.track_frame(a.pad_fp, a.time_fp, a.bin_off, a.n_slices, a.slice_len)
    fb = O.track_frame(b.pad_fp, b.time_fp, b.bin_off, b.n_slices, b.slice_len)
    np.testing.assert_array_equal(fa["ftrk_off"], fb["ftrk_off"])
    np.testing.assert_array_equal(fa["ftrk_hits"], fb["ftrk_hits"])
    assert (fa["next"] >= 0).sum() > 20


@pytest.fixture(scope="module")
def frame6():
    evs = [synth.make_event(c) for c in synth.batch_configs(6, seed0=2000)]
    tf = synth.time_frame(evs, per_drift=5.0)
    return evs, tf, O.track_frame(tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices, tf.slice_len)


def _dominant(mc, hits):
    v = mc[hits]
    v = v[v >= 0]
    if len(v) == 0:
        return -1, 0.0
    u, c = np.unique(v, return_counts=True)
    return u[c.argmax()], c.max() / len(hits)


def test_slice_links_join_the_same_particle(frame6):
    evs, tf, f = frame6
    off, hits = f["trk_off"], f["trk_hits"]
    links = [(s, t) for s, t in enumerate(f["next"]) if t >= 0]
    assert len(links) > 1000
    same = sum(_dominant(tf.mc, hits[off[s]:off[s + 1]])[0] == _dominant(tf.mc, hits[off[t]:off[t + 1]])[0]
               for s, t in links)
    assert same / len(links) > 0.97


def test_particles_cut_by_a_slice_boundary_are_joined(frame6):
    """Particles that do not loop (pT > 0.3 GeV) and were found as pure (>= 90 %) tracks in two
    consecutive slices end in one frame track in more than 90 % of the cases."""
    evs, tf, f = frame6
    off, hits = f["trk_off"], f["trk_hits"]
    sl = np.searchsorted(f["ev_trk_off"], np.arange(len(off) - 1), side="right") - 1
    pieces = {}
    for t in range(len(off) - 1):
        p, pur = _dominant(tf.mc, hits[off[t]:off[t + 1]])
        if p >= 0 and pur >= 0.9 and evs[p >> 32].trk_pt[p & 0xffffffff] > 0.3:
            pieces.setdefault(p, []).append((sl[t], t))
    cut = [v for v in pieces.values() if len(v) == 2 and abs(v[0][0] - v[1][0]) == 1]
    assert len(cut) > 500
    joined = sum(f["flabel"][hits[off[v[0][1]]]] == f["flabel"][hits[off[v[1][1]]]] for v in cut)
    assert joined / len(cut) > 0.9


def test_frame_tracks_partition_the_slice_tracks(frame6):
    evs, tf, f = frame6
    assert np.array_equal(np.sort(f["ftrk_hits"]), np.sort(f["trk_hits"]))
    assert len(np.unique(f["ftrk_hits"])) == len(f["ftrk_hits"])
    owner = np.repeat(np.arange(len(f["ftrk_off"]) - 1), np.diff(f["ftrk_off"]))
    np.testing.assert_array_equal(f["flabel"][f["ftrk_hits"]], owner)
    # a link goes from slice j+1 to slice j, and every track has at most one predecessor
    sl = np.searchsorted(f["ev_trk_off"], np.arange(len(f["trk_off"]) - 1), side="right") - 1
    s = np.nonzero(f["next"] >= 0)[0]
    assert np.all(sl[s] == sl[f["next"][s]] + 1)
    assert len(np.unique(f["next"][s])) == len(s)


def test_frame_with_empty_slices_keeps_offsets():
    """Two collisions far apart (a whole number of slices between them, so that each is cut where
    it would be cut alone) leave empty slices in the middle of the frame: the frame holds exactly
    the slice tracks and frame tracks of the two collisions tracked alone."""
    evs = [synth.make_event(synth.EventConfig(n_tracks=300, noise_frac=0.1, seed=s)) for s in (41, 42)]

    def frame(events, t0):
        tf = synth.time_frame(events, slice_len=16000, t0=t0)
        return tf, O.track_frame(tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices, tf.slice_len)

    tf, f = frame(evs, [0, 96000])
    assert np.any(np.diff(tf.ev_off) == 0)
    assert np.all(np.diff(f["trk_off"]) >= 10)
    alone = [frame([ev], [0])[1] for ev in evs]
    assert len(f["trk_off"]) - 1 == sum(len(a["trk_off"]) - 1 for a in alone)
    assert len(f["ftrk_off"]) - 1 == sum(len(a["ftrk_off"]) - 1 for a in alone)
    assert len(f["trk_hits"]) == sum(len(a["trk_hits"]) for a in alone)
