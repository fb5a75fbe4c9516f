"""Error paths of the C ABI on a GPU: argument validation, reservation, capacity overflow, bounds,
and a bounded device wait that runs out.  Every failure is made on the host or by a wait that
nothing completes; no test faults, traps or hangs the GPU."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1712_09434_gb300 import capi, synth
from tests import _events, _gpu

pytestmark = pytest.mark.gpu


def test_invalid_arguments_and_reservation():
    ev = _events.event("c1")
    ctx = capi.Context()                                   # nothing reserved yet
    cl = _gpu.clusters_of(ev)
    tr = capi.Tracks(ev.n_clusters, 1, 1000, ev.n_clusters)
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_track_event(cl, tr)
    assert e.value.code == capi.TPC_ERR_NOT_RESERVED
    ctx.reserve(ev.n_clusters // 2, 1)
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_track_event(cl, tr)
    assert e.value.code == capi.TPC_ERR_NOT_RESERVED
    ctx.reserve(ev.n_clusters, 1)                          # grows
    bad = capi.Tracks(ev.n_clusters, 1, 1000, ev.n_clusters)
    bad.trk_hits = None
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_track_event(cl, bad)
    assert e.value.code == capi.TPC_ERR_INVALID_ARG
    ctx.tpc_track_event(cl, tr)
    assert ctx.tpc_sync_status() == capi.TPC_OK
    ctx.close()


def test_output_capacity_overflow_is_reported_not_written():
    ev = _events.event("c1")
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    cap_t, cap_h, tail = 8, 64, 4096
    tr = capi.Tracks(ev.n_clusters, 1, cap_t, cap_h)
    # each bounded output is the head of a larger buffer whose tail must stay untouched
    outer = {}
    for name, n, dt in [("trk_off", cap_t + 1, torch.int32), ("trk_hits", cap_h, torch.int32),
                        ("par", 5 * cap_t, torch.float32), ("cov", 15 * cap_t, torch.float32),
                        ("chi2", cap_t, torch.float32), ("ndf", cap_t, torch.int32), ("xref", cap_t, torch.float32)]:
        big = torch.full((n + tail,), 12345, dtype=dt, device="cuda")
        setattr(tr, name, big[:n])
        outer[name] = (big, n)
    ctx.tpc_track_event(cl, tr)
    assert ctx.tpc_sync_status() == capi.TPC_ERR_CAPACITY
    for name, (big, n) in outer.items():
        assert bool((big[n:] == 12345).all()), name
    assert int(tr.n_tracks.item()) > cap_t                 # the true count is still reported
    # the context is usable afterwards and gives the full result
    tr2 = capi.Tracks(ev.n_clusters, 1, 4096, ev.n_clusters)
    ctx.tpc_track_event(cl, tr2)
    assert ctx.tpc_sync_status() == capi.TPC_OK
    assert int(tr2.n_tracks.item()) == int(tr.n_tracks.item())
    ctx.close()


def test_row_bin_beyond_the_local_index_range_is_a_bounds_error():
    # 70000 clusters in one (sector, row) bin: row-local indices are 16 bit
    n = 70000
    pad = np.sort(np.random.default_rng(1).integers(-1000, 1000, n)).astype(np.int16)
    tim = np.full(n, 1000, np.uint16)
    bin_off = np.zeros(36 * 159 + 1, np.int32)
    bin_off[5:] = n                                          # all in bin 4 (sector 0, row 4)
    ctx = _gpu.make_context(n, 1)
    cl = capi.Clusters.from_numpy(pad, tim, bin_off, 1)
    tr = capi.Tracks(n, 1, 1024, n)
    ctx.tpc_track_event(cl, tr)
    assert ctx.tpc_sync_status() == capi.TPC_ERR_BOUNDS
    ctx.close()


def test_bounded_wait_times_out_and_reports():
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    rc = capi.lib().tpc_selftest_wait_timeout(ctypes.c_void_p(st.data_ptr()), 1000,
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == capi.TPC_OK
    torch.cuda.synchronize()
    assert int(st.item()) == capi.TPC_ERR_TIMEOUT
    # the context and the device stay usable
    ev = _events.event("c1")
    ctx = _gpu.make_context(ev.n_clusters, 1)
    g = _gpu.run(ctx, _gpu.clusters_of(ev))
    assert g["n_tracks"] > 50
    ctx.close()


def test_slice_merge_arguments_and_capacity():
    """tpc_merge_slices: slice lengths outside [1, 32001] and missing outputs are invalid; a frame
    output too small for the frame tracks is a capacity error on the device, with nothing written
    beyond it."""
    tf = synth.time_frame([_events.event("c1")], t0=[0], slice_len=16000)
    ctx = _gpu.make_context(tf.n_clusters, tf.n_slices)
    cl = capi.Clusters.from_numpy(tf.pad_fp, tf.time_fp, tf.bin_off, tf.n_slices)
    st = capi.Tracks(tf.n_clusters, tf.n_slices, 4096, tf.n_clusters)
    ctx.tpc_track_batch(cl, st)
    assert ctx.tpc_sync_status() == capi.TPC_OK
    fr = capi.Tracks(tf.n_clusters, 1, 4096, tf.n_clusters)
    for bad_len in (0, -5, 32002):
        with pytest.raises(capi.TpcError) as e:
            ctx.tpc_merge_slices(cl, st, bad_len, fr)
        assert e.value.code == capi.TPC_ERR_INVALID_ARG
    nolabel = capi.Tracks(tf.n_clusters, 1, 4096, tf.n_clusters)
    nolabel.label = None
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_merge_slices(cl, st, tf.slice_len, nolabel)
    assert e.value.code == capi.TPC_ERR_INVALID_ARG
    # room for 5 frame tracks only: the sentinel after trk_off[5] stays untouched
    small = capi.Tracks(tf.n_clusters, 1, 5, tf.n_clusters)
    small.trk_off = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    ctx.tpc_merge_slices(cl, st, tf.slice_len, small)
    assert ctx.tpc_sync_status() == capi.TPC_ERR_CAPACITY
    assert small.trk_off[6:].cpu().tolist() == [-7, -7]
    ctx.tpc_merge_slices(cl, st, tf.slice_len, fr)
    assert ctx.tpc_sync_status() == capi.TPC_OK
    assert int(fr.n_tracks.item()) > 50
    ctx.close()


def _bad_offsets(n, nbins, kind):
    """Bin offsets that break the layout rule 0 = bo[0] <= ... <= bo[nbins] = n."""
    bo = np.linspace(0, n, nbins + 1).astype(np.int64)
    if kind == "past_end":          # the offsets run past the clusters (a write past the grid)
        bo = np.linspace(0, 5 * n, nbins + 1).astype(np.int64)
    elif kind == "decreasing":
        bo[nbins // 2] = bo[nbins // 2 - 1] - 3
    elif kind == "short":           # clusters after the last bin
        bo[-1] = n - 100
    elif kind == "negative":
        bo[1] = -50
    return bo.astype(np.int32)


@pytest.mark.parametrize("kind", ["past_end", "decreasing", "short", "negative"])
def test_malformed_bin_offsets_are_a_bounds_error_with_nothing_written_outside(kind):
    """Bin offsets outside [0, n_clusters], decreasing, or not ending at n_clusters: every call
    reports TPC_ERR_BOUNDS, finds no track, leaves the bytes after its outputs untouched, and the
    context works normally afterwards."""
    ev = _events.event("c1")
    n, nbins = ev.n_clusters, 36 * 159
    ctx = _gpu.make_context(n, 1)
    bad = capi.Clusters.from_numpy(ev.pad_fp, ev.time_fp, _bad_offsets(n, nbins, kind), 1)
    tail = 4096
    for batch in (False, True):
        tr = capi.Tracks(n, 1, 1024, n)
        outer = {}
        for name, m, dt in [("label", n, torch.int32), ("trk_off", 1025, torch.int32), ("trk_hits", n, torch.int32)]:
            big = torch.full((m + tail,), 12345, dtype=dt, device="cuda")
            setattr(tr, name, big[:m])
            outer[name] = (big, m)
        if batch:
            ctx.tpc_track_batch(bad, tr)
        else:
            ctx.tpc_track_event(bad, tr)
        assert ctx.tpc_sync_status() == capi.TPC_ERR_BOUNDS
        assert int(tr.n_tracks.item()) == 0
        assert bool((tr.label == -1).all())
        for name, (big, m) in outer.items():
            assert bool((big[m:] == 12345).all()), name
    good = _gpu.run(ctx, _gpu.clusters_of(ev))
    assert good["n_tracks"] > 50
    # the refit of those tracks against the malformed offsets: also a bounds error
    s = torch.empty(1, dtype=torch.float64, device="cuda")
    th = torch.tensor(synth.theta_nominal(), dtype=torch.float64, device="cuda")
    ctx.tpc_refit_grad(bad, good["tracks_obj"], th, s, None)
    assert ctx.tpc_sync_status() == capi.TPC_ERR_BOUNDS
    # the matching steps that look up the first hit's sector in the offsets: bounds errors too, and
    # nothing written past their outputs
    nt = good["n_tracks"]
    pair = torch.full((nt + tail,), 777, dtype=torch.int32, device="cuda")
    ctx.tpc_looper_pairs(bad, good["tracks_obj"], pair[:nt])
    assert ctx.tpc_sync_status() == capi.TPC_ERR_BOUNDS
    assert bool((pair[nt:] == 777).all())
    its = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    mt = torch.full((nt + tail,), 777, dtype=torch.int32, device="cuda")
    mi = torch.full((4 + tail,), 777, dtype=torch.int32, device="cuda")
    ctx.tpc_its_match(bad, good["tracks_obj"], its, mt[:nt], mi[:4])
    assert ctx.tpc_sync_status() == capi.TPC_ERR_BOUNDS
    assert bool((mt[nt:] == 777).all()) and bool((mi[4:] == 777).all())
    ctx.close()
