"""tpc_links_noalloc: neighbour finding for callers that cannot allocate device memory.

Code recorded into a CUDA graph by stream capture, a plug-in inside a framework that owns the
GPU's memory, or real-time code that allocates only at start-up cannot let the library call
cudaMalloc.  This entry point runs the grid and neighbour-finding kernels of the tracking path
with their scratch in a static device array.  Here it is called through the C ABI twice in a row
(a large event, then a small one, so that leftovers of the first call in the shared array would
show) and must reproduce, bit for bit, the links the context-based tracking call computes.  This
file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from paper_1712_09434_gb300 import capi, synth
from tests import _events, _gpu

pytestmark = pytest.mark.gpu


def _reference_links(ev):
    ctx = _gpu.make_context(ev.n_clusters, 1)
    g = _gpu.run(ctx, _gpu.clusters_of(ev), stages=True)
    ctx.close()
    return g["up"], g["down"]


def _noalloc_links(ev):
    cl = _gpu.clusters_of(ev)
    n = max(ev.n_clusters, 1)
    up = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    down = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = capi.tpc_links_noalloc(capi.default_geometry(), cl, up, down, status)
    assert rc == capi.TPC_OK, capi.lib().tpc_strerror(rc)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return up.cpu().numpy()[:ev.n_clusters], down.cpu().numpy()[:ev.n_clusters]


def test_noalloc_links_equal_the_tracking_path_on_two_calls_in_a_row():
    big = _events.event("c2")          # 914k clusters: most of the static scratch
    small = _events.event("c1")        # then a small event over the leftovers
    assert big.n_clusters <= capi.TPC_NOALLOC_MAX_CLUSTERS
    for ev in (big, small):
        ref_up, ref_down = _reference_links(ev)
        up, down = _noalloc_links(ev)
        np.testing.assert_array_equal(up, ref_up)
        np.testing.assert_array_equal(down, ref_down)


def test_noalloc_rejects_inputs_beyond_the_static_scratch():
    ev = _events.event("c1")
    cl = _gpu.clusters_of(ev)
    cl.n_clusters = capi.TPC_NOALLOC_MAX_CLUSTERS + 1      # rejected before any device access
    up = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = capi.tpc_links_noalloc(capi.default_geometry(), cl, up, up)
    assert rc == capi.TPC_ERR_CAPACITY
    batch = synth.concat_events([ev] * 3)                   # 3 * 5724 bins > TPC_NOALLOC_MAX_BINS
    cb = _gpu.clusters_of(batch, 3)
    rc = capi.tpc_links_noalloc(capi.default_geometry(), cb, up, up)
    assert rc == capi.TPC_ERR_CAPACITY


def test_noalloc_malformed_bin_offsets_are_a_bounds_error():
    """Offsets running past the clusters would index past the static scratch: the call reports
    TPC_ERR_BOUNDS in its status word, makes no link, and the next call works normally."""
    ev = _events.event("c1")
    n, nbins = ev.n_clusters, 36 * 159
    bo = np.linspace(0, 5 * n, nbins + 1).astype(np.int32)
    cl = capi.Clusters.from_numpy(ev.pad_fp, ev.time_fp, bo, 1)
    tail = 1024
    up = torch.full((n + tail,), -7, dtype=torch.int32, device="cuda")
    down = torch.full((n + tail,), -7, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = capi.tpc_links_noalloc(capi.default_geometry(), cl, up[:n], down[:n], status)
    assert rc == capi.TPC_OK
    torch.cuda.synchronize()
    assert int(status.item()) & 4                        # the library's bounds bit
    assert bool((up[:n] == -1).all()) and bool((down[:n] == -1).all())
    assert bool((up[n:] == -7).all()) and bool((down[n:] == -7).all())
    ref_up, ref_down = _reference_links(ev)
    up2, down2 = _noalloc_links(ev)
    np.testing.assert_array_equal(up2, ref_up)
    np.testing.assert_array_equal(down2, ref_down)
