"""Stored fixtures under tests/golden/: two hand-worked examples (neighbour finding, helix steps;
the derivations are in the files) and the oracle's output on the single-sector event, written by
tests/golden/make_oracle_regression.py from the oracle alone."""
import hashlib
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_09434_gb300 import synth
from tests import _events

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name, tag):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if line and line[0] == tag:
            out.append(line[1:])
    return out


def links_example():
    cl = np.array([[int(v) for v in r] for r in _rows("links_worked_example.txt", "cluster")])
    assert np.all(cl[:, 0] == np.arange(len(cl)))
    row, pad, tim = cl[:, 1], cl[:, 2], cl[:, 3]
    b = row                                   # sector 0
    bin_off = np.searchsorted(b, np.arange(synth.N_SECTORS * synth.N_ROWS + 1)).astype(np.int32)
    up = -np.ones(len(cl), np.int32)
    down = -np.ones(len(cl), np.int32)
    for c, u, d in (map(int, r) for r in _rows("links_worked_example.txt", "link")):
        up[c], down[c] = u, d
    return pad.astype(np.int16), tim.astype(np.uint16), bin_off, up, down


def test_links_worked_example():
    pad, tim, bin_off, up, down = links_example()
    u, d = O.links(pad, tim, bin_off)
    np.testing.assert_array_equal(u, up)
    np.testing.assert_array_equal(d, down)


def test_helix_worked_example():
    for r in _rows("helix_worked_example.txt", "case"):
        a = [float(v) for v in r if v != "|"]
        x1, y1, z1, snp1, tl, qpt, x2, y2, z2, snp2, arc = a
        ok, p, F = O.propagate(x1, np.array([y1, z1, snp1, tl, qpt]), x2)
        assert ok
        np.testing.assert_allclose(p, [y2, z2, snp2, tl, qpt], rtol=1e-12, atol=1e-11)


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a.astype("<i4")).tobytes()).hexdigest()


def _regression():
    kv = {r[0]: r[1] for r in (l.split() for l in open(os.path.join(GOLDEN, "oracle_c1_regression.txt"))
                               if l.strip() and not l.startswith("#") and not l.startswith("track"))}
    tr = np.array([[float(v) for v in r] for r in _rows("oracle_c1_regression.txt", "track")])
    return kv, tr


def test_oracle_reproduces_its_stored_single_sector_output():
    kv, tr = _regression()
    ev = _events.event("c1")
    assert ev.n_clusters == int(kv["n_clusters"])
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    assert _digest(o["trk_off"]) == kv["trk_off_sha256"]
    assert _digest(o["trk_hits"]) == kv["trk_hits_sha256"]
    assert _digest(o["label"]) == kv["label_sha256"]
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    np.testing.assert_array_equal(f["ndf"], tr[:, 4].astype(int))
    np.testing.assert_allclose(f["chi2"], tr[:, 5], rtol=1e-9)
    np.testing.assert_allclose(f["par"], tr[:, 6:11], rtol=1e-9, atol=1e-12)


@pytest.mark.gpu
def test_cuda_links_worked_example():
    from tests import _gpu
    pad, tim, bin_off, up, down = links_example()
    ctx = _gpu.make_context(64)
    from paper_1712_09434_gb300 import capi
    g = _gpu.run(ctx, capi.Clusters.from_numpy(pad, tim, bin_off, 1), stages=True)
    ctx.close()
    np.testing.assert_array_equal(g["up"], up)
    np.testing.assert_array_equal(g["down"], down)


@pytest.mark.gpu
def test_cuda_path_reproduces_the_stored_oracle_output():
    """Bit-exact tracks and FP32 refit parameters against the stored FP64 values (no oracle run)."""
    from tests import _gpu
    kv, tr = _regression()
    ev = _events.event("c1")
    ctx = _gpu.make_context(ev.n_clusters)
    g = _gpu.run(ctx, _gpu.clusters_of(ev))
    ctx.close()
    assert _digest(g["trk_off"]) == kv["trk_off_sha256"]
    assert _digest(g["trk_hits"]) == kv["trk_hits_sha256"]
    assert _digest(g["label"]) == kv["label_sha256"]
    np.testing.assert_array_equal(g["ndf"], tr[:, 4].astype(int))
    good = tr[:, 5] < 5 * np.maximum(tr[:, 4], 1)
    scale = np.maximum(np.maximum(np.abs(tr[:, 6:11]), [1.0, 1.0, 1e-2, 1e-2, 1e-2]), tr[:, 11:16])
    err = np.abs(g["par"] - tr[:, 6:11]) / scale
    assert err[good].max() < 1e-4, err[good].max(axis=0)
