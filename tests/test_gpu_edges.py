"""CUDA path against the oracle on hand-constructed events that sit on the edges of the following
rule (the constructions of the oracle's edge pins, run through the whole tracking): every integer
stage must be bit-exact, including ties between equally distant clusters in two Z slabs of the
grid and a search window that spans three slabs."""
import types

import numpy as np
import pytest

from oracle import oracle as O
from tests import _gpu
from tests._constructed import edge_events
from tests.test_gpu_parity import _compare_stages

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = _gpu.make_context(200_000, 4)
    yield c
    c.close()


def test_edge_events_every_integer_stage_bit_exact(ctx):
    evs = edge_events()
    assert len(evs) >= 2
    for pad, tim, bin_off, _ in evs:
        ev = types.SimpleNamespace(pad_fp=pad, time_fp=tim, bin_off=bin_off, n_clusters=len(pad))
        o = O.track_event(pad, tim, bin_off, keep_stages=True)
        assert len(o["trk_off"]) > 10
        g = _gpu.run(ctx, _gpu.clusters_of(ev), stages=True)
        _compare_stages(ev, o, g)
        gb = _gpu.run(ctx, _gpu.clusters_of(ev), batch=True)
        np.testing.assert_array_equal(gb["trk_hits"], o["trk_hits"])
