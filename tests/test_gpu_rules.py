"""CUDA path against the oracle with the rules for inefficient data switched on (tpc_set_rules:
links across one empty row, the gap merge inside a sector): every integer stage bit-exact on the
named events, on an event with dead pad rows and dropped clusters, on hand-built edge events of
both rules, and in the batched graph form."""
import types

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_09434_gb300 import capi, synth
from tests import _events, _gpu
from tests._constructed import rule_events
from tests.test_gpu_parity import _compare_stages, _compare_tracks

pytestmark = pytest.mark.gpu

ALL = capi.TPC_RULE_SKIP_ROW | capi.TPC_RULE_GAP_MERGE


@pytest.fixture(scope="module")
def ctx():
    c = _gpu.make_context(4_200_000, 64)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ineff():
    return synth.make_event(synth.inefficient_central())


def _run(ctx, ev, rules, n_events=1, **kw):
    ctx.tpc_set_rules(rules)
    try:
        return _gpu.run(ctx, _gpu.clusters_of(ev, n_events), n_events=n_events, **kw)
    finally:
        ctx.tpc_set_rules(0)


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_rules_every_integer_stage_bit_exact(ctx, name):
    ev = _events.event(name)
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off, keep_stages=True, rules=ALL)
    g = _run(ctx, ev, ALL, stages=True)
    _compare_stages(ev, o, g)


@pytest.mark.parametrize("rules", [0, capi.TPC_RULE_SKIP_ROW, capi.TPC_RULE_GAP_MERGE, ALL])
def test_inefficient_event_bit_exact_under_every_rule_set(ctx, ineff, rules):
    """20,000 tracks with dead rows 60-61 and 100-111 and 5 % of the crossings dropped."""
    o = O.track_event(ineff.pad_fp, ineff.time_fp, ineff.bin_off, keep_stages=True, rules=rules)
    g = _run(ctx, ineff, rules, stages=True)
    _compare_stages(ineff, o, g)
    eff, n, fake = synth.track_quality(ineff, g["trk_off"], g["trk_hits"])
    print("rules %d: %d tracks, found-whole efficiency %.3f of %d particles, fake fraction %.3f" % (
        rules, g["n_tracks"], eff, n, fake))
    if rules & capi.TPC_RULE_GAP_MERGE:
        assert eff > 0.5


def test_rule_edge_events_bit_exact(ctx):
    for pad, tim, bin_off, _ in rule_events():
        ev = types.SimpleNamespace(pad_fp=pad, time_fp=tim, bin_off=bin_off, n_clusters=len(pad))
        o = O.track_event(pad, tim, bin_off, keep_stages=True, rules=ALL)
        g = _run(ctx, ev, ALL, stages=True)
        _compare_stages(ev, o, g)
        assert (o["gap_next"] >= 0).sum() >= 4             # the gap constructions are joined


def test_rules_in_the_batch_graph_equal_the_plain_form(ctx):
    cfgs = synth.batch_configs(n_events=4, seed0=2300)
    for c in cfgs:
        c.n_tracks = min(c.n_tracks, 3000)
        c.dead_rows = ((100, 111),)
        c.drop_frac = 0.05
    evs = [synth.make_event(c) for c in cfgs]
    b = synth.concat_events(evs)
    gb = _run(ctx, b, ALL, n_events=b.n_events, batch=True)
    for e, ev in enumerate(evs):
        o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off, rules=ALL)
        t0, t1 = gb["ev_trk_off"][e], gb["ev_trk_off"][e + 1]
        off = gb["trk_off"][t0:t1 + 1]
        np.testing.assert_array_equal(off - off[0], o["trk_off"])
        np.testing.assert_array_equal(gb["trk_hits"][off[0]:off[-1]] - b.ev_off[e], o["trk_hits"])


def test_unknown_rule_bits_are_rejected(ctx):
    with pytest.raises(capi.TpcError) as e:
        ctx.tpc_set_rules(4)
    assert e.value.code == capi.TPC_ERR_INVALID_ARG
