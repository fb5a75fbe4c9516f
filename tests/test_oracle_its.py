"""Pins of the oracle's TPC-ITS matching (the drift calibration of the paper's sections 2.1 and 6
matches TPC tracks to inner-tracker tracks) against facts outside the oracle: exact tracks meet
their own particle's ITS track, the match chi2 of true pairs follows the chi2 distribution of its
four degrees of freedom, the z window edge, fakes, and the mutual-best rule.  No GPU."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_09434_gb300 import synth
from tests import _events


def _tracks_and_fit(ev):
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    sec = ev.sector[o["trk_hits"][o["trk_off"][:-1]]].astype(np.int32)
    lead = np.array([np.bincount(np.maximum(ev.mc_track[o["trk_hits"][a:b]], 0)).argmax()
                     for a, b in zip(o["trk_off"][:-1], o["trk_off"][1:])], np.int64)
    return o, f, sec, lead


@pytest.fixture(scope="module")
def exact():
    ev = _events.noise_free(n_tracks=400, seed=21)
    o, f, sec, lead = _tracks_and_fit(ev)
    its, part = synth.its_tracks(ev, eff=1.0, fake_frac=0.0, smear=False)
    return ev, o, f, sec, lead, its, part


def test_exact_tracks_match_their_own_particle(exact):
    """Unsmeared clusters and exact ITS tracks: every matched TPC track is matched to the ITS track
    of its own particle, most tracks are matched, and the chi2 is at the quantisation level."""
    ev, o, f, sec, lead, its, part = exact
    mt, mi, c2 = O.its_match(f, sec, its)
    m = mt >= 0
    assert m.sum() > 0.8 * len(mt)
    assert np.all(part[mt[m]] == lead[m])
    assert np.all(mi[mt[m]] == np.nonzero(m)[0])
    assert np.median(c2[m]) < 0.1


@pytest.mark.parametrize("dz,matched", [(1.98, True), (2.02, False), (-1.98, True), (-2.02, False)])
def test_z_window_is_two_cm(exact, dz, matched):
    """z at the vertex is only windowed (|dz| <= 2 cm, the drift calibration is unknown at matching
    time): exact ITS tracks moved by 1.98 cm still match, by 2.02 cm none do, for the tracks of at
    least 30 hits (fitted on unsmeared clusters, their extrapolated z is within 0.01 cm of 0)."""
    ev, o, f, sec, lead, its, part = exact
    moved = its.copy()
    moved[:, 1] += dz
    mt, _, _ = O.its_match(f, sec, moved)
    long_ = np.diff(o["trk_off"]) >= 30          # short tracks extrapolate to the vertex less well
    n = (mt[long_] >= 0).sum()
    assert (n > 0.8 * long_.sum()) if matched else n == 0


def test_match_chi2_follows_four_degrees_of_freedom():
    """Smeared clusters and ITS tracks at the nominal calibration: more than 99.9 % of the matches
    join the right particle, none takes a fake, and the chi2 of the true pairs has the mean (4) and
    the median (3.36) of a chi2 with four degrees of freedom (the gate of 100 truncates nothing of
    it)."""
    ev = _events.event("c2")
    o, f, sec, lead = _tracks_and_fit(ev)
    its, part = synth.its_tracks(ev)
    mt, mi, c2 = O.its_match(f, sec, its)
    m = mt >= 0
    right = part[mt[m]] == lead[m]
    assert right.mean() > 0.999
    assert (part[mt[m]] < 0).sum() == 0
    c = c2[m][right]
    n = len(c)
    assert n > 3000
    assert abs(c.mean() - 4.0) < 3 * np.sqrt(8.0 / n) + 0.05, c.mean()
    assert abs(np.median(c) - 3.357) < 0.15, np.median(c)


def test_fake_only_list_gives_few_matches():
    """An ITS list of fakes only (random azimuth, z0 ~ N(0, 5 cm)): almost no TPC track matches."""
    ev = _events.event("c2")
    o, f, sec, lead = _tracks_and_fit(ev)
    its, part = synth.its_tracks(ev, eff=0.0, fake_frac=0.0)
    rng = np.random.default_rng(5)
    real, _ = synth.its_tracks(ev)
    fakes = real.copy()
    fakes[:, 0] = rng.uniform(0, 2 * np.pi, len(fakes))
    fakes[:, 1] = rng.normal(0, 5.0, len(fakes))
    mt, _, _ = O.its_match(f, sec, fakes)
    assert (mt >= 0).mean() < 0.01


def test_mutual_best_prefers_the_closer_of_two_copies(exact):
    """Each exact ITS track duplicated with q/pT off by 2 sigma: the exact copy is matched and the
    shifted copy is left unmatched."""
    ev, o, f, sec, lead, its, part = exact
    shifted = its.copy()
    shifted[:, 3] += 2.0 * shifted[:, 7]
    both = np.concatenate([its, shifted])
    mt, mi, _ = O.its_match(f, sec, both)
    m = mt >= 0
    assert m.sum() > 0.8 * len(mt)
    assert np.all(mt[m] < len(its))
    assert np.all(mi[len(its):] == -1)
