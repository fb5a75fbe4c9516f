"""Pins of the oracle's looper-leg pairing (segment merging of the paper's section 3 applied to the two
legs of a low-pT looper) against facts outside the oracle: circles and far-point z built from first
principles, the generator's exact helices (centre, radius, z at the far point, which leg goes out),
the window edges of every gate, the mutual-best rule, and the truth of the pairs on a looper-rich
event.  No GPU."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1712_09434_gb300 import synth
from tests import _events

KB = -0.299792458e-2 * 0.5          # curvature per q/pT at Bz = 0.5 T (1/cm per c/GeV)
LC = O.loop_constants()


def _alpha(k):
    return math.radians(((k % 18) + 0.5) * 20.0)


def _state_on_circle(cx, cy, R, psi, ccw, k, z, tl):
    """Fit state (par, xref) of a track at the point of angle psi on the circle (centre (cx, cy),
    radius R, global frame) moving counter-clockwise (ccw) or clockwise, in the frame of sector k,
    written from the geometry: position, unit tangent and signed curvature."""
    px, py = cx + R * math.cos(psi), cy + R * math.sin(psi)
    tx, ty = (-math.sin(psi), math.cos(psi)) if ccw else (math.sin(psi), -math.cos(psi))
    a = _alpha(k)
    xl = px * math.cos(a) + py * math.sin(a)
    yl = -px * math.sin(a) + py * math.cos(a)
    txl = tx * math.cos(a) + ty * math.sin(a)
    tyl = -tx * math.sin(a) + ty * math.cos(a)
    assert txl > 0.0, "the fit direction points outwards in the sector frame"
    C = (1.0 if ccw else -1.0) / R
    return np.array([yl, z, tyl, tl, C / KB]), xl


def _far_turn(cx, cy, psi, ccw):
    """Turning angle from the point at angle psi to the far point of the circle (angle of the centre
    seen from the beam), along the direction of motion."""
    phi_f = math.atan2(cy, cx)
    d = (phi_f - psi) if ccw else (psi - phi_f)
    return d % (2.0 * math.pi)


def _legs(cx, cy, R, tl, z_far, k_out=None, k_ret=None, dpsi=1.0):
    """Two legs of one looper circle: the point of each leg dpsi before the far point on either side,
    both moving towards it, each leg's z chosen so that it reaches z_far at the far point with its own
    tan lambda (the returning leg's is the opposite of the outgoing one)."""
    phi_f = math.atan2(cy, cx)
    # outgoing leg moving counter-clockwise towards the far point, returning leg clockwise
    psi_a, psi_b = phi_f - dpsi, phi_f + dpsi
    legs = []
    for psi, ccw, t, kk in ((psi_a, True, tl, k_out), (psi_b, False, -tl, k_ret)):
        px, py = cx + R * math.cos(psi), cy + R * math.sin(psi)
        k = kk if kk is not None else int(math.floor((math.atan2(py, px) % (2 * math.pi)) / math.radians(20.0))) % 18
        if z_far < 0:
            k += 18
        z = z_far - t * R * _far_turn(cx, cy, psi, ccw)
        par, xref = _state_on_circle(cx, cy, R, psi, ccw, k, z, t)
        legs.append((par, xref, k))
    return legs


def _pairs(legs, events=None):
    par = np.array([l[0] for l in legs])
    xref = np.array([l[1] for l in legs])
    sec = np.array([l[2] for l in legs], np.int32)
    f = dict(par=par, xref=xref, ndf=np.full(len(legs), 20, np.int32))
    return O.looper_pairs(f, sec, events)


def test_constants():
    assert LC == {"RMAX": 130.0, "CMIN": 40.0, "DC": 5.0, "DR": 5.0, "DZ": 8.0, "DTL": 0.05}


@pytest.mark.parametrize("seed", range(12))
def test_circle_of_constructed_states(seed):
    """Centre, radius, curvature sign and far-point z of states written from the circle geometry,
    both directions of motion, any sector and side."""
    rng = np.random.default_rng(seed)
    phi_c = rng.uniform(0, 2 * math.pi)
    R = rng.uniform(45.0, 120.0)
    rc = R + rng.uniform(-3.0, 3.0)
    cx, cy = rc * math.cos(phi_c), rc * math.sin(phi_c)
    tl = rng.uniform(-1.0, 1.0)
    for (par, xref, k), ccw in zip(_legs(cx, cy, R, tl, 60.0 if tl > 0 else -60.0, dpsi=rng.uniform(0.3, 1.2)),
                                   (True, False)):
        ok, ocx, ocy, oR, zap, otl, sgn = O.loop_circle(par, xref, k)
        assert ok
        assert abs(ocx - cx) < 1e-9 and abs(ocy - cy) < 1e-9 and abs(oR - R) < 1e-9
        assert sgn == (1.0 if ccw else -1.0) and otl == par[3]
        assert abs(zap - (60.0 if tl > 0 else -60.0)) < 1e-9


LOOPER_SEEDS = (5, 7, 8, 11, 15, 18, 19, 21, 28, 39, 45, 47, 48)


@pytest.mark.parametrize("seed", LOOPER_SEEDS)
def test_exact_looper_legs_are_paired(seed):
    """One looper from the vertex, unsmeared clusters (1/128 cm quantisation only): the tracker finds
    its two legs, the oracle pairs them, the outgoing leg is the one whose clusters come first along
    the particle's path, and each leg's circle is the generator's: centre (-sin phi0, cos phi0)/C,
    radius 1/|C|, z at the far point tan lambda * pi / |C| (half a turn from the vertex)."""
    ev = synth.make_event(synth.EventConfig(n_tracks=1, noise_frac=0.0, looper_frac=1.0, seed=seed, smear=0.0))
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    off, hits = o["trk_off"], o["trk_hits"]
    assert len(off) == 3
    sec = ev.sector[hits[off[:-1]]].astype(np.int32)
    pair, leg, D = O.looper_pairs(f, sec)
    assert list(pair) == [1, 0]
    s_mean = [ev.true_s[hits[a:b]].mean() for a, b in zip(off[:-1], off[1:])]
    out = int(np.argmin(s_mean))
    assert leg[out] == 1 and leg[1 - out] == 2
    C = KB * ev.trk_q[0] / ev.trk_pt[0]
    phi0, tl = ev.trk_phi0[0], math.sinh(ev.trk_eta[0])
    cx, cy, R = -math.sin(phi0) / C, math.cos(phi0) / C, 1.0 / abs(C)
    for t in range(2):
        ok, ocx, ocy, oR, zap, otl, sgn = O.loop_circle(f["par"][t], f["xref"][t], int(sec[t]))
        assert ok
        assert math.hypot(ocx - cx, ocy - cy) < 0.3 and abs(oR - R) < 0.3, (ocx, ocy, oR, cx, cy, R)
        assert abs(zap - tl * math.pi * R) < 0.5
        # the outgoing leg turns like the particle, the returning leg (fitted outwards) the other way
        assert sgn == (np.sign(C) if t == out else -np.sign(C))
        assert np.sign(otl) == (np.sign(tl) if t == out else -np.sign(tl))


def _base(R=80.0, phi_c=0.7, tl=0.4, z_far=90.0):
    return R * math.cos(phi_c), R * math.sin(phi_c), R, tl, z_far


def test_two_legs_of_one_circle_are_paired():
    cx, cy, R, tl, zf = _base()
    pair, leg, D = _pairs(_legs(cx, cy, R, tl, zf))
    assert list(pair) == [1, 0] and list(leg) == [1, 2] and D[0] < 1e-12


@pytest.mark.parametrize("shift,paired", [(4.99, True), (5.01, False)])
def test_centre_window_edge(shift, paired):
    """The returning leg's circle moved by `shift` cm (its radius kept) perpendicular to the line from
    the beam, so that only the centre gate can fail; the far-point z follows the moved circle."""
    cx, cy, R, tl, zf = _base()
    a = _legs(cx, cy, R, tl, zf)[0]
    u = (-cy / math.hypot(cx, cy), cx / math.hypot(cx, cy))
    b = _legs(cx + shift * u[0], cy + shift * u[1], R, tl, zf)[1]
    pair, _, _ = _pairs([a, b])
    assert (pair[0] == 1) == paired and (pair[1] == 0) == paired


@pytest.mark.parametrize("dR,paired", [(4.99, True), (5.01, False), (-4.99, True), (-5.01, False)])
def test_radius_window_edge(dR, paired):
    """Radius of the returning leg changed by dR with its centre kept."""
    cx, cy, R, tl, zf = _base()
    a = _legs(cx, cy, R, tl, zf)[0]
    b = _legs(cx, cy, R + dR, tl, zf)[1]
    assert (_pairs([a, b])[0][0] == 1) == paired


@pytest.mark.parametrize("dz,paired", [(7.99, True), (8.01, False), (-7.99, True), (-8.01, False)])
def test_far_point_z_window_edge(dz, paired):
    cx, cy, R, tl, zf = _base()
    a = _legs(cx, cy, R, tl, zf)[0]
    b = _legs(cx, cy, R, tl, zf + dz)[1]
    assert (_pairs([a, b])[0][0] == 1) == paired


@pytest.mark.parametrize("dtl,paired", [(0.0499, True), (0.0501, False), (-0.0499, True), (-0.0501, False)])
def test_tan_lambda_window_edge(dtl, paired):
    """The returning leg's tan lambda is -(tan lambda + dtl); its z is set so that it still reaches the
    same far-point z."""
    cx, cy, R, tl, zf = _base()
    a = _legs(cx, cy, R, tl, zf)[0]
    b = _legs(cx, cy, R, tl + dtl, zf)[1]
    assert (_pairs([a, b])[0][0] == 1) == paired


def test_same_curvature_sign_or_other_event_is_not_paired():
    cx, cy, R, tl, zf = _base()
    a, b = _legs(cx, cy, R, tl, zf)
    pair, _, _ = _pairs([a, b], events=np.array([0, 1], np.int32))
    assert list(pair) == [-1, -1]
    # the outgoing leg twice: same circle, same curvature sign
    pair, _, _ = _pairs([a, a])
    assert list(pair) == [-1, -1]


@pytest.mark.parametrize("R,paired", [(129.9, True), (130.1, False)])
def test_radius_limit(R, paired):
    cx, cy, R_, tl, zf = _base(R=R, phi_c=0.7, tl=0.2, z_far=100.0)
    assert (_pairs(_legs(cx, cy, R_, tl, zf))[0][0] == 1) == paired


@pytest.mark.parametrize("rc,paired", [(40.1, True), (39.9, False)])
def test_centre_distance_limit(rc, paired):
    """A circle of radius 60 whose centre lies rc from the beam."""
    R, phi_c = 60.0, 2.0
    cx, cy = rc * math.cos(phi_c), rc * math.sin(phi_c)
    assert (_pairs(_legs(cx, cy, R, 0.3, 50.0, dpsi=0.5))[0][0] == 1) == paired


def test_mutual_best():
    """A (outgoing) has two candidate partners B and C; B is nearer. Without a fourth leg, A and B
    pair and C is left. A fourth leg D (outgoing, on B's circle exactly) is nearer to both B and C
    than A is: B pairs with D, and A, whose best (B) chose D, stays unpaired."""
    cx, cy, R, tl, zf = _base()
    A = _legs(cx, cy, R, tl, zf)[0]
    B = _legs(cx, cy, R + 1.0, tl, zf)[1]
    Cl = _legs(cx, cy, R + 2.0, tl, zf)[1]
    pair, _, _ = _pairs([A, B, Cl])
    assert list(pair) == [1, 0, -1]
    Dl = _legs(cx, cy, R + 1.0, tl, zf)[0]
    pair, _, _ = _pairs([A, B, Cl, Dl])
    assert pair[1] == 3 and pair[3] == 1
    # one round of mutual best: A's best (B) and C's best (D) are taken, so A and C stay unpaired
    assert pair[0] == -1 and pair[2] == -1


def test_looper_rich_event_pairs_are_true():
    """A smeared event of 3,000 particles, 30 % of them loopers: more than 98 % of the pairs join two
    legs of one particle (measured: all 616), and the outgoing leg is the one whose clusters come first
    along the path wherever |tan lambda| > 0.01."""
    ev = synth.make_event(synth.EventConfig(n_tracks=3000, noise_frac=0.1, looper_frac=0.3, seed=1011))
    o = O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)
    f = O.fit(ev.pad_fp, ev.time_fp, ev.bin_off, o["trk_off"], o["trk_hits"])
    off, hits = o["trk_off"], o["trk_hits"]
    sec = ev.sector[hits[off[:-1]]].astype(np.int32)
    pair, leg, D = O.looper_pairs(f, sec)
    m = pair >= 0
    lead = np.array([np.bincount(np.maximum(ev.mc_track[hits[a:b]], 0)).argmax() for a, b in zip(off[:-1], off[1:])])
    s_med = np.array([np.nanmedian(ev.true_s[hits[a:b]]) for a, b in zip(off[:-1], off[1:])])
    print("pairs", m.sum() // 2, "same particle", (lead[m] == lead[pair[m]]).mean())
    assert m.sum() // 2 > 300
    assert (lead[m] == lead[pair[m]]).mean() > 0.98
    # the direction is decided by the sign of tan lambda: only where it is above the fit's resolution
    same = m & (lead == lead[np.maximum(pair, 0)]) & (np.abs(f["par"][:, 3]) > 0.01)
    first = s_med < s_med[np.maximum(pair, 0)]
    assert same.sum() > 500
    assert np.all((leg[same] == 1) == first[same])
    assert np.all(pair[pair[m]] == np.nonzero(m)[0])


def test_same_curvature_sign_alone_blocks_the_pair():
    """A second leg on the same circle moving the same way round (same curvature sign), with the
    opposite tan lambda and the same far-point z, so that every other gate passes."""
    cx, cy, R, tl, zf = _base()
    a = _legs(cx, cy, R, tl, zf)[0]
    phi_f = math.atan2(cy, cx)
    psi = phi_f - 0.6
    z = zf + tl * R * _far_turn(cx, cy, psi, True)
    k = int(math.floor((math.atan2(cy + R * math.sin(psi), cx + R * math.cos(psi)) % (2 * math.pi)) / math.radians(20.0)))
    par, xref = _state_on_circle(cx, cy, R, psi, True, k % 18, z, -tl)
    b = (par, xref, k % 18)
    assert O.loop_circle(par, xref, k % 18)[5] == -tl
    assert abs(O.loop_circle(par, xref, k % 18)[4] - zf) < 1e-9
    assert list(_pairs([a, b])[0]) == [-1, -1]


def test_score_counts_the_far_point_z():
    """Two returning legs on A's circle, one 1 cm and one 2 cm off in far-point z: A takes the nearer,
    whichever comes first in the list."""
    cx, cy, R, tl, zf = _base()
    A = _legs(cx, cy, R, tl, zf)[0]
    near = _legs(cx, cy, R, tl, zf + 1.0)[1]
    far = _legs(cx, cy, R, tl, zf + 2.0)[1]
    assert _pairs([A, far, near])[0][0] == 2
    assert _pairs([A, near, far])[0][0] == 1
