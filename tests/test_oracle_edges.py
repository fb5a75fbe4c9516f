"""Edge pins of the oracle's integer track finding on hand-constructed inputs (no GPU).

Each test names the reading it pins (R-5 .. R-9 of the design notes, the readings of the paper's
section 3: CA seeding, Kalman following, selection, sector merging) and sits exactly on the edge
of one rule, so that an off-by-one, a '<' for a '<=', a wrong growth of the search radius, a
dropped stop condition or a wrong tie-break fails here:

  R-7 following: at most 7 consecutive empty rows are bridged; the search radius after k misses
      is 77 + 38 k (a cluster at exactly that distance is taken, one LSB further is not); equal
      distances go to the lower cluster index; the slope limit |v_Y| <= 320 LSB/row, the sector
      acceptance |Y| <= ymax(row) and the drift range 0 <= Z <= 32000 stop the extension.
  R-9 merge: the windows |dY|, |dZ| <= 192, the extrapolation distance |XT - x2| <= 2048, the
      outward direction dx > 0, adjacent sectors of one side only.
  R-10 assembly: a cycle of merge links is cut in front of its smallest segment.
  R-6 / R-7 cleaning and chains: every mutual link is kept and every start of a chain of at least
      five hits gives a chain (brute force on tiny sectors).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests._constructed import Builder, chain_links, ymax

W_F0, W_F1 = 77, 38


def _follow(builder, chain_pts):
    pad, tim, bin_off, index = builder.build()
    hits = [index[p] for p in chain_pts]
    up2 = chain_links(len(pad), hits)
    h, cn = O.follow(pad, tim, bin_off, np.array([hits[0]], np.int32), np.array([len(hits)], np.int32), up2)
    return set(h[0, :cn[0]].tolist()), index


def _y(r):
    return -300 + 7 * r


def _z(r):
    return 5000 + 40 * r


# ---------------------------------------------------------------------------------------------
# R-7 following
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("gap", [0, 1, 6, 7, 8, 9])
def test_following_bridges_at_most_seven_empty_rows_outwards(gap):
    """R-7: the extension stops after M_MISS = 8 consecutive empty rows."""
    b = Builder()
    chain = b.line(0, range(20, 40), -300, 7, 5000, 40)
    beyond = b.line(0, range(40 + gap, 101), -300, 7, 5000, 40)
    cand, index = _follow(b, chain)
    found = {index[p] for p in beyond} & cand
    assert (len(found) == len(beyond)) if gap <= 7 else not found, (gap, len(found))


@pytest.mark.parametrize("gap", [7, 8])
def test_following_bridges_at_most_seven_empty_rows_inwards(gap):
    """R-7 in the descending direction (filter re-initialised at the chain's outer end)."""
    b = Builder()
    chain = b.line(0, range(60, 80), -300, 7, 5000, 40)
    below = b.line(0, range(5, 60 - gap), -300, 7, 5000, 40)
    cand, index = _follow(b, chain)
    found = {index[p] for p in below} & cand
    assert (len(found) == len(below)) if gap <= 7 else not found


def test_following_misses_reset_after_a_found_cluster():
    """R-7: the miss counter restarts at a found cluster: gaps of 7, one cluster, 7 again."""
    b = Builder()
    chain = b.line(0, range(20, 40), -300, 7, 5000, 40)
    rest = b.line(0, [47, 55, 56, 57], -300, 7, 5000, 40)
    cand, index = _follow(b, chain)
    assert {index[p] for p in rest} <= cand


def _pythagorean(w):
    """Integer (a, b) with a^2 + b^2 = w^2, a, b > 0, if any."""
    for a in range(1, w):
        b2 = w * w - a * a
        b = math.isqrt(b2)
        if b * b == b2 and b > 0:
            return a, b
    return None


@pytest.mark.parametrize("k", range(8))
def test_following_search_radius_is_77_plus_38_per_miss(k):
    """R-7: after k consecutive misses a cluster at distance exactly 77 + 38 k from the prediction
    is taken and one at one LSB more is not (along Y, along Z, both signs, and on the diagonal
    where w is the hypotenuse of an integer right triangle)."""
    w = W_F0 + W_F1 * k
    offsets = [((w, 0), True), ((w + 1, 0), False), ((-w, 0), True), ((-w - 1, 0), False),
               ((0, w), True), ((0, w + 1), False), ((0, -w), True), ((0, -w - 1), False)]
    tri = _pythagorean(w)
    if tri is not None:
        a, c = tri
        offsets += [((a, c), True), ((a, c + 1), False), ((-c, a), True), ((-c - 1, a), False)]
    R = 40 + k
    for (dy, dz), inside in offsets:
        b = Builder()
        chain = b.line(0, range(20, 40), -300, 7, 5000, 40)
        b.line(0, range(R + 1, R + 15), -300, 7, 5000, 40)
        p = b.add(0, R, _y(R) + dy, _z(R) + dz)
        cand, index = _follow(b, chain)
        assert (index[p] in cand) == inside, (k, dy, dz, inside)


def test_following_equal_distances_go_to_the_lower_cluster_index():
    """R-7: nearest cluster by (d^2, index); on equal d^2 the lower index (smaller pad, then time)."""
    R = 40
    for (a, b_), want in [(((-30, 0), (30, 0)), 0), (((0, -30), (0, 30)), 0), (((30, 0), (0, -30)), 1),
                          (((-40, 0), (20, 0)), 1)]:
        b = Builder()
        chain = b.line(0, range(20, 40), -300, 7, 5000, 40)
        pa = b.add(0, R, _y(R) + a[0], _z(R) + a[1])
        pb = b.add(0, R, _y(R) + b_[0], _z(R) + b_[1])
        cand, index = _follow(b, chain)
        ia, ib = index[pa], index[pb]
        lower = min(ia, ib)
        if a[0] ** 2 + a[1] ** 2 == b_[0] ** 2 + b_[1] ** 2:
            assert lower in cand and max(ia, ib) not in cand
        else:
            assert ([ia, ib][want] in cand) and ([ia, ib][1 - want] not in cand)


@pytest.mark.parametrize("slope,taken", [(320, True), (321, False), (-320, True), (-321, False)])
def test_following_stops_beyond_the_slope_limit(slope, taken):
    """R-7: the extension stops when |v_Y| > V_MAX = 320 LSB per row."""
    b = Builder()
    y0 = -1500 if slope > 0 else 1500
    chain = [b.add(0, r, y0 + slope * (r - 20), 8000 + 10 * r) for r in range(20, 25)]
    p = b.add(0, 25, y0 + slope * 5, 8250)
    cand, index = _follow(b, chain)
    assert (index[p] in cand) == taken


@pytest.mark.parametrize("side", [1, -1])
@pytest.mark.parametrize("off,taken", [(0, True), (1, False)])
def test_following_stops_outside_the_sector_acceptance(side, off, taken):
    """R-7: a prediction with |Y| > ymax(row) = floor(x_row tan 10 deg / LSB) stops the extension,
    even when a cluster sits exactly there; at |Y| = ymax the cluster is taken."""
    R = 30
    target = side * (ymax(R) + off)
    b = Builder()
    chain = [b.add(0, r, target - side * 40 * (R - r), 6000 + 20 * r) for r in range(20, R)]
    p = b.add(0, R, target, 6000 + 20 * R)
    cand, index = _follow(b, chain)
    assert (index[p] in cand) == taken


@pytest.mark.parametrize("zR,taken", [(0, True), (-1, False), (32000, True), (32001, False)])
def test_following_stops_when_the_prediction_leaves_the_drift_range(zR, taken):
    """R-7: a predicted Z outside [0, round(z_max / LSB)] = [0, 32000] stops the extension."""
    R = 30
    sz = -50 if zR <= 0 else 50
    b = Builder()
    chain = [b.add(0, r, 100 + 5 * r, zR - sz * (R - r)) for r in range(20, R)]
    p = b.add(0, R, 100 + 5 * R, min(max(zR, 0), 32001))
    cand, index = _follow(b, chain)
    assert (index[p] in cand) == taken


# ---------------------------------------------------------------------------------------------
# R-9 merge decision
# ---------------------------------------------------------------------------------------------

C30 = round(math.cos(math.radians(20.0)) * 2 ** 30)
S30 = round(math.sin(math.radians(20.0)) * 2 ** 30)


def _rot(X, Y, sgn):
    """Sector rotation of R-9 by sgn * 20 degrees with Q30 constants and floor shifts."""
    return (X * C30 + sgn * Y * S30) >> 30, (-sgn * X * S30 + Y * C30) >> 30


# outer end of S in sector 0 (LSB): the hit three before the last one and the last hit, r ~ 229 cm
S_END = (29000, 3800, 12000, 29400, 3900, 12100)


def _predicted(s_end, sgn, XT):
    X1, Y1, Z1, X2, Y2, Z2 = s_end
    x1, y1 = _rot(X1, Y1, sgn)
    x2, y2 = _rot(X2, Y2, sgn)
    return y1 + ((XT - x1) * (y2 - y1)) // (x2 - x1), Z1 + ((XT - x1) * (Z2 - Z1)) // (x2 - x1), x2


def test_merge_rotation_matches_the_plane_rotation():
    """The Q30 rotation agrees with the real rotation by 20 degrees to within one LSB (an
    independent check of the sign convention: T = next sector is a rotation by -20 degrees)."""
    for X, Y in [(29000, 3800), (12000, -1500), (30000, 5000)]:
        for sgn in (1, -1):
            a = math.radians(20.0)
            xe = X * math.cos(a) + sgn * Y * math.sin(a)
            ye = -sgn * X * math.sin(a) + Y * math.cos(a)
            x, y = _rot(X, Y, sgn)
            assert abs(x - xe) <= 1 and abs(y - ye) <= 1


@pytest.mark.parametrize("ks,kt,sgn", [(0, 1, 1), (1, 0, -1), (17, 0, 1), (0, 17, -1), (18, 19, 1), (35, 18, 1)])
def test_merge_windows_are_192_inclusive(ks, kt, sgn):
    """R-9: |dY| <= 192 and |dZ| <= 192 LSB at the extrapolated point match, 193 does not; D is
    dY^2 + dZ^2."""
    XT = _rot(S_END[3], S_END[4], sgn)[0] + 300
    yp, zp, _ = _predicted(S_END, sgn, XT)
    for d, ok in [(0, True), (192, True), (-192, True), (193, False), (-193, False)]:
        assert (O.merge_decide(ks, S_END, kt, (XT, yp + d, zp)) == d * d) if ok else \
            O.merge_decide(ks, S_END, kt, (XT, yp + d, zp)) is None
        assert (O.merge_decide(ks, S_END, kt, (XT, yp, zp + d)) == d * d) if ok else \
            O.merge_decide(ks, S_END, kt, (XT, yp, zp + d)) is None
    assert O.merge_decide(ks, S_END, kt, (XT, yp + 192, zp - 192)) == 2 * 192 * 192


def test_merge_extrapolation_distance_is_2048_inclusive():
    """R-9: T's first row may lie at most 2048 LSB (16 cm) from S's rotated outer end, either way."""
    x2 = _rot(S_END[3], S_END[4], 1)[0]
    for dx, ok in [(2048, True), (2049, False), (-2048, True), (-2049, False), (0, True)]:
        XT = x2 + dx
        yp, zp, _ = _predicted(S_END, 1, XT)
        r = O.merge_decide(0, S_END, 1, (XT, yp, zp))
        assert (r == 0) if ok else r is None, (dx, r)


def test_merge_needs_an_outward_segment_end():
    """R-9: an end whose rotated direction has dx <= 0 never matches."""
    X1, Y1, Z1, X2, Y2, Z2 = S_END
    inward = (X2, Y2, Z2, X1, Y1, Z1)                   # the same line walked inwards
    x1, _ = _rot(X2, Y2, 1)
    for XT in range(x1 - 600, x1 + 601, 50):
        for YT in range(-4000, 4001, 50):
            assert O.merge_decide(0, inward, 1, (XT, YT, Z1)) is None
    # a rotated end with x2 == x1 exactly (dx = 0): pick X2, Y2 on the line orthogonal to the new x
    flat = None
    for dY in range(1, 2000):
        for dX in range(-2000, 0):
            if _rot(X1 + dX, Y1 + dY, 1)[0] == _rot(X1, Y1, 1)[0]:
                flat = (X1, Y1, Z1, X1 + dX, Y1 + dY, Z2)
                break
        if flat:
            break
    assert flat is not None
    assert O.merge_decide(0, flat, 1, (_rot(X1, Y1, 1)[0] + 100, 0, Z1)) is None


def test_merge_only_between_adjacent_sectors_of_one_side():
    """R-9: sectors two apart, the same sector, or the other z side never match."""
    XT = _rot(S_END[3], S_END[4], 1)[0] + 300
    yp, zp, _ = _predicted(S_END, 1, XT)
    assert O.merge_decide(0, S_END, 1, (XT, yp, zp)) == 0
    for kt in (0, 2, 16, 18, 19, 35):
        assert O.merge_decide(0, S_END, kt, (XT, yp, zp)) is None


# ---------------------------------------------------------------------------------------------
# R-10 assembly
# ---------------------------------------------------------------------------------------------

def _segments(n_seg, n_hits=10, n_rows=159):
    seg = -np.ones((n_seg, n_rows), np.int32)
    for s in range(n_seg):
        seg[s, :n_hits] = np.arange(s * n_hits, (s + 1) * n_hits)
    return seg, np.full(n_seg, n_hits, np.int32)


@pytest.mark.parametrize("nxt,tracks", [
    ([-1, 3, -1, 5, -1, 1], [[0], [1, 3, 5], [2], [4]]),          # cycle 1 -> 3 -> 5 -> 1
    ([-1, -1, -1, -1, 5, 4], [[0], [1], [2], [3], [4, 5]]),       # cycle 4 <-> 5
    ([2, -1, 0, 4, 3, -1], [[0, 2], [1], [3, 4], [5]]),           # two 2-cycles
    ([1, 2, 3, 4, 5, 0], [[0, 1, 2, 3, 4, 5]]),                   # one cycle through all
    ([3, -1, 1, -1, -1, 2], [[0, 3], [4], [5, 2, 1]]),            # plain chains, no cycle
])
def test_assembly_cuts_a_cycle_in_front_of_its_smallest_segment(nxt, tracks):
    """R-10: one track per chain of links, ordered by the index of its first segment; a cycle is
    cut in front of its smallest segment, which then starts the track."""
    seg, segn = _segments(len(nxt))
    off, hits, label = O.assemble(10 * len(nxt), seg, segn, np.array(nxt, np.int32))
    assert len(off) - 1 == len(tracks)
    for t, segs in enumerate(tracks):
        want = np.concatenate([np.arange(s * 10, s * 10 + 10) for s in segs])
        np.testing.assert_array_equal(hits[off[t]:off[t + 1]], want)
        assert np.all(label[want] == t)


# ---------------------------------------------------------------------------------------------
# R-6 / R-7 cleaning and chains: brute force on tiny sectors
# ---------------------------------------------------------------------------------------------

def test_cleaning_keeps_every_mutual_link_and_chains_are_complete():
    """Random row-respecting link arrays on tiny sectors: the cleaned links are exactly the mutual
    ones, and the chains are exactly the walks from every start (an up-link and no kept down-link)
    of at least five hits, in start order."""
    rng = np.random.default_rng(11)
    n_chain_total = 0
    for trial in range(300):
        n_rows = 12
        per_row = rng.integers(1, 4, n_rows)
        rows = np.repeat(np.arange(n_rows), per_row)
        n = len(rows)
        first = np.concatenate([[0], np.cumsum(per_row)])
        up = -np.ones(n, np.int32)
        down = -np.ones(n, np.int32)
        for c in range(n):
            r = rows[c]
            if 0 < r < n_rows - 1 and rng.random() < 0.9:
                up[c] = rng.integers(first[r + 1], first[r + 2])
                down[c] = rng.integers(first[r - 1], first[r])
        up2, down2 = O.clean(up, down)
        for c in range(n):
            assert up2[c] == (up[c] if up[c] >= 0 and down[up[c]] == c else -1)
            assert down2[c] == (down[c] if down[c] >= 0 and up[down[c]] == c else -1)
        want = []
        for c in range(n):
            if up2[c] < 0 or down2[c] >= 0:
                continue
            walk = [c]
            while up2[walk[-1]] >= 0:
                walk.append(up2[walk[-1]])
            if len(walk) >= 5:
                want.append((c, len(walk)))
        st, ln = O.chains(up2, down2)
        assert list(zip(st.tolist(), ln.tolist())) == want
        n_chain_total += len(want)
    assert n_chain_total > 30
