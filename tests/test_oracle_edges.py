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
  R-5' / R-7' / R-9' (rules for inefficient data, off by default): links across one empty row with
      the window doubled and the cut scaled by the row distances; the following's filter steps
      once per row across a skipped row; the gap merge inside a sector (gaps of 8 to 23 empty
      rows, the following's radius, both extrapolations, the stop rules, mutual best).
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


# ---------------------------------------------------------------------------------------------
# Rules for inefficient data (off by default): links across one empty row, gap merge in a sector
# ---------------------------------------------------------------------------------------------

def _brute_links_skip(pad, tim, bin_off, n_rows, n_sectors, W=384, DMAX=13600):
    """Naive enumeration of the skip-row rule: a side whose neighbouring row has no cluster in the
    window takes the row after it with the window doubled; residual b*u + a*d - (a+b)*c with
    a, b the row distances; cut 6 D <= (a^2 + b^2 + (a+b)^2) D_MAX; minimum (D, u, d)."""
    n = len(pad)
    up = -np.ones(n, np.int32)
    down = -np.ones(n, np.int32)
    P, T = pad.astype(np.int64), tim.astype(np.int64)

    def cands(b, c, w):
        return [x for x in range(bin_off[b], bin_off[b + 1]) if abs(P[x] - P[c]) <= w and abs(T[x] - T[c]) <= w]

    for s in range(n_sectors):
        for r in range(1, n_rows - 1):
            b = s * n_rows + r
            for c in range(bin_off[b], bin_off[b + 1]):
                us, a = cands(b + 1, c, W), 1
                if not us and r + 2 <= n_rows - 1:
                    us, a = cands(b + 2, c, 2 * W), 2
                ds, bb = cands(b - 1, c, W), 1
                if not ds and r - 2 >= 0:
                    ds, bb = cands(b - 2, c, 2 * W), 2
                k = a * a + bb * bb + (a + bb) ** 2
                best = None
                for u in us:
                    for d in ds:
                        D = (bb * P[u] + a * P[d] - (a + bb) * P[c]) ** 2 + (bb * T[u] + a * T[d] - (a + bb) * T[c]) ** 2
                        if 6 * D <= k * DMAX and (best is None or (D, u, d) < best):
                            best = (D, u, d)
                if best is not None:
                    up[c], down[c] = best[1], best[2]
    return up, down


def _tiny_sparse_event(rng, n_rows=10, n_sectors=2, max_per_row=3, empty=0.35):
    pads, tims, bins = [], [], []
    for s in range(n_sectors):
        for r in range(n_rows):
            k = 0 if rng.random() < empty else int(rng.integers(1, max_per_row + 1))
            y = rng.integers(-500, 501, k)
            z = 8000 + rng.integers(-500, 501, k)
            o = np.lexsort((z, y))
            pads.append(y[o]); tims.append(z[o]); bins.append(np.full(k, s * n_rows + r))
    b = np.concatenate(bins)
    return (np.concatenate(pads).astype(np.int16), np.concatenate(tims).astype(np.uint16),
            np.searchsorted(b, np.arange(n_sectors * n_rows + 1)).astype(np.int32))


def test_skip_row_links_match_brute_force_on_tiny_sectors():
    """R-5 with the skip-row rule against a naive enumeration, on tiny sectors with many empty
    rows and windows (so that both a = 2 and b = 2 occur)."""
    rng = np.random.default_rng(300)
    g = O.geometry(n_sectors=2, n_rows=10)
    n_skip = 0
    for trial in range(60):
        pad, tim, bin_off = _tiny_sparse_event(rng)
        up, down = O.links(pad, tim, bin_off, g, rules=O.RULE_SKIP_ROW)
        bu, bd = _brute_links_skip(pad, tim, bin_off, 10, 2)
        np.testing.assert_array_equal(up, bu)
        np.testing.assert_array_equal(down, bd)
        rows = np.repeat(np.arange(20) % 10, np.diff(bin_off))
        has = up >= 0
        n_skip += int((np.abs(rows[up[has]] - rows[has]) == 2).sum() + (np.abs(rows[down[has]] - rows[has]) == 2).sum())
        # without the rule only links to the neighbouring rows (the plain reading)
        u0, _ = O.links(pad, tim, bin_off, g)
        assert np.all((u0 < 0) | (np.abs(rows[np.maximum(u0, 0)] - rows) == 1))
    assert n_skip > 20


@pytest.mark.parametrize("a,b,limit", [(2, 1, 178), (1, 2, 178), (2, 2, 116)])
def test_skip_row_cut_scales_with_the_row_distance(a, b, limit):
    """A straight line with the row(s) next to c removed: the partner across the empty row links at
    displacements up to the scaled cut and not one LSB beyond.  (a, b) = (2, 1): k = 14, 6 D <=
    14 * 13600 allows a residual of 178 (31684) and not 179 (32041); with the displacement on the
    partner two rows away the residual is b * delta.  (2, 2): k = 24, residual 2 * delta, 232 (delta =
    116) passes and 234 (117) does not."""
    g = O.geometry(n_sectors=1, n_rows=7)
    y = lambda r: 100 + 30 * r
    z = lambda r: 9000 + 20 * r
    for delta, ok in [(limit, True), (limit + 1, False)]:
        # c on row 3; the up partner a rows up, the down partner b rows down; the displacement sits
        # on the partner across the empty row (on the up partner when both sides skip)
        pts = {3: (y(3), z(3))}
        pts[3 + a] = (y(3 + a) + (delta if a == 2 else 0), z(3 + a))
        pts[3 - b] = (y(3 - b) + (delta if (b == 2 and a == 1) else 0), z(3 - b))
        rows = sorted(pts)
        pad = np.array([pts[r][0] for r in rows], np.int16)
        tim = np.array([pts[r][1] for r in rows], np.uint16)
        bin_off = np.searchsorted(np.array(rows), np.arange(8)).astype(np.int32)
        up, down = O.links(pad, tim, bin_off, g, rules=O.RULE_SKIP_ROW)
        c = rows.index(3)
        assert (up[c] >= 0) == ok, (a, b, delta, up[c], down[c])
        u0, _ = O.links(pad, tim, bin_off, g)
        assert u0[c] == -1                      # the plain reading never links across the gap


def test_following_steps_one_row_per_predict_across_a_skipped_row():
    """R-7 with a chain that skips a row: the filter predicts twice across the skip (a single
    prediction would double the slope), so the extension finds every cluster of the line."""
    b = Builder()
    rows = [20, 21, 23, 24, 26, 27, 28, 29]          # rows 22 and 25 skipped inside the chain
    chain = [b.add(0, r, -300 + 40 * r, 5000 + 25 * r) for r in rows]
    beyond = b.line(0, range(30, 80), -300, 40, 5000, 25)
    below = b.line(0, range(5, 20), -300, 40, 5000, 25)
    cand, index = _follow(b, chain)
    assert {index[p] for p in beyond} <= cand
    assert {index[p] for p in below} <= cand


def _gap_segments(builder, segs):
    """Segments (lists of points, ascending rows) as the selection's kept-hit arrays."""
    pad, tim, bin_off, index = builder.build()
    seg = -np.ones((len(segs), 159), np.int32)
    for k, pts in enumerate(segs):
        seg[k, :len(pts)] = [index[p] for p in pts]
    return pad, tim, bin_off, seg, np.array([len(p) for p in segs], np.int32)


@pytest.mark.parametrize("gap", [7, 8, 12, 24, 25])
def test_gap_merge_joins_a_straight_track_across_dead_rows(gap):
    """R-9' (gap merge): two pieces of one straight track separated by `gap` empty rows are joined
    when at least 8 rows are empty (fewer are the following's to bridge) and the second piece starts
    at most 24 rows past the first piece's end."""
    b = Builder()
    s1 = b.line(3, range(30, 60), -300, 9, 7000, 30)
    s2 = b.line(3, range(60 + gap, min(60 + gap + 30, 159)), -300, 9, 7000, 30)
    pad, tim, bin_off, seg, segn = _gap_segments(b, [s1, s2])
    nxt = O.gap_merge(pad, tim, bin_off, seg, segn)
    rt_minus_rs = gap + 1
    assert (nxt[0] == 1) == (8 <= gap and rt_minus_rs <= 24), (gap, nxt)
    assert nxt[1] == -1


@pytest.mark.parametrize("gap", [8, 12, 20])
def test_gap_merge_window_is_the_radius_after_the_missed_rows(gap):
    """The second piece shifted parallel by delta in Y: both the forward prediction of the first
    piece and the backward prediction of the second are off by delta, so the link holds iff delta <=
    77 + 38 (k - 1) with k the row distance between the two ends."""
    w = 77 + 38 * gap
    for delta, ok in [(w, True), (w + 1, False), (-w, True), (-w - 1, False)]:
        b = Builder()
        s1 = b.line(4, range(30, 60), -300, 9, 7000, 30)
        s2 = [b.add(4, r, -300 + 9 * r + delta, 7000 + 30 * r) for r in range(60 + gap, 60 + gap + 30)]
        pad, tim, bin_off, seg, segn = _gap_segments(b, [s1, s2])
        nxt = O.gap_merge(pad, tim, bin_off, seg, segn)
        assert (nxt[0] == 1) == ok, (gap, delta)


def test_gap_merge_stops_where_the_track_leaves_the_sector():
    """A piece whose extrapolation leaves the sector acceptance inside the gap is not joined to a
    piece that starts further on at the extrapolated position (it left the sector there)."""
    R0, gap = 60, 12
    slope = 90
    b = Builder()
    # ends at row 59 about 10 rows before it would cross |y| = ymax
    y_end = ymax(R0 + 6) - 6 * slope
    s1 = [b.add(5, r, y_end - slope * (R0 - 1 - r), 7000 + 30 * r) for r in range(R0 - 30, R0)]
    s2 = [b.add(5, r, min(y_end + slope * (r - R0 + 1), ymax(r)), 7000 + 30 * r) for r in range(R0 + gap, R0 + gap + 20)]
    pad, tim, bin_off, seg, segn = _gap_segments(b, [s1, s2])
    assert O.gap_merge(pad, tim, bin_off, seg, segn)[0] == -1


def test_gap_merge_takes_the_mutual_best_pair():
    """Two candidate second pieces: the nearer one to the extrapolation is linked, the other not."""
    b = Builder()
    s1 = b.line(6, range(30, 60), -300, 9, 7000, 30)
    near = [b.add(6, r, -300 + 9 * r + 40, 7000 + 30 * r) for r in range(72, 100)]
    far = [b.add(6, r, -300 + 9 * r - 200, 7000 + 30 * r) for r in range(72, 100)]
    pad, tim, bin_off, seg, segn = _gap_segments(b, [s1, far, near])
    nxt = O.gap_merge(pad, tim, bin_off, seg, segn)
    assert nxt[0] == 2 and nxt[1] == -1 and nxt[2] == -1


def test_rules_leave_an_efficient_event_nearly_unchanged_and_help_an_inefficient_one():
    """Sanity of the readings (the paper prints no efficiency): with the rules the found-whole
    efficiency of an event with dead rows rises well above the plain tracking's, and on the same
    event shape without inefficiency it does not drop."""
    from paper_1712_09434_gb300 import synth
    ev = synth.make_event(synth.inefficient_central(n_tracks=3000))
    e0 = synth.track_quality(ev, *(lambda r: (r["trk_off"], r["trk_hits"]))(O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off)))
    e3 = synth.track_quality(ev, *(lambda r: (r["trk_off"], r["trk_hits"]))(O.track_event(ev.pad_fp, ev.time_fp, ev.bin_off, rules=3)))
    assert e3[0] > e0[0] + 0.3, (e0, e3)
    cfg = synth.central_event(n_tracks=3000)
    ef = synth.make_event(cfg)
    f0 = synth.track_quality(ef, *(lambda r: (r["trk_off"], r["trk_hits"]))(O.track_event(ef.pad_fp, ef.time_fp, ef.bin_off)))
    f3 = synth.track_quality(ef, *(lambda r: (r["trk_off"], r["trk_hits"]))(O.track_event(ef.pad_fp, ef.time_fp, ef.bin_off, rules=3)))
    assert f3[0] > f0[0] - 0.01, (f0, f3)


def test_following_skip_keeps_the_prediction_exact():
    """A steep line (150 LSB per row) whose chain skips the row before its last hit: stepping the
    filter once per row keeps the prediction at the first extension row exact, so the line's
    cluster there (distance 0) wins over a decoy 54 LSB below it; a single prediction across the
    skip would put the prediction on the decoy."""
    b = Builder()
    rows = [20, 21, 22, 23, 24, 25, 26, 27, 29]
    chain = [b.add(0, r, -2500 + 150 * r, 6000 + 10 * r) for r in rows]
    true30 = b.add(0, 30, -2500 + 150 * 30, 6300)
    decoy = b.add(0, 30, -2500 + 150 * 30 - 54, 6300)
    cand, index = _follow(b, chain)
    assert index[true30] in cand and index[decoy] not in cand


def test_gap_merge_needs_both_extrapolations():
    """The second piece starts on the first piece's extrapolation but runs at a slope 60 LSB per row
    steeper: its own extrapolation back to the first piece's end misses by 60 x 13 = 780 > 533 (the
    radius after 12 empty rows), so the pieces are not joined."""
    b = Builder()
    s1 = b.line(7, range(30, 60), -300, 9, 7000, 30)
    y72 = -300 + 9 * 72
    s2 = [b.add(7, r, y72 + 69 * (r - 72), 7000 + 30 * r) for r in range(72, 100)]
    pad, tim, bin_off, seg, segn = _gap_segments(b, [s1, s2])
    assert O.gap_merge(pad, tim, bin_off, seg, segn)[0] == -1
    # the same piece continuing the first one's slope is joined
    b = Builder()
    s1 = b.line(7, range(30, 60), -300, 9, 7000, 30)
    s2 = b.line(7, range(72, 100), -300, 9, 7000, 30)
    pad, tim, bin_off, seg, segn = _gap_segments(b, [s1, s2])
    assert O.gap_merge(pad, tim, bin_off, seg, segn)[0] == 1
