"""Hand-constructed cluster sets for the edge pins (no tracking arithmetic): exact straight tracks
on chosen rows of chosen sectors, single clusters placed at chosen offsets, and the binning of
the detector layout (clusters sorted by (sector, row, pad, time))."""
import math

import numpy as np

N_SECTORS, N_ROWS = 36, 159
LSB = 1.0 / 128.0


def row_x(r):
    return 85.0 + r * 162.0 / 158.0


def ymax(r):
    """Half width of the sector acceptance at row r in LSB (the geometry's definition)."""
    return math.floor(row_x(r) * math.tan(math.radians(10.0)) / LSB)


class Builder:
    """Collects (sector, row, y, z) points and bins them like the detector layout."""

    def __init__(self):
        self.pts = []

    def add(self, sector, row, y, z):
        self.pts.append((int(sector), int(row), int(y), int(z)))
        return self.pts[-1]

    def line(self, sector, rows, y0, sy, z0, sz):
        """Exact straight track: y = y0 + sy*row, z = z0 + sz*row on the given rows."""
        return [self.add(sector, r, y0 + sy * r, z0 + sz * r) for r in rows]

    def build(self):
        pts = sorted(set(self.pts))
        assert len(pts) == len(self.pts), "duplicate points"
        sec = np.array([p[0] for p in pts], np.int64)
        row = np.array([p[1] for p in pts], np.int64)
        pad = np.array([p[2] for p in pts], np.int64)
        tim = np.array([p[3] for p in pts], np.int64)
        assert pad.min(initial=0) >= -32768 and pad.max(initial=0) < 32768
        assert tim.min(initial=0) >= 0 and tim.max(initial=0) < 65536
        b = sec * N_ROWS + row
        bin_off = np.searchsorted(b, np.arange(N_SECTORS * N_ROWS + 1)).astype(np.int32)
        index = {p: i for i, p in enumerate(pts)}
        return pad.astype(np.int16), tim.astype(np.uint16), bin_off, index


def chain_links(n, hits):
    """Cleaned up-links of one hand-made chain (cluster indices in ascending rows)."""
    up2 = -np.ones(n, np.int32)
    for a, b in zip(hits[:-1], hits[1:]):
        up2[a] = b
    return up2


def edge_events():
    """Events made of hand-placed straight tracks, one construction per sector, each sitting on an
    edge of the following rule: gaps of 7 and 8 empty rows, clusters at exactly the search radius
    after k misses and one LSB beyond, equal distances inside one Z slab and across two slabs,
    a window spanning three Z slabs, the slope limit, the acceptance edge and the drift range.
    Tracks run along chains that the neighbour finding forms on its own (exact lines)."""
    events = []
    b = Builder()
    sec = iter(range(N_SECTORS))

    def flush():
        nonlocal b, sec
        events.append(b)
        b = Builder()
        sec = iter(range(N_SECTORS))

    def next_sector():
        try:
            return next(sec)
        except StopIteration:
            flush()
            return next(sec)

    y = lambda r: -300 + 7 * r
    z = lambda r: 5000 + 40 * r
    for gap in (7, 8):
        s = next_sector()
        b.line(s, range(20, 40), -300, 7, 5000, 40)
        b.line(s, range(40 + gap, 101), -300, 7, 5000, 40)
    for k in range(8):
        w = 77 + 38 * k
        for dy, dz in ((w, 0), (w + 1, 0), (0, -w), (0, -w - 1)):
            s = next_sector()
            R = 40 + k
            b.line(s, range(20, 40), -300, 7, 5000, 40)
            b.line(s, range(R + 1, R + 15), -300, 7, 5000, 40)
            b.add(s, R, y(R) + dy, z(R) + dz)
    # equal distances: one slab, and across the slab boundary at Z = 20 * 512 (the lower index in
    # the higher slab), and a window of three slabs after 7 misses
    zb = 20 * 512
    for pts in (((-30, 0), (30, 0)), ((0, -30), (0, 30)), ((-30, 30), (30, -30))):
        s = next_sector()
        R = 40
        b.line(s, range(20, 40), -300, 7, zb - 40 * 40, 40)
        b.line(s, range(R + 1, R + 15), -300, 7, zb - 40 * 40, 40)
        for dy, dz in pts:
            b.add(s, R, y(R) + dy, zb + dz)
    s = next_sector()
    R = 47
    z0 = zb + 250 - 40 * R
    b.line(s, range(20, 40), -300, 7, z0, 40)
    b.line(s, range(R + 1, R + 15), -300, 7, z0, 40)
    b.add(s, R, y(R), zb + 250 - 300)
    b.add(s, R, y(R), zb + 250 + 300)
    for slope in (320, 321, -320, -321):
        s = next_sector()
        y0 = -1500 if slope > 0 else 1500
        for r in range(20, 26):
            b.add(s, r, y0 + slope * (r - 20), 8000 + 10 * r)
    for side in (1, -1):
        for off in (0, 1):
            s = next_sector()
            R = 30
            target = side * (ymax(R) + off)
            for r in range(20, R + 1):
                b.add(s, r, target - side * 40 * (R - r), 6000 + 20 * r)
    for zR in (0, -1, 32000, 32001):
        s = next_sector()
        R = 30
        sz = -50 if zR <= 0 else 50
        for r in range(20, R):
            b.add(s, r, 100 + 5 * r, zR - sz * (R - r))
        b.add(s, R, 100 + 5 * R, min(max(zR, 0), 32001))
    flush()
    return [e.build() for e in events]


def rule_events():
    """Events for the rules on inefficient data, one construction per sector: straight tracks with
    single empty rows (links across them) and with the partner across the empty row displaced to
    the edge of the scaled cut; two pieces of a track separated by 7 to 25 empty rows; the second
    piece shifted parallel by the gap radius and one LSB more; a second piece of a steeper slope;
    a piece whose extrapolation leaves the sector inside the gap."""
    events = []
    b = Builder()
    sec = iter(range(N_SECTORS))

    def next_sector():
        nonlocal b, sec
        try:
            return next(sec)
        except StopIteration:
            events.append(b)
            b = Builder()
            sec = iter(range(N_SECTORS))
            return next(sec)

    for missing in ([40], [40, 60], [40, 42], [40, 41]):
        s = next_sector()
        b.line(s, [r for r in range(20, 90) if r not in missing], -300, 11, 6000, 25)
    # the partner across an empty row displaced: residual limits 178 (one side skips) and 116
    # (both sides skip, displacement on the up partner)
    for both, delta in ((False, 178), (False, 179), (True, 116), (True, 117)):
        s = next_sector()
        rows = [r for r in range(20, 60) if r not in ((39, 41) if both else (41,))]
        for r in rows:
            b.add(s, r, -300 + 11 * r + (delta if r == 42 else 0), 6000 + 25 * r)
    for gap in (7, 8, 12, 23, 24, 25):
        s = next_sector()
        b.line(s, range(30, 60), -300, 9, 7000, 30)
        b.line(s, range(60 + gap, min(60 + gap + 30, N_ROWS)), -300, 9, 7000, 30)
    for gap in (8, 12):
        w = 77 + 38 * gap
        for delta in (w, w + 1, -w, -w - 1):
            s = next_sector()
            b.line(s, range(30, 60), -300, 9, 7000, 30)
            for r in range(60 + gap, 60 + gap + 30):
                b.add(s, r, -300 + 9 * r + delta, 7000 + 30 * r)
    s = next_sector()
    b.line(s, range(30, 60), -300, 9, 7000, 30)
    for r in range(72, 100):
        b.add(s, r, -300 + 9 * 72 + 69 * (r - 72), 7000 + 30 * r)
    s = next_sector()
    y_end = ymax(66) - 6 * 90
    for r in range(30, 60):
        b.add(s, r, y_end - 90 * (59 - r), 7000 + 30 * r)
    for r in range(72, 92):
        b.add(s, r, min(y_end + 90 * (r - 59), ymax(r)), 7000 + 30 * r)
    events.append(b)
    return [e.build() for e in events]
