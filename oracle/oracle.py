"""Python front end of the CPU oracle (test infrastructure only).

Loads the plain C oracle (``tpc_oracle.c``, FP64 / int64, single thread) through ctypes and runs
the track-reconstruction steps of the paper's section 3 on one event at a time.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this module; the
CUDA library never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tpc_oracle.c")
LIB = os.path.join(HERE, "libtpc_oracle.so")

_lib = None


def build(force=False):
    """Compile the oracle with gcc (no fast-math: IEEE double semantics)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class GeomIn(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("x_first", ctypes.c_double), ("x_last", ctypes.c_double),
                ("half_angle_deg", ctypes.c_double), ("z_max", ctypes.c_double),
                ("lsb", ctypes.c_double), ("bz", ctypes.c_double)]


def geometry(n_sectors=36, n_rows=159, x_first=85.0, x_last=247.0, half_angle_deg=10.0,
             z_max=250.0, lsb=1.0 / 128.0, bz=0.5):
    return GeomIn(n_sectors, n_rows, x_first, x_last, half_angle_deg, z_max, lsb, bz)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        _lib.or_chi2_total.restype = ctypes.c_double
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _geom(g):
    return ctypes.byref(g if g is not None else geometry())


# optional rules for inefficient data (bit flags; off by default)
RULE_SKIP_ROW = 1       # a link may skip one row where the neighbouring row has no candidate
RULE_GAP_MERGE = 2      # segments of one sector joined across a gap of pad rows


def links(pad, tim, bin_off, g=None, rules=0):
    """S2 neighbour finding: (up, down) per cluster."""
    n = pad.shape[0]
    up = np.empty(n, np.int32)
    down = np.empty(n, np.int32)
    rc = lib().or_links_rules(_geom(g), _p(pad), _p(tim), _p(bin_off), ctypes.c_int32(n), ctypes.c_int32(rules),
                              _p(up), _p(down))
    assert rc == 0, rc
    return up, down


def clean(up, down):
    """S3 link cleaning: mutual links only."""
    n = up.shape[0]
    up2 = np.empty(n, np.int32)
    down2 = np.empty(n, np.int32)
    lib().or_clean(ctypes.c_int32(n), _p(up), _p(down), _p(up2), _p(down2))
    return up2, down2


def chains(up2, down2):
    """S4 chains of at least N_SEED hits: (start, length), ordered by start cluster."""
    n = up2.shape[0]
    cap = n // 5 + 1
    st = np.empty(cap, np.int32)
    ln = np.empty(cap, np.int32)
    nc = lib().or_chains(ctypes.c_int32(n), _p(up2), _p(down2), _p(st), _p(ln), ctypes.c_int32(cap))
    assert nc >= 0, nc
    return st[:nc].copy(), ln[:nc].copy()


def follow(pad, tim, bin_off, chain_start, chain_len, up2, g=None):
    """S5 track following: candidate hit lists [n_chains, n_rows] (-1 padded) and counts."""
    gg = g if g is not None else geometry()
    nc = chain_start.shape[0]
    hits = np.empty((max(nc, 1), gg.n_rows), np.int32)
    cnt = np.empty(max(nc, 1), np.int32)
    rc = lib().or_follow(ctypes.byref(gg), _p(pad), _p(tim), _p(bin_off), ctypes.c_int32(pad.shape[0]),
                         ctypes.c_int32(nc), _p(chain_start), _p(chain_len), _p(up2), _p(hits), _p(cnt))
    assert rc == 0, rc
    return hits[:nc], cnt[:nc]


def select(n_clusters, cand_hits, cand_n, cand_start, n_rows=159):
    """S6 sequential greedy selection: kept hits per candidate and accepted flags."""
    nc = cand_n.shape[0]
    seg = np.empty((max(nc, 1), n_rows), np.int32)
    segn = np.empty(max(nc, 1), np.int32)
    acc = np.empty(max(nc, 1), np.int32)
    ch = np.ascontiguousarray(cand_hits, dtype=np.int32) if nc else np.zeros((1, n_rows), np.int32)
    lib().or_select(ctypes.c_int32(n_clusters), ctypes.c_int32(n_rows), ctypes.c_int32(nc), _p(ch),
                    _p(np.ascontiguousarray(cand_n, np.int32)), _p(np.ascontiguousarray(cand_start, np.int32)),
                    _p(seg), _p(segn), _p(acc))
    return seg[:nc], segn[:nc], acc[:nc]


def merge(pad, tim, bin_off, seg_hits, seg_n, g=None, gap_next=None):
    """S7 merge links: next[segment] or -1.  gap_next (gap links inside a sector, or None): segments
    with a gap successor are no outer ends, segments with a gap predecessor no first segments."""
    nc = seg_n.shape[0]
    nxt = np.empty(max(nc, 1), np.int32)
    sh = np.ascontiguousarray(seg_hits, np.int32) if nc else np.zeros((1, 159), np.int32)
    gn = np.ascontiguousarray(gap_next, np.int32) if gap_next is not None else None
    rc = lib().or_merge(_geom(g), _p(pad), _p(tim), _p(bin_off), ctypes.c_int32(pad.shape[0]),
                        ctypes.c_int32(nc), _p(sh), _p(np.ascontiguousarray(seg_n, np.int32)),
                        _p(gn) if gn is not None else ctypes.c_void_p(0), _p(nxt))
    assert rc == 0, rc
    return nxt[:nc]


def gap_merge(pad, tim, bin_off, seg_hits, seg_n, g=None):
    """S7' gap links inside a sector: gap_next[segment] or -1."""
    nc = seg_n.shape[0]
    nxt = np.empty(max(nc, 1), np.int32)
    sh = np.ascontiguousarray(seg_hits, np.int32) if nc else np.zeros((1, 159), np.int32)
    rc = lib().or_gap_merge(_geom(g), _p(pad), _p(tim), _p(bin_off), ctypes.c_int32(pad.shape[0]),
                            ctypes.c_int32(nc), _p(sh), _p(np.ascontiguousarray(seg_n, np.int32)), _p(nxt))
    assert rc == 0, rc
    return nxt[:nc]


def assemble(n_clusters, seg_hits, seg_n, nxt, n_rows=159):
    """Merged tracks: (trk_off, trk_hits, label)."""
    nc = seg_n.shape[0]
    cap_h = int(seg_n.sum()) + 1
    cap_t = nc + 1
    off = np.zeros(cap_t + 1, np.int32)
    hits = np.empty(cap_h, np.int32)
    label = np.empty(max(n_clusters, 1), np.int32)
    sh = np.ascontiguousarray(seg_hits, np.int32) if nc else np.zeros((1, n_rows), np.int32)
    nt = lib().or_assemble(ctypes.c_int32(n_clusters), ctypes.c_int32(n_rows), ctypes.c_int32(nc), _p(sh),
                           _p(np.ascontiguousarray(seg_n, np.int32)), _p(np.ascontiguousarray(nxt, np.int32)),
                           _p(off), _p(hits), _p(label), ctypes.c_int32(cap_t), ctypes.c_int32(cap_h))
    assert nt >= 0, nt
    return off[:nt + 1].copy(), hits[:off[nt]].copy(), label[:n_clusters].copy()


def track_event(pad, tim, bin_off, g=None, keep_stages=False, rules=0):
    """S2-S7 on one event; returns a dict with the final tracks (and every stage if asked).  rules:
    RULE_SKIP_ROW and / or RULE_GAP_MERGE (0: the plain readings)."""
    pad = np.ascontiguousarray(pad, np.int16)
    tim = np.ascontiguousarray(tim, np.uint16)
    bin_off = np.ascontiguousarray(bin_off, np.int32)
    n = pad.shape[0]
    up, down = links(pad, tim, bin_off, g, rules)
    up2, down2 = clean(up, down)
    cst, cln = chains(up2, down2)
    ch, cn = follow(pad, tim, bin_off, cst, cln, up2, g)
    seg, segn, acc = select(n, ch, cn, cst)
    gap = gap_merge(pad, tim, bin_off, seg, segn, g) if rules & RULE_GAP_MERGE else None
    nxt = merge(pad, tim, bin_off, seg, segn, g, gap_next=gap)
    links_all = np.where(gap >= 0, gap, nxt).astype(np.int32) if gap is not None else nxt
    off, hits, label = assemble(n, seg, segn, links_all)
    out = dict(trk_off=off, trk_hits=hits, label=label)
    if keep_stages:
        out.update(up=up, down=down, up2=up2, down2=down2, chain_start=cst, chain_len=cln,
                   cand_hits=ch, cand_n=cn, seg_hits=seg, seg_n=segn, accepted=acc, next=links_all,
                   gap_next=gap if gap is not None else -np.ones_like(nxt))
    return out


def frame_merge(pad, tim, bin_off, n_slices, slice_len, trk_off, trk_hits, ev_trk_off, g=None):
    """S11 slice merge of a time frame: links next[track] (slice j+1 -> slice j) or -1."""
    nt = int(trk_off.shape[0]) - 1
    nxt = np.empty(max(nt, 1), np.int32)
    rc = lib().or_frame_merge(_geom(g), _p(np.ascontiguousarray(pad, np.int16)),
                              _p(np.ascontiguousarray(tim, np.uint16)), _p(np.ascontiguousarray(bin_off, np.int32)),
                              ctypes.c_int32(pad.shape[0]), ctypes.c_int32(n_slices), ctypes.c_int32(slice_len),
                              ctypes.c_int32(nt), _p(np.ascontiguousarray(trk_off, np.int32)),
                              _p(np.ascontiguousarray(trk_hits, np.int32)),
                              _p(np.ascontiguousarray(ev_trk_off, np.int32)), _p(nxt))
    assert rc == 0, rc
    return nxt[:nt]


def frame_assemble(n_clusters, trk_off, trk_hits, nxt):
    """Frame tracks from the slice tracks and their links: (ftrk_off, ftrk_hits, flabel)."""
    nt = int(trk_off.shape[0]) - 1
    off = np.zeros(nt + 2, np.int32)
    hits = np.empty(max(int(trk_hits.shape[0]), 1), np.int32)
    label = np.empty(max(n_clusters, 1), np.int32)
    nf = lib().or_frame_assemble(ctypes.c_int32(n_clusters), ctypes.c_int32(nt),
                                 _p(np.ascontiguousarray(trk_off, np.int32)),
                                 _p(np.ascontiguousarray(trk_hits, np.int32)), _p(np.ascontiguousarray(nxt, np.int32)),
                                 _p(off), _p(hits), _p(label), ctypes.c_int32(nt + 1), ctypes.c_int32(hits.shape[0]))
    assert nf >= 0, nf
    return off[:nf + 1].copy(), hits[:off[nf]].copy(), label[:n_clusters].copy()


def track_frame(pad, tim, bin_off, n_slices, slice_len, g=None):
    """A time frame: S2-S7 on every slice (as one event each, tracks concatenated in slice order
    with global cluster indices), then the S11 slice merge and the frame tracks."""
    gg = g if g is not None else geometry()
    nbe = gg.n_sectors * gg.n_rows
    bin_off = np.ascontiguousarray(bin_off, np.int64)
    offs, hits, ev_trk_off, n_hits = [np.zeros(1, np.int64)], [], [0], 0
    for j in range(n_slices):
        a, b = int(bin_off[j * nbe]), int(bin_off[(j + 1) * nbe])
        o = track_event(pad[a:b], tim[a:b], (bin_off[j * nbe:(j + 1) * nbe + 1] - a).astype(np.int32), g)
        offs.append(o["trk_off"][1:].astype(np.int64) + n_hits)
        n_hits += int(o["trk_off"][-1])
        hits.append(o["trk_hits"].astype(np.int64) + a)
        ev_trk_off.append(ev_trk_off[-1] + len(o["trk_off"]) - 1)
    trk_off = np.concatenate(offs).astype(np.int32)
    trk_hits = np.concatenate(hits).astype(np.int32) if hits else np.zeros(0, np.int32)
    ev_trk_off = np.array(ev_trk_off, np.int32)
    n = int(pad.shape[0])
    label = -np.ones(n, np.int32)
    label[trk_hits] = np.repeat(np.arange(len(trk_off) - 1, dtype=np.int32), np.diff(trk_off))
    nxt = frame_merge(pad, tim, bin_off.astype(np.int32), n_slices, slice_len, trk_off, trk_hits, ev_trk_off, g)
    foff, fhits, flabel = frame_assemble(n, trk_off, trk_hits, nxt)
    return dict(trk_off=trk_off, trk_hits=trk_hits, ev_trk_off=ev_trk_off, label=label, next=nxt,
                ftrk_off=foff, ftrk_hits=fhits, flabel=flabel)


def fit(pad, tim, bin_off, trk_off, trk_hits, theta=None, g=None):
    """S8 FP64 Kalman refit: dict(par [T,5], xref [T], cov [T,15], chi2 [T], ndf [T])."""
    gg = g if g is not None else geometry()
    nt = trk_off.shape[0] - 1
    th = np.zeros(1 + 2 * gg.n_sectors) if theta is None else np.asarray(theta, np.float64).copy()
    if theta is None:
        th[0] = 1.0
    par = np.empty((max(nt, 1), 5))
    xref = np.empty(max(nt, 1))
    cov = np.empty((max(nt, 1), 15))
    chi2 = np.empty(max(nt, 1))
    ndf = np.empty(max(nt, 1), np.int32)
    rc = lib().or_fit(ctypes.byref(gg), _p(np.ascontiguousarray(pad, np.int16)),
                      _p(np.ascontiguousarray(tim, np.uint16)), _p(np.ascontiguousarray(bin_off, np.int32)),
                      ctypes.c_int32(pad.shape[0]), ctypes.c_int32(nt), _p(np.ascontiguousarray(trk_off, np.int32)),
                      _p(np.ascontiguousarray(trk_hits, np.int32)), _p(th), _p(par), _p(xref), _p(cov), _p(chi2),
                      _p(ndf))
    assert rc == 0, rc
    return dict(par=par[:nt], xref=xref[:nt], cov=cov[:nt], chi2=chi2[:nt], ndf=ndf[:nt])


def _weights(weight, n_trk):
    if weight is None:
        return None
    w = np.ascontiguousarray(weight, np.float64)
    assert w.shape[0] >= n_trk
    return w


def _refs(ref, n_trk):
    if ref is None:
        return None
    r = np.ascontiguousarray(ref, np.float64).reshape(-1)
    assert r.shape[0] == 8 * n_trk
    return r


def chi2_total(pad, tim, bin_off, trk_off, trk_hits, theta, g=None, weight=None, ref=None, mode=0):
    """Weighted sum of chi2 (weight per track, None = 1) of the FP64 refit at calibration theta;
    ref [T, 8] (None = none) adds the reference measurements at the vertex of every track; mode 1
    takes the measurement errors in the raw coordinates, scaled into the calibrated ones by the
    transformation (-2 log L for Gaussian raw errors)."""
    gg = g if g is not None else geometry()
    th = np.ascontiguousarray(theta, np.float64)
    nt = trk_off.shape[0] - 1
    w = _weights(weight, nt)
    r = _refs(ref, nt)
    return lib().or_chi2_total(ctypes.byref(gg), _p(np.ascontiguousarray(pad, np.int16)),
                               _p(np.ascontiguousarray(tim, np.uint16)), _p(np.ascontiguousarray(bin_off, np.int32)),
                               ctypes.c_int32(pad.shape[0]), ctypes.c_int32(nt),
                               _p(np.ascontiguousarray(trk_off, np.int32)), _p(np.ascontiguousarray(trk_hits, np.int32)),
                               _p(w) if w is not None else ctypes.c_void_p(0),
                               _p(r) if r is not None else ctypes.c_void_p(0), ctypes.c_int32(mode), _p(th))


def grad_fd(pad, tim, bin_off, trk_off, trk_hits, theta, h=(1e-6, 1e-4, 1e-4), g=None, weight=None, ref=None,
            mode=0):
    """Reference gradient d(sum w chi2)/d(theta) by FP64 central differences."""
    gg = g if g is not None else geometry()
    th = np.ascontiguousarray(theta, np.float64)
    nt = trk_off.shape[0] - 1
    w = _weights(weight, nt)
    r = _refs(ref, nt)
    grad = np.empty(1 + 2 * gg.n_sectors)
    hh = np.asarray(h, np.float64)
    rc = lib().or_grad_fd(ctypes.byref(gg), _p(np.ascontiguousarray(pad, np.int16)),
                          _p(np.ascontiguousarray(tim, np.uint16)), _p(np.ascontiguousarray(bin_off, np.int32)),
                          ctypes.c_int32(pad.shape[0]), ctypes.c_int32(nt),
                          _p(np.ascontiguousarray(trk_off, np.int32)), _p(np.ascontiguousarray(trk_hits, np.int32)),
                          _p(w) if w is not None else ctypes.c_void_p(0),
                          _p(r) if r is not None else ctypes.c_void_p(0), ctypes.c_int32(mode), _p(th), _p(hh),
                          _p(grad))
    assert rc == 0, rc
    return grad


def its_match(fit_out, first_sector, its, g=None):
    """TPC-ITS matching at the vertex (see or_its_match): fit_out = fit(...) of the TPC tracks,
    first_sector = sector of every track's first hit, its = [n_its, 8] ITS tracks.  Returns
    (match of every TPC track (ITS index or -1), match of every ITS track (TPC index or -1), chi2 of
    each match)."""
    nt = int(fit_out["par"].shape[0])
    its = np.ascontiguousarray(its, np.float64).reshape(-1, 8)
    ni = its.shape[0]
    mt = np.empty(max(nt, 1), np.int32)
    mi = np.empty(max(ni, 1), np.int32)
    c2 = np.zeros(max(nt, 1))
    rc = lib().or_its_match(_geom(g), ctypes.c_int32(nt), _p(np.ascontiguousarray(fit_out["par"], np.float64)),
                            _p(np.ascontiguousarray(fit_out["cov"], np.float64)),
                            _p(np.ascontiguousarray(fit_out["xref"], np.float64)),
                            _p(np.ascontiguousarray(fit_out["ndf"], np.int32)),
                            _p(np.ascontiguousarray(first_sector, np.int32)), ctypes.c_int32(ni), _p(its),
                            _p(mt), _p(mi), _p(c2))
    assert rc == 0, rc
    return mt[:nt], mi[:ni], c2[:nt]


def looper_pairs(fit_out, first_sector, event=None, g=None):
    """Looper-leg pairing (see or_looper_pairs): fit_out = fit(...) of the tracks, first_sector =
    sector of every track's first hit, event = event of every track (all 0 if None).  Returns
    (partner of every track or -1, leg of every track: 1 outgoing, 2 returning, 0 unpaired,
    D of each pair)."""
    nt = int(fit_out["par"].shape[0])
    ev = np.zeros(max(nt, 1), np.int32) if event is None else np.ascontiguousarray(event, np.int32)
    pair = np.empty(max(nt, 1), np.int32)
    leg = np.empty(max(nt, 1), np.int32)
    D = np.zeros(max(nt, 1))
    rc = lib().or_looper_pairs(_geom(g), ctypes.c_int32(nt), _p(np.ascontiguousarray(fit_out["par"], np.float64)),
                               _p(np.ascontiguousarray(fit_out["xref"], np.float64)),
                               _p(np.ascontiguousarray(fit_out["ndf"], np.int32)),
                               _p(np.ascontiguousarray(first_sector, np.int32)), _p(ev), _p(pair), _p(leg), _p(D))
    assert rc == 0, rc
    return pair[:nt], leg[:nt], D[:nt]


def loop_circle(par, xref, sector, ndf=1, g=None):
    """(candidate?, centre x, centre y, R, far-point z, tan lambda, curvature sign) of one fitted
    track (see or_loop_circle)."""
    out = np.zeros(6)
    ok = lib().or_loop_circle(_geom(g), _p(np.ascontiguousarray(par, np.float64)), ctypes.c_double(xref),
                              ctypes.c_int32(sector), ctypes.c_int32(ndf), _p(out))
    assert ok >= 0
    return (bool(ok),) + tuple(out.tolist())


def loop_constants():
    buf = np.zeros(8)
    k = lib().or_loop_constants(_p(buf), ctypes.c_int(8))
    return dict(zip(["RMAX", "CMIN", "DC", "DR", "DZ", "DTL"], buf[:k].tolist()))


def its_constants():
    buf = np.zeros(8)
    k = lib().or_its_constants(_p(buf), ctypes.c_int(8))
    return dict(zip(["SIGMA_Y", "DPHI", "DTL", "DZ", "CHI2"], buf[:k].tolist()))


def rule_constants():
    buf = np.zeros(8, np.int64)
    k = lib().or_rule_constants(_p(buf), ctypes.c_int(8))
    return dict(zip(["RULE_SKIP_ROW", "RULE_GAP_MERGE", "GAP_MAX"], buf[:k].tolist()))


def constants():
    buf = np.zeros(32, np.int64)
    k = lib().or_constants(_p(buf), ctypes.c_int(32))
    names = ["W_LINK", "D_MAX", "N_SEED", "M_MISS", "W_F0", "W_F1", "V_MAX", "N_MIN", "W_MERGE",
             "MERGE_XMAX", "MERGE_BACK"]
    return dict(zip(names, buf[:k].tolist()))


def merge_decide(ks, s_end, kt, t_first, g=None):
    """S7 decision on integer end points: s_end = (X1, Y1, Z1, X2, Y2, Z2) of S (the hit MERGE_BACK
    positions before its outer end, and its last hit) in the frame of sector ks; t_first = (XT, YT,
    ZT) of T's first hit in the frame of sector kt.  Returns D = dY^2 + dZ^2 on a match, else None."""
    D = ctypes.c_int64(-1)
    se = np.ascontiguousarray(s_end, np.int64)
    tf = np.ascontiguousarray(t_first, np.int64)
    ok = lib().or_merge_decide(_geom(g), ctypes.c_int32(ks), _p(se), ctypes.c_int32(kt), _p(tf), ctypes.byref(D))
    assert ok in (0, 1), ok
    return int(D.value) if ok == 1 else None


def transform(sector, row, pad, tim, theta, g=None):
    """S0: transformed (x, y, z) [n, 3] for clusters given by sector, row and raw coordinates."""
    n = len(pad)
    xyz = np.empty((max(n, 1), 3))
    rc = lib().or_transform(_geom(g), ctypes.c_int32(n), _p(np.ascontiguousarray(sector, np.int32)),
                            _p(np.ascontiguousarray(row, np.int32)), _p(np.ascontiguousarray(pad, np.int16)),
                            _p(np.ascontiguousarray(tim, np.uint16)), _p(np.ascontiguousarray(theta, np.float64)),
                            _p(xyz))
    assert rc == 0, rc
    return xyz[:n]


def fit_xyz(sector, xyz, g=None, ref=None):
    """S8 on exact points (hit order): (ok, par[5], xref, cov[15], chi2).  With ref (8 values) the
    reference measurements at the vertex are added and the state is reported at x = 0."""
    nh = len(sector)
    par = np.zeros(5)
    cov = np.zeros(15)
    xref = ctypes.c_double(0.0)
    chi2 = ctypes.c_double(0.0)
    ok = lib().or_fit_xyz(_geom(g), ctypes.c_int32(nh), _p(np.ascontiguousarray(sector, np.int32)),
                          _p(np.ascontiguousarray(xyz, np.float64)), _p(par), ctypes.byref(xref), _p(cov),
                          ctypes.byref(chi2),
                          _p(np.ascontiguousarray(ref, np.float64)) if ref is not None else ctypes.c_void_p(0))
    return bool(ok == 1), par, xref.value, cov, chi2.value


def propagate(x, p, xh, g=None):
    """One helix step: (ok, p_out[5], F[5,5])."""
    po = np.zeros(5)
    F = np.zeros(25)
    ok = lib().or_propagate(_geom(g), ctypes.c_double(x), _p(np.ascontiguousarray(p, np.float64)),
                            ctypes.c_double(xh), _p(po), _p(F))
    return bool(ok == 1), po, F.reshape(5, 5)


def cov_matrix(c15):
    """Full symmetric 5x5 from the 15-element lower triangle (row-major)."""
    m = np.zeros((5, 5))
    k = 0
    for i in range(5):
        for j in range(i + 1):
            m[i, j] = m[j, i] = c15[k]
            k += 1
    return m
