"""Seeded synthetic TPC events (input generator shared by the tests, the oracle and the bench).

This module only *simulates detector input*: charged helices from the origin in a uniform
solenoidal field, their crossings with the pad-row planes of the 36 TPC sectors, Gaussian
cluster smearing, uniform noise, an optional injected calibration distortion, and the fixed-point
quantisation of the raw (pad, time) coordinates.  It holds none of the tracking arithmetic: no
neighbour finding, no Kalman filter, no merging.  The geometry follows the pad-row layout of the
ALICE TPC that the paper's tracker reconstructs (159 pad rows, 18 sectors per side; section 3 and
section 5.1 of the paper), with the sizes and distributions of the synthetic workloads stated in
the design notes.

Crossing points are computed in closed form: a helix from the origin with transverse direction
phi0 and signed curvature C has turning angle psi = phi0 + C*s after transverse path s, and its
local x in a sector frame rotated by alpha is (sin(psi-alpha) - sin(phi0-alpha))/C, so the
crossing with the plane x = x_r solves sin(psi-alpha) = sin(phi0-alpha) + C*x_r.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Detector geometry (pad-row layout of the configs: 159 rows at 85..247 cm, uniform pitch).
N_SECTORS = 36
N_ROWS = 159
X_FIRST = 85.0
X_LAST = 247.0
HALF_ANGLE_DEG = 10.0
Z_MAX = 250.0
LSB = 1.0 / 128.0
BZ = 0.5
R_OUT = 251.0
CLIGHT = 0.299792458e-2          # GeV / (T cm)
KB = -CLIGHT * BZ                # curvature per unit q/pT  [1/cm per c/GeV]
Z_MAX_LSB = int(round(Z_MAX / LSB))

ROW_X = X_FIRST + np.arange(N_ROWS) * (X_LAST - X_FIRST) / (N_ROWS - 1)
TAN_HALF = math.tan(math.radians(HALF_ANGLE_DEG))


def sector_alpha(k):
    """Centre angle of sector k (radians); sectors k and k+18 share the same phi."""
    return np.deg2rad(((np.asarray(k) % 18) + 0.5) * 2.0 * HALF_ANGLE_DEG)


def sector_side(k):
    """+1 for the A side (z > 0, sectors 0..17), -1 for the C side (18..35)."""
    return np.where(np.asarray(k) < 18, 1, -1)


def round_half_away(v):
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


@dataclasses.dataclass
class EventConfig:
    n_tracks: int
    noise_frac: float
    looper_frac: float = 0.0
    single_sector: bool = False
    seed: int = 0
    smear: float = 0.1
    theta: np.ndarray | None = None      # injected calibration [s_vd, d_0..35, a_0..35]
    # cluster inefficiency: rows without any cluster in every sector (inclusive ranges), and the
    # probability that a track crossing gives no cluster (drawn from a separate seeded stream, so
    # that the other draws of the event do not change)
    dead_rows: tuple = ()
    drop_frac: float = 0.0


@dataclasses.dataclass
class Event:
    pad_fp: np.ndarray        # int16  [N]   y / LSB in the sector frame
    time_fp: np.ndarray       # uint16 [N]   drift length / LSB
    charge: np.ndarray        # uint16 [N]   (not read by the tracking)
    bin_off: np.ndarray       # int32  [36*159+1] cluster ranges per (sector, row)
    mc_track: np.ndarray      # int32  [N]   generating track or -1 (noise)
    true_xyz: np.ndarray      # f64    [N,3] exact physical crossing point (sector frame)
    true_snp: np.ndarray      # f64    [N]   exact local sin(phi) of the helix at that point
    true_s: np.ndarray        # f64    [N]   transverse path length from the vertex to that point
    sector: np.ndarray        # int16  [N]
    row: np.ndarray           # int16  [N]
    trk_q: np.ndarray         # f64    [T]
    trk_pt: np.ndarray
    trk_eta: np.ndarray
    trk_phi0: np.ndarray
    config: EventConfig

    @property
    def n_clusters(self):
        return int(self.pad_fp.shape[0])


def theta_nominal():
    th = np.zeros(73)
    th[0] = 1.0
    return th


def _sample_pt(rng, n, n_loop):
    pt = np.empty(n)
    k = 0
    n_norm = n - n_loop
    while k < n_norm:
        v = rng.exponential(0.6, size=max(16, 2 * (n_norm - k)))
        v = v[v > 0.1][: n_norm - k]
        pt[k:k + v.size] = v
        k += v.size
    pt[n_norm:] = rng.uniform(0.05, 0.15, size=n_loop)
    return pt


def _crossings(phi0, C, tl, s_end, sectors, theta):
    """All plane crossings of helices (arrays over (track, sector) pairs) with the 159 rows.

    Returns per-crossing arrays (pair index, row, s, y_raw, x_phys, y_phys, sin phi_local)."""
    P = phi0.shape[0]
    alpha = sector_alpha(sectors)
    x = ROW_X[None, :]                                     # [1, R]
    a0 = (phi0 - alpha)[:, None]
    Cc = C[:, None]
    v = np.sin(a0) + Cc * x                                # sin(psi - alpha) at the crossing
    ok = np.abs(v) <= 1.0
    vb = np.clip(v, -1.0, 1.0)
    out = []
    for branch in (0, 1):
        b = np.arcsin(vb) if branch == 0 else math.pi - np.arcsin(vb)
        delta = alpha[:, None] + b - phi0[:, None]
        t = np.mod(delta, 2 * math.pi)
        t = np.where(Cc < 0, t - 2 * math.pi, t)
        s = t / Cc
        good = ok & (s > 0) & (s < s_end[:, None])
        pi, ri = np.nonzero(good)
        s = s[pi, ri]
        out.append((pi, ri, s))
    pi = np.concatenate([o[0] for o in out])
    ri = np.concatenate([o[1] for o in out])
    s = np.concatenate([o[2] for o in out])
    al = alpha[pi]
    ph = phi0[pi]
    Cv = C[pi]
    xr = ROW_X[ri]

    def local(sv):
        psi = ph + Cv * sv
        xl = (np.sin(psi - al) - np.sin(ph - al)) / Cv
        yl = (np.cos(ph - al) - np.cos(psi - al)) / Cv
        return xl, yl, np.cos(psi - al)

    if theta is not None:
        a_k = theta[37 + sectors[pi]]
        # The pad row collects the charge whose *raw* position lies on its plane: solve
        # raw_x(P(s)) = x_r with Newton steps from the undistorted crossing.
        for _ in range(6):
            xl, yl, cphi = local(s)
            rho_p = np.hypot(xl, yl)
            rho_r = (rho_p + 85.0 * a_k / 162.0) / (1.0 + a_k / 162.0)
            f = xl * rho_r / rho_p - xr
            s = s - np.clip(f / np.where(np.abs(cphi) > 1e-3, cphi, 1e-3), -1.0, 1.0)
        xl, yl, _ = local(s)
        rho_p = np.hypot(xl, yl)
        rho_r = (rho_p + 85.0 * a_k / 162.0) / (1.0 + a_k / 162.0)
        y_raw = yl * rho_r / rho_p
        # keep only converged solutions (near-tangent crossings are dropped)
        conv = np.abs(xl * rho_r / rho_p - xr) < 1e-9
        pi, ri, s, xr = pi[conv], ri[conv], s[conv], xr[conv]
        xl, yl, y_raw = xl[conv], yl[conv], y_raw[conv]
        ph, Cv, al = ph[conv], Cv[conv], al[conv]
    else:
        xl, yl, _ = local(s)
        y_raw = yl
    snp = np.sin(ph + Cv * s - al)
    return pi, ri, s, y_raw, xl, yl, snp


def make_event(cfg: EventConfig) -> Event:
    rng = np.random.default_rng(cfg.seed)
    n = int(cfg.n_tracks)
    n_loop = int(round(cfg.looper_frac * n))
    q = rng.choice(np.array([-1.0, 1.0]), size=n)
    pt = _sample_pt(rng, n, n_loop)
    eta = rng.uniform(-0.9, 0.9, size=n)
    if cfg.single_sector:
        eta = np.abs(eta)
        phi0 = rng.uniform(0.0, math.radians(2 * HALF_ANGLE_DEG), size=n)
    else:
        phi0 = rng.uniform(0.0, 2 * math.pi, size=n)
    theta = None if cfg.theta is None else np.asarray(cfg.theta, dtype=np.float64)

    C = KB * q / pt
    tl = np.sinh(eta)
    absC = np.abs(C)
    turn = 2 * math.pi / absC
    v_out = R_OUT * absC / 2
    s_exit = np.where(v_out < 1, 2 * np.arcsin(np.minimum(v_out, 1.0)) / absC, turn)
    s_z = np.where(tl != 0, Z_MAX / np.maximum(np.abs(tl), 1e-300), np.inf)
    s_end = np.minimum(np.minimum(s_exit, s_z), turn)
    v_in = X_FIRST * absC / 2
    reach = v_in < 1
    s_in = np.where(reach, 2 * np.arcsin(np.minimum(v_in, 1.0)) / absC, 0.0)
    s_last = np.minimum(s_end, turn - s_in)
    # Position angle of a circle through the origin is phi0 + C*s/2: it fixes the sector.
    ph_a = phi0 + C * s_in / 2
    ph_b = phi0 + C * s_last / 2
    w = math.radians(2 * HALF_ANGLE_DEG)
    j_lo = np.floor(np.minimum(ph_a, ph_b) / w).astype(np.int64) - 1
    j_hi = np.floor(np.maximum(ph_a, ph_b) / w).astype(np.int64) + 1
    side_off = np.where(tl >= 0, 0, 18)
    live = np.nonzero(reach & (s_last > s_in))[0]
    span = j_hi[live] - j_lo[live] + 1
    width = int(min(max(span.max(initial=1), 1), 18))
    jj = j_lo[live][:, None] + np.arange(width)[None, :]
    ok = np.arange(width)[None, :] < np.minimum(span, 18)[:, None]
    pt_i = np.broadcast_to(live[:, None], jj.shape)[ok]
    ks = np.mod(jj[ok], 18)
    if cfg.single_sector:
        sel = ks == 0
        pt_i, ks = pt_i[sel], ks[sel]
    # one (track, sector) pair per distinct sector
    uniq = np.unique(pt_i.astype(np.int64) * 18 + ks)
    pair_trk = uniq // 18
    pair_sec = uniq % 18 + side_off[pair_trk]

    sig_trk, sig_sec, sig_row, sig_y, sig_d, sig_true = [], [], [], [], [], []
    chunk = 8192
    for c0 in range(0, pair_trk.size, chunk):
        tr = pair_trk[c0:c0 + chunk]
        se = pair_sec[c0:c0 + chunk]
        pi, ri, s, y_raw, xl, yl, snp = _crossings(phi0[tr], C[tr], tl[tr], s_end[tr], se, theta)
        t_i = tr[pi]
        k_i = se[pi]
        z = s * tl[t_i]
        side = sector_side(k_i)
        keep = (np.abs(y_raw) <= ROW_X[ri] * TAN_HALF) & (np.abs(z) <= Z_MAX)
        keep &= np.where(side > 0, z >= 0, z < 0)
        t_i, k_i, ri, y_raw, z, side = t_i[keep], k_i[keep], ri[keep], y_raw[keep], z[keep], side[keep]
        xl, yl, snp = xl[keep], yl[keep], snp[keep]
        if theta is not None:
            d_raw = (Z_MAX - side * (z - theta[1 + k_i])) / theta[0]
        else:
            d_raw = Z_MAX - side * z
        sig_trk.append(t_i)
        sig_sec.append(k_i)
        sig_row.append(ri)
        sig_y.append(y_raw)
        sig_d.append(d_raw)
        sig_true.append(np.stack([xl, yl, z, snp, s[keep]], axis=1))
    if sig_trk:
        sig_trk = np.concatenate(sig_trk)
        sig_sec = np.concatenate(sig_sec)
        sig_row = np.concatenate(sig_row)
        sig_y = np.concatenate(sig_y)
        sig_d = np.concatenate(sig_d)
        sig_true = np.concatenate(sig_true)
    else:
        sig_trk = np.zeros(0, np.int64)
        sig_sec = sig_row = sig_trk.copy()
        sig_y = sig_d = np.zeros(0)
        sig_true = np.zeros((0, 5))
    # Generation order: deterministic (track, sector, row) order before smearing.
    o = np.argsort((sig_trk * N_SECTORS + sig_sec) * N_ROWS + sig_row, kind="stable")
    sig_trk, sig_sec, sig_row = sig_trk[o], sig_sec[o], sig_row[o]
    sig_y, sig_d, sig_true = sig_y[o], sig_d[o], sig_true[o]
    ns = sig_trk.size
    y_m = sig_y + rng.normal(0.0, cfg.smear, size=ns) if cfg.smear > 0 else sig_y.copy()
    d_m = sig_d + rng.normal(0.0, cfg.smear, size=ns) if cfg.smear > 0 else sig_d.copy()
    inside = (d_m >= 0.0) & (d_m <= Z_MAX)
    sig_trk, sig_sec, sig_row = sig_trk[inside], sig_sec[inside], sig_row[inside]
    y_m, d_m, sig_true = y_m[inside], d_m[inside], sig_true[inside]
    ns = sig_trk.size

    if cfg.drop_frac > 0 or cfg.dead_rows:
        keep = np.ones(ns, bool)
        if cfg.drop_frac > 0:
            keep &= np.random.default_rng([cfg.seed, 0x1eaf]).random(ns) >= cfg.drop_frac
        for r0, r1 in cfg.dead_rows:
            keep &= (sig_row < r0) | (sig_row > r1)
        sig_trk, sig_sec, sig_row = sig_trk[keep], sig_sec[keep], sig_row[keep]
        y_m, d_m, sig_true = y_m[keep], d_m[keep], sig_true[keep]
        ns = sig_trk.size

    n_noise = int(round(cfg.noise_frac * ns))
    if cfg.single_sector:
        nz_sec = np.zeros(n_noise, np.int64)
    else:
        nz_sec = rng.integers(0, N_SECTORS, size=n_noise)
    nz_row = rng.integers(0, N_ROWS, size=n_noise)
    ymax = ROW_X[nz_row] * TAN_HALF
    nz_y = rng.uniform(-1.0, 1.0, size=n_noise) * ymax
    nz_d = rng.uniform(0.0, Z_MAX, size=n_noise)
    if cfg.dead_rows:
        alive = np.ones(n_noise, bool)
        for r0, r1 in cfg.dead_rows:
            alive &= (nz_row < r0) | (nz_row > r1)
        nz_sec, nz_row, nz_y, nz_d = nz_sec[alive], nz_row[alive], nz_y[alive], nz_d[alive]
        n_noise = int(alive.sum())

    sec = np.concatenate([sig_sec, nz_sec]).astype(np.int64)
    row = np.concatenate([sig_row, nz_row]).astype(np.int64)
    pad = round_half_away(np.concatenate([y_m, nz_y]) / LSB).astype(np.int64)
    tim = round_half_away(np.concatenate([d_m, nz_d]) / LSB).astype(np.int64)
    tim = np.clip(tim, 0, Z_MAX_LSB)
    mc = np.concatenate([sig_trk, np.full(n_noise, -1)]).astype(np.int64)
    true_xyz = np.concatenate([sig_true, np.full((n_noise, 5), np.nan)])
    charge = rng.integers(20, 1000, size=sec.size)
    # (sector, row, pad, time) order; the stable sort keeps generation order for equal keys.
    key = (((sec * N_ROWS + row) << 16) + (pad + 32768)) << 16 | tim
    o = np.argsort(key, kind="stable")
    sec, row, pad, tim, mc = sec[o], row[o], pad[o], tim[o], mc[o]
    true_snp = true_xyz[o, 3].copy()
    true_s = true_xyz[o, 4].copy()
    true_xyz, charge = true_xyz[o, :3].copy(), charge[o]
    b = sec * N_ROWS + row
    bin_off = np.searchsorted(b, np.arange(N_SECTORS * N_ROWS + 1), side="left").astype(np.int32)
    return Event(pad_fp=pad.astype(np.int16), time_fp=tim.astype(np.uint16),
                 charge=charge.astype(np.uint16), bin_off=bin_off, mc_track=mc.astype(np.int32),
                 true_xyz=true_xyz, true_snp=true_snp, true_s=true_s, sector=sec.astype(np.int16), row=row.astype(np.int16),
                 trk_q=q, trk_pt=pt, trk_eta=eta, trk_phi0=phi0, config=cfg)


# --- named workloads -------------------------------------------------------------------------

def single_sector(seed=1001, n_tracks=200):
    """Single sector: 200 tracks, 10 % noise, all folded into sector 0."""
    return EventConfig(n_tracks=n_tracks, noise_frac=0.10, single_sector=True, seed=seed)


def full_event(seed=1002, n_tracks=5000):
    """Full 36-sector event: 5,000 tracks, 15 % noise."""
    return EventConfig(n_tracks=n_tracks, noise_frac=0.15, seed=seed)


def central_event(seed=1003, n_tracks=20000):
    """Central-Pb-Pb-shaped event: 20,000 tracks incl. 10 % low-pT loopers, 30 % noise."""
    return EventConfig(n_tracks=n_tracks, noise_frac=0.30, looper_frac=0.10, seed=seed)


def inefficient_central(seed=1006, n_tracks=20000):
    """The central-shaped event with cluster inefficiency: 5 % of the track crossings give no
    cluster (single-row gaps) and two ranges of dead pad rows in every sector, rows 60-61 (a gap
    the following bridges, the neighbour finding does not) and rows 100-111 (twelve rows, more than
    the following bridges)."""
    return EventConfig(n_tracks=n_tracks, noise_frac=0.30, looper_frac=0.10, seed=seed,
                       dead_rows=((60, 61), (100, 111)), drop_frac=0.05)


def batch_configs(n_events=64, seed0=2000):
    """Batched workload: multiplicities log-uniform in [100, 20000], 20 % noise."""
    rng = np.random.default_rng(seed0)
    mult = np.floor(np.exp(rng.uniform(math.log(100), math.log(20000), size=n_events))).astype(int)
    return [EventConfig(n_tracks=int(m), noise_frac=0.20, looper_frac=0.10, seed=seed0 + e)
            for e, m in enumerate(mult)]


def calib_theta(seed=1005):
    """Injected calibration: drift-velocity scale 1.003, d_k ~ N(0, 0.05 cm), a_k ~ N(0, 0.1 cm)."""
    rng = np.random.default_rng(seed)
    th = np.empty(73)
    th[0] = 1.003
    th[1:37] = rng.normal(0.0, 0.05, size=36)
    th[37:73] = rng.normal(0.0, 0.1, size=36)
    return th


def calib_event(seed=1005, n_tracks=20000):
    """Central event with the injected calibration distortion."""
    return EventConfig(n_tracks=n_tracks, noise_frac=0.30, looper_frac=0.10, seed=seed,
                       theta=calib_theta(seed))


# Resolutions of the reference track at the vertex (inner-tracker-like): vertex point, z0, tan
# lambda, relative q/pT.
REF_SIGMA_V = 0.01
REF_SIGMA_Z0 = 0.01
REF_SIGMA_TL = 1e-3
REF_SIGMA_QPT_REL = 0.01


def vertex_references(ev: Event, trk_off, trk_hits, seed=1006, purity=0.9, smear=True, max_first_row=8,
                      min_hits=30):
    """Reference measurements at the vertex for reconstructed tracks, as float64 [T, 8] in the
    layout of the refit's anchor input: (sigma_v, z0, sigma_z0, tan lambda, sigma_tl, q/pT,
    sigma_qpt, 0).  A track is matched to the generating particle that holds at least `purity` of
    its hits, provided the track runs along the particle's outgoing path (the particle's path
    length from the vertex increases along the track's hit order; the returning leg of a looper
    points away from the vertex and gets no reference) and the particle's direction at the vertex
    is within |sin phi| < 0.9 of the first hit's sector frame.  As in a matching at the inner wall
    of the TPC, only tracks that start within the first `max_first_row` pad rows and have at least
    `min_hits` hits are matched.  The reference values are that particle's
    (z0 = 0, tan lambda = sinh eta, q/pT) smeared with seeded Gaussian noise (exact values if smear
    is False).  Unmatched tracks get a zero record (no reference)."""
    trk_off = np.asarray(trk_off)
    trk_hits = np.asarray(trk_hits)
    nt = trk_off.shape[0] - 1
    rng = np.random.default_rng(seed)
    noise = rng.normal(0.0, 1.0, size=(nt, 3)) if smear else np.zeros((nt, 3))
    out = np.zeros((nt, 8))
    for t in range(nt):
        lab = ev.mc_track[trk_hits[trk_off[t]:trk_off[t + 1]]]
        lab = lab[lab >= 0]
        if lab.size == 0:
            continue
        vals, cnt = np.unique(lab, return_counts=True)
        p = int(vals[np.argmax(cnt)])
        if cnt.max() < purity * (trk_off[t + 1] - trk_off[t]):
            continue
        own = trk_hits[trk_off[t]:trk_off[t + 1]]
        if own.size < min_hits or int(ev.row[own[0]]) > max_first_row:
            continue
        path = ev.true_s[own[ev.mc_track[own] == p]]
        if path.size < 2 or not np.all(np.diff(path) > 0):
            continue
        # the step to the vertex runs in the frame of the first hit's sector: keep it well inside
        # the local parametrisation (|sin phi| < 0.9 at the vertex)
        if abs(math.sin(ev.trk_phi0[p] - sector_alpha(int(ev.sector[own[0]])))) >= 0.9:
            continue
        tl = math.sinh(ev.trk_eta[p])
        qpt = ev.trk_q[p] / ev.trk_pt[p]
        sq = REF_SIGMA_QPT_REL * abs(qpt)
        out[t] = (REF_SIGMA_V, REF_SIGMA_Z0 * noise[t, 0], REF_SIGMA_Z0, tl + REF_SIGMA_TL * noise[t, 1],
                  REF_SIGMA_TL, qpt + sq * noise[t, 2], sq, 0.0)
    return out


# ITS-like reference tracks (the inner tracker's tracks, matched to TPC tracks for the drift
# calibration, sections 2.1 and 6 of the paper): resolution of the direction at the vertex, of z0,
# tan lambda and q/pT, efficiency per particle, and the fraction of fake tracks
ITS_SIGMA_PHI = 1e-3
ITS_SIGMA_Z0 = 0.01
ITS_SIGMA_TL = 1e-3
ITS_SIGMA_QPT_REL = 0.01
ITS_EFF = 0.95
ITS_FAKE_FRAC = 0.02


def its_tracks(ev: Event, seed=1007, eff=ITS_EFF, fake_frac=ITS_FAKE_FRAC, smear=True):
    """Reference tracks of the inner tracker for the particles of ev, as float64 [n_its, 8]:
    (phi0, z0, tan lambda, q/pT, sigma_phi0, sigma_z0, sigma_tl, sigma_qpt) at the production vertex
    (global azimuth of the momentum, z at the vertex, exactly 0 for a true track).  Each particle
    gives a track with probability `eff`, smeared with seeded Gaussian noise (exact if smear is
    False); fake tracks, a `fake_frac` share, take the kinematics of random particles with a random
    azimuth and z0 ~ N(0, 5 cm).  Returns (tracks, particle index or -1 for fakes).  The rows come
    in a random order (no relation to the particle order)."""
    rng = np.random.default_rng(seed)
    npart = len(ev.trk_pt)
    keep = np.nonzero(rng.random(npart) < eff)[0]
    n_fake = int(round(fake_frac * keep.size))
    noise = rng.normal(0.0, 1.0, size=(keep.size, 4)) if smear else np.zeros((keep.size, 4))
    tl = np.sinh(ev.trk_eta[keep])
    qpt = ev.trk_q[keep] / ev.trk_pt[keep]
    sq = ITS_SIGMA_QPT_REL * np.abs(qpt)
    rec = np.stack([np.mod(ev.trk_phi0[keep] + ITS_SIGMA_PHI * noise[:, 0], 2 * math.pi),
                    ITS_SIGMA_Z0 * noise[:, 1], tl + ITS_SIGMA_TL * noise[:, 2], qpt + sq * noise[:, 3],
                    np.full(keep.size, ITS_SIGMA_PHI), np.full(keep.size, ITS_SIGMA_Z0),
                    np.full(keep.size, ITS_SIGMA_TL), sq], axis=1)
    if n_fake and npart:
        src = rng.integers(0, npart, n_fake)
        ftl = np.sinh(ev.trk_eta[src])
        fq = ev.trk_q[src] / ev.trk_pt[src]
        fake = np.stack([rng.uniform(0.0, 2 * math.pi, n_fake), rng.normal(0.0, 5.0, n_fake), ftl, fq,
                         np.full(n_fake, ITS_SIGMA_PHI), np.full(n_fake, ITS_SIGMA_Z0),
                         np.full(n_fake, ITS_SIGMA_TL), ITS_SIGMA_QPT_REL * np.abs(fq)], axis=1)
        rec = np.concatenate([rec, fake])
        part = np.concatenate([keep, np.full(n_fake, -1)])
    else:
        part = keep
    o = rng.permutation(rec.shape[0])
    return rec[o], part[o].astype(np.int64)


@dataclasses.dataclass
class Batch:
    pad_fp: np.ndarray
    time_fp: np.ndarray
    charge: np.ndarray
    bin_off: np.ndarray       # int32 [n_events*36*159+1], global offsets
    ev_off: np.ndarray        # int64 [n_events+1] cluster offsets per event
    events: list

    @property
    def n_events(self):
        return len(self.events)

    @property
    def n_clusters(self):
        return int(self.pad_fp.shape[0])


def concat_events(events) -> Batch:
    ev_off = np.zeros(len(events) + 1, np.int64)
    for i, e in enumerate(events):
        ev_off[i + 1] = ev_off[i] + e.n_clusters
    nb = N_SECTORS * N_ROWS
    bin_off = np.empty(len(events) * nb + 1, np.int64)
    for i, e in enumerate(events):
        bin_off[i * nb:(i + 1) * nb] = e.bin_off[:nb].astype(np.int64) + ev_off[i]
    bin_off[-1] = ev_off[-1]
    if ev_off[-1] >= 2**31:
        raise ValueError("batch exceeds 2^31 clusters")
    return Batch(pad_fp=np.concatenate([e.pad_fp for e in events]),
                 time_fp=np.concatenate([e.time_fp for e in events]),
                 charge=np.concatenate([e.charge for e in events]),
                 bin_off=bin_off.astype(np.int32), ev_off=ev_off, events=list(events))


# ---- continuous readout: time frames sliced along the drift-time axis -------------------------

DRIFT_LSB = 32000          # one full drift length in LSB (250 cm / LSB)


@dataclasses.dataclass
class TimeFrame:
    """Collisions overlaid in one continuous readout stream and cut into slices of slice_len LSB
    of readout time.  Readout time of a cluster = t0 of its collision + its drift length (both in
    LSB of drift length).  Slice j holds the clusters with j*slice_len <= time < (j+1)*slice_len,
    with time_fp = time - j*slice_len; inside a slice the clusters are sorted by (sector, row, pad,
    time_fp, collision, index in the collision), and the slices are concatenated in order."""
    pad_fp: np.ndarray        # int16  [N]
    time_fp: np.ndarray       # uint16 [N] slice-local readout time
    bin_off: np.ndarray       # int32  [n_slices*36*159+1] global cluster offsets per (slice, sector, row)
    ev_off: np.ndarray        # int64  [n_slices+1] cluster offsets per slice
    slice_len: int
    t0: np.ndarray            # int64  [K] collision times
    mc: np.ndarray            # int64  [N] collision << 32 | generating track, or -1 (noise)
    collisions: list

    @property
    def n_slices(self):
        return int(self.ev_off.shape[0] - 1)

    @property
    def n_clusters(self):
        return int(self.pad_fp.shape[0])


def time_frame(events, per_drift=5.0, slice_len=DRIFT_LSB, seed=3000, t0=None) -> TimeFrame:
    """Overlay the events at collision times of a Poisson process with per_drift collisions per
    drift length on average (the first at time 0), or at the given times t0, and slice the
    stream."""
    if not 1 <= slice_len <= Z_MAX_LSB + 1:      # slice-local times stay inside [0, Z_MAX_LSB]
        raise ValueError("slice_len must lie in [1, %d]" % (Z_MAX_LSB + 1))
    K = len(events)
    if t0 is None:
        rng = np.random.default_rng(seed)
        gaps = rng.exponential(DRIFT_LSB / per_drift, size=K)
        gaps[0] = 0.0
        t0 = np.floor(np.cumsum(gaps)).astype(np.int64)
    t0 = np.asarray(t0, np.int64)
    if t0.shape != (K,) or (K and t0.min() < 0):
        raise ValueError("t0 must hold one non-negative time per event")
    nb = N_SECTORS * N_ROWS
    parts = []
    for k, e in enumerate(events):
        n = e.n_clusters
        b = np.repeat(np.arange(nb), np.diff(e.bin_off[:nb + 1].astype(np.int64)))
        tau = t0[k] + e.time_fp.astype(np.int64)
        mc = np.where(e.mc_track >= 0, (np.int64(k) << 32) | e.mc_track.astype(np.int64), -1)
        parts.append((b, e.pad_fp.astype(np.int64), tau, np.full(n, k, np.int64), np.arange(n, dtype=np.int64), mc))
    b, pad, tau, col, idx, mc = (np.concatenate([p[i] for p in parts]) for i in range(6))
    sl = tau // slice_len
    loc = tau - sl * slice_len
    n_sl = int(sl.max()) + 1 if sl.size else 1
    gbin = sl * nb + b
    o = np.lexsort((idx, col, loc, pad, gbin))
    gbin, pad, loc, mc = gbin[o], pad[o], loc[o], mc[o]
    bin_off = np.searchsorted(gbin, np.arange(n_sl * nb + 1), side="left")
    if bin_off[-1] >= 2**31:
        raise ValueError("time frame exceeds 2^31 clusters")
    ev_off = bin_off[::nb].astype(np.int64)
    return TimeFrame(pad_fp=pad.astype(np.int16), time_fp=loc.astype(np.uint16), bin_off=bin_off.astype(np.int32),
                     ev_off=ev_off, slice_len=int(slice_len), t0=t0, mc=mc, collisions=list(events))


def track_quality(ev: Event, trk_off, trk_hits, min_pt=0.3, min_hits=30, purity=0.9, coverage=0.8):
    """Truth matching of reconstructed tracks (a sanity figure; the paper prints none for these
    events).  A generating particle with pT > min_pt and at least min_hits clusters, not a looper
    (pT > 0.15 GeV), is found whole when one track holds at least `coverage` of its clusters and
    at least `purity` of that track's hits are its clusters.  Returns (efficiency, particles, fake
    fraction of tracks below `purity`)."""
    trk_off = np.asarray(trk_off)
    trk_hits = np.asarray(trk_hits)
    nt = trk_off.shape[0] - 1
    n_of = np.bincount(ev.mc_track[ev.mc_track >= 0], minlength=len(ev.trk_pt))
    want = (ev.trk_pt > max(min_pt, 0.15)) & (n_of >= min_hits)
    found = np.zeros(len(ev.trk_pt), bool)
    fakes = 0
    for t in range(nt):
        lab = ev.mc_track[trk_hits[trk_off[t]:trk_off[t + 1]]]
        n = lab.size
        lab = lab[lab >= 0]
        if lab.size == 0:
            fakes += 1
            continue
        vals, cnt = np.unique(lab, return_counts=True)
        k = int(np.argmax(cnt))
        p, c = int(vals[k]), int(cnt[k])
        if c < purity * n:
            fakes += 1
            continue
        if c >= coverage * n_of[p]:
            found[p] = True
    n_want = int(want.sum())
    return float(found[want].sum() / max(n_want, 1)), n_want, fakes / max(nt, 1)
