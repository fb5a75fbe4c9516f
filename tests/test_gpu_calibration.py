"""Calibration recovery on the GPU: the central event with an injected calibration (drift-velocity
scale 1.003, per-sector z offsets ~N(0, 0.05 cm), radial distortions ~N(0, 0.1 cm), seed 1005) is
tracked, and 20 preconditioned gradient steps of the refit's -2 log L (raw measurement errors
carried through the transformation, plus the reference measurements at the vertex; references
with chi2 > 25 dropped after the first 10 steps) move theta from the nominal values to the
injected ones.

The bar: every parameter within 5 statistical standard errors sigma = sqrt(diag(2 H^-1)) of its
injected value, and in each block (s_vd, d_k, a_k) a remaining distortion |theta - theta*| no
larger than 3 times its statistical expectation sqrt(sum sigma^2) (for d_k the expectation is
about 8 % of the injected distortion: 0.004 cm per sector against offsets of 0.05 cm).  Without the
references the Hessian has near-null directions (per-side z shift with the drift-velocity scale,
and the pure radial scale), which is why they are part of the objective."""
import numpy as np
import pytest
import torch

from paper_1712_09434_gb300 import calib, synth
from tests import _events, _gpu

pytestmark = pytest.mark.gpu

BLOCKS = (slice(0, 1), slice(1, 37), slice(37, 73))


def _setup():
    ev = _events.event("c5")
    ctx = _gpu.make_context(ev.n_clusters, 1)
    cl = _gpu.clusters_of(ev)
    g = _gpu.run(ctx, cl)
    nt = g["n_tracks"]
    ok = (g["ndf"] > 0) & (g["chi2"] < 5.0 * np.maximum(g["ndf"], 1))
    w = torch.tensor(ok.astype(np.float32), device="cuda")
    ref = synth.vertex_references(ev, g["trk_off"], g["trk_hits"])
    anchor = torch.tensor(ref.astype(np.float32), device="cuda")
    return ev, ctx, cl, g, w, anchor, nt, ref


def test_calibration_recovered_in_20_gradient_steps():
    ev, ctx, cl, g, w, anchor, nt, ref = _setup()
    th_star = synth.calib_theta(1005)
    th0 = synth.theta_nominal()
    res, n_drop, n_calls = calib.calibrate(ctx, cl, g["tracks_obj"], w, ref, th0, steps=20)
    pull = (res.theta - th_star) / res.sigma
    frac = [np.linalg.norm(res.theta[b] - th_star[b]) / np.linalg.norm(th0[b] - th_star[b]) for b in BLOCKS]
    expect = [np.sqrt(np.sum(res.sigma[b] ** 2)) / np.linalg.norm(th0[b] - th_star[b]) for b in BLOCKS]
    ev_ref = np.linalg.eigvalsh(res.hessian)
    f0 = calib.Objective(ctx, cl, g["tracks_obj"], w, None)
    ev_noref = np.linalg.eigvalsh(calib.hessian(f0, th0))
    print("tracks %d, weighted %d, with references %d (%d dropped), %d calls" % (
        nt, int(w.sum().item()), int((ref[:, 0] > 0).sum()), n_drop, n_calls))
    print("sum chi2 per step:", ["%.1f" % h[1] for h in res.history])
    print("remaining distortion per block (s_vd, d, a):", np.round(frac, 5), "statistical expectation",
          np.round(expect, 5))
    print("max |pull| per block:", [float(np.abs(pull[b]).max()) for b in BLOCKS])
    print("sigma per block (median):", [float(np.median(res.sigma[b])) for b in BLOCKS])
    print("Hessian eigenvalues, smallest 3: with references %s, without %s" % (ev_ref[:3], ev_noref[:3]))
    assert ev_ref[0] > 0.0, ev_ref[:3]
    assert res.history[-1][1] < res.history[0][1]
    assert np.all(np.array(frac) < 3.0 * np.array(expect)), (frac, expect)
    assert np.all(np.abs(pull) < 5.0), pull
    ctx.close()
