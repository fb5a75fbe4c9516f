"""Calibration feedback as gradient steps (the online calibration loop of sections 2 and 6, turned
into an optimisation of the refit's sum of chi2 over the transformation parameters).

theta = [s_vd, d_0..d_35, a_0..a_35]; the objective and its gradient come from tpc_refit_grad
(FP32 Kalman refit + hand-written adjoint, FP64 reductions).  The steps are preconditioned by the
Hessian at the starting point, built from central differences of the adjoint gradient (2 x 73
gradient calls), so that the three parameter blocks with their different units move together:

    theta_{k+1} = theta_k - H0^-1 grad f(theta_k)

The statistical precision of the result is sqrt(diag(2 H^-1)) (sum chi2 is -2 log L up to a
constant).  Host logic only: every evaluation runs through the C ABI.
"""
from __future__ import annotations

import dataclasses
import json
import os

import numpy as np
import torch

# central-difference steps of the Hessian, per block (s_vd, d_k [cm], a_k [cm]): z shifts of up to
# 0.025 cm, large against the FP32 rounding of the per-track sums and small against the ~1 cm reach
# of the objective's quadratic region
HESS_STEP = (1e-4, 1e-2, 1e-2)


@dataclasses.dataclass
class CalibResult:
    theta: np.ndarray           # final parameters
    history: list               # (step, sum chi2, |grad|) per evaluation
    hessian: np.ndarray         # preconditioner at the start
    sigma: np.ndarray           # statistical precision sqrt(diag(2 H^-1))


class Objective:
    """f(theta) and its gradient through the C ABI for fixed tracks, weights and references.
    error_model 1 (raw errors carried through the transformation) is the unbiased choice for a
    calibration: with fixed calibrated errors a theta that shrinks the data also shrinks the
    residuals."""

    def __init__(self, context, clusters, tracks, weight=None, anchor=None, error_model=1):
        self.context, self.clusters, self.tracks = context, clusters, tracks
        self.weight, self.anchor, self.error_model = weight, anchor, error_model
        self.s = torch.empty(1, dtype=torch.float64, device="cuda")
        self.n_calls = 0

    def __call__(self, theta):
        th = torch.as_tensor(np.asarray(theta, np.float64), device="cuda")
        g = torch.empty_like(th)
        self.context.tpc_refit_grad(self.clusters, self.tracks, th, self.s, g, self.weight, self.anchor,
                                    self.error_model)
        st = self.context.tpc_sync_status()
        if st != 0:
            raise RuntimeError("tpc_refit_grad device status %d" % st)
        self.n_calls += 1
        return float(self.s.item()), g.cpu().numpy()


    def track_chi2(self, theta):
        """Per-track weighted chi2 at theta (the records of the refit, device -> host)."""
        self(theta)
        nt = int(self.tracks.n_tracks.item())
        rec = torch.empty(max(nt, 1) * REC_WORDS, dtype=torch.float32, device="cuda")
        self.context.tpc_debug_copy(11, rec)
        return rec.view(-1, REC_WORDS)[:nt, 0].cpu().numpy().astype(np.float64)


REC_WORDS = 26          # per-track record of the refit (see tpc_debug_copy)


def reject_references(context, clusters, tracks, weight, ref, theta, error_model=1, cut=25.0):
    """Drop the reference of every track whose reference terms add more than `cut` to its chi2
    at theta (a wrong match); returns the new [T, 8] reference array and the number dropped."""
    with_ref = Objective(context, clusters, tracks, weight,
                         torch.tensor(ref.astype(np.float32), device="cuda"), error_model)
    without = Objective(context, clusters, tracks, weight, None, error_model)
    d = with_ref.track_chi2(theta) - without.track_chi2(theta)
    bad = (ref[:, 0] > 0) & (d > cut)
    out = ref.copy()
    out[bad] = 0.0
    return out, int(bad.sum())


def hessian(f, theta, steps=HESS_STEP, n_sectors=36):
    """Symmetrised Hessian by central differences of the gradient."""
    n = theta.shape[0]
    H = np.empty((n, n))
    for j in range(n):
        h = steps[0] if j == 0 else (steps[1] if j <= n_sectors else steps[2])
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        H[:, j] = (f(tp)[1] - f(tm)[1]) / (2 * h)
    return 0.5 * (H + H.T)


def calibrate(context, clusters, tracks, weight, ref, theta0, steps=20, error_model=1, cut=25.0):
    """The calibration loop: half of the steps with all references, then the references whose
    chi2 exceeds `cut` are dropped and the other half runs from there (Hessian re-taken)."""
    a = torch.tensor(ref.astype(np.float32), device="cuda")
    f1 = Objective(context, clusters, tracks, weight, a, error_model)
    r1 = fit_calibration(f1, theta0, steps=steps // 2)
    ref2, n_drop = reject_references(context, clusters, tracks, weight, ref, r1.theta, error_model, cut)
    f2 = Objective(context, clusters, tracks, weight, torch.tensor(ref2.astype(np.float32), device="cuda"),
                   error_model)
    r2 = fit_calibration(f2, r1.theta, steps=steps - steps // 2)
    r2.history = r1.history + r2.history
    return r2, n_drop, f1.n_calls + f2.n_calls


def fit_calibration(f, theta0, steps=20, H=None):
    """`steps` preconditioned gradient steps from theta0 (H: preconditioner, default the Hessian
    at theta0)."""
    theta = np.asarray(theta0, np.float64).copy()
    if H is None:
        H = hessian(f, theta)
    Hinv = np.linalg.inv(H)
    history = []
    for k in range(steps):
        val, g = f(theta)
        history.append((k, val, float(np.linalg.norm(g))))
        theta = theta - Hinv @ g
    val, g = f(theta)
    history.append((steps, val, float(np.linalg.norm(g))))
    sigma = np.sqrt(np.maximum(np.diag(2.0 * Hinv), 0.0))
    return CalibResult(theta=theta, history=history, hessian=H, sigma=sigma)


def save_theta(path, theta, n_sectors=36, meta=None):
    """Store a calibration (the calibration objects of the paper's online loop are kept for offline
    use) as JSON: s_vd, d_k and a_k by name, plus free-form metadata."""
    th = np.asarray(theta, np.float64)
    assert th.shape == (1 + 2 * n_sectors,)
    doc = {"s_vd": float(th[0]), "d": th[1:1 + n_sectors].tolist(), "a": th[1 + n_sectors:].tolist(),
           "meta": meta or {}}
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
    os.replace(tmp, path)


def load_theta(path):
    """Inverse of save_theta: the float64 theta vector [s_vd, d_0.., a_0..]."""
    doc = json.load(open(path))
    return np.concatenate([[doc["s_vd"]], doc["d"], doc["a"]]).astype(np.float64)
