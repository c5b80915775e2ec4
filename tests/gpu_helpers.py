"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI.

check() asserts a measured error against its tolerance and, when the
environment variable SCGR_PARITY_LOG names a file, appends the measurement
to it (one JSON object per line: test id, quantity, value, tolerance), so
that a GPU run states the error of every result against the FP64 oracle
(tests/parity_report.py tabulates the log).

check_rows() adds the per-row view of a force check: a relative L2 over many
rows can hide a single row whose sum cancels, so every checked row i must meet

    |f_got,i - f_i| / |f_i| <= C_ROW * 2^-24 * kappa'_i,
    kappa'_i = sum_j w_ij (|X_j - c| + |Y_i - c|) / |f_i|,

with c the reference mean (the frame in which the kernel accumulates
sum_j w_ij X_j and sum_j w_ij, whose difference is f_i).  kappa'_i is at least
the condition number kappa_i = sum_j |w_ij r_ij| / |f_i| of the Eq. 5 sum (the
triangle inequality), which is logged beside it.  The bound counts the
rounding of each pair weight (ex2, sqrt, a few products: < 8 ulp), the
float32 tile sums under Kahan compensation across tiles, and the squared
distance evaluated as |X'|^2 + |Y'|^2 - 2 X'.Y', whose absolute error
(about 2^-24 (|X'|^2 + |Y'|^2)) enters f_i only through w_ij r_ij and so
stays within the same magnitude sums; C_ROW = 64 leaves room for all of them.
W_i is a sum of positive terms (condition 1): its per-row relative error must
stay below C_ROW * 2^-24."""
import json
import math
import os

import numpy as np
import torch

from paper_1902_01061_gb300 import scgr


def rot_err_deg(Ra, Rb):
    """angle of Ra^T Rb in degrees, from the chord: ||Ra - Rb||_F = 2 sqrt(2) sin(angle / 2)
    (accurate for small angles, where the arccos of the trace is not)"""
    chord = float(np.linalg.norm(np.asarray(Ra, np.float64) - np.asarray(Rb, np.float64)))
    return math.degrees(2.0 * math.asin(min(1.0, chord / (2.0 * math.sqrt(2.0)))))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


C_ROW = 64.0
EPS32 = 2.0 ** -24


def check_rows(what, got4, f_ref, W_ref, Y, X, aY, aX, sigma, p, g_mode, rows=None):
    """Per-row force parity (see the module docstring).  got4: GPU rows
    (fx, fy, fz, W) for template rows `rows` (all if None) of the template at
    positions Y; f_ref, W_ref: the oracle's values for the same rows.
    Returns (worst per-row relative error of f, worst kappa_i)."""
    import oracle as O
    got4 = np.asarray(got4, np.float64)
    f_ref = np.asarray(f_ref, np.float64)
    W_ref = np.asarray(W_ref, np.float64)
    Y = np.asarray(Y, np.float64)
    X = np.asarray(X, np.float64)
    c = X.mean(axis=0)
    rows_idx = np.arange(len(Y)) if rows is None else np.asarray(rows)
    A, B, Wm = O.force_row_magnitudes(Y, X, aY, aX, sigma, p, g_mode, rows_idx, centre=c)
    fn = np.linalg.norm(f_ref, axis=1)
    live = fn > 0
    err = np.linalg.norm(got4[:, :3] - f_ref, axis=1)
    rel = err[live] / fn[live]
    kappa = A[live] / fn[live]
    bound = (B[live] + np.linalg.norm(Y[rows_idx][live] - c, axis=1) * Wm[live]) / fn[live]
    ratio = rel / (EPS32 * bound)
    i_worst = int(np.argmax(ratio)) if ratio.size else 0
    check(f"{what}: per-row f error / (2^-24 kappa'_i), worst row", float(ratio.max()) if ratio.size else 0.0, C_ROW)
    check(f"{what}: per-row relative error of f_i, worst row", float(rel.max()) if rel.size else 0.0, float("inf"))
    check(f"{what}: row condition kappa_i of the row nearest its bound",
          float(kappa[i_worst]) if kappa.size else 0.0, float("inf"))
    check(f"{what}: row condition kappa_i, largest", float(kappa.max()) if kappa.size else 0.0, float("inf"))
    check(f"{what}: row condition kappa_i, median", float(np.median(kappa)) if kappa.size else 0.0, float("inf"))
    wpos = W_ref > 0
    relW = np.abs(got4[:, 3][wpos] - W_ref[wpos]) / W_ref[wpos]
    check(f"{what}: per-row relative error of W_i / 2^-24, worst row", float(relW.max() / EPS32) if relW.size else 0.0,
          C_ROW)
    return (float(rel.max()) if rel.size else 0.0), (float(kappa.max()) if kappa.size else 0.0)


def check(quantity, value, tol):
    """assert value <= tol, recording the measurement in SCGR_PARITY_LOG"""
    value = float(value)
    path = os.environ.get("SCGR_PARITY_LOG")
    if path:
        test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
        with open(path, "a") as fh:
            fh.write(json.dumps({"test": test, "quantity": quantity, "value": value, "tol": float(tol)}) + "\n")
    assert value <= tol, (quantity, value, tol)


def pose_errors(R, t, s, Ro, to, so, diag):
    """(rotation error in degrees, translation error / bbox diagonal, relative scale error)"""
    return (rot_err_deg(R, Ro), float(np.linalg.norm(np.asarray(t) - np.asarray(to))) / diag,
            abs(s - so) / abs(so))


def check_pose(what, R, t, s, Ro, to, so, diag, rot_tol=0.5, t_tol=1e-3, s_tol=1e-5):
    """the pose tolerances: 0.5 degrees, 1e-3 of the diagonal, 1e-5 relative scale"""
    er, et, es = pose_errors(R, t, s, Ro, to, so, diag)
    check(f"{what}: rotation (deg)", er, rot_tol)
    check(f"{what}: translation / bbox diagonal", et, t_tol)
    check(f"{what}: scale (relative)", es, s_tol)


def max_rel(got, ref, floor=1e-12):
    """largest |got - ref| / max(|ref|, floor)"""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor))) if ref.size else 0.0


class Gpu:
    """One context over device copies of X and Y0."""

    def __init__(self, X, Y0, tune=None, **prm):
        self.params = scgr.scgr_default_params(**prm)
        self.ctx = scgr.scgr_create(self.params)
        for key, value in (tune or {}).items():
            scgr.scgr_set_tuning(self.ctx, key, value)
        self.X = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
        self.Y0 = torch.from_numpy(np.ascontiguousarray(Y0, np.float32)).cuda()
        self.n, self.m = len(X), len(Y0)
        scgr.scgr_set_reference(self.ctx, self.X)
        scgr.scgr_set_template(self.ctx, self.Y0)
        scgr.scgr_compute_descriptors(self.ctx)

    def close(self):
        if self.ctx is not None:
            scgr.scgr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def knn(self, which):
        n = self.n if which == 0 else self.m
        out = torch.empty((n, self.params.k), dtype=torch.int32, device="cuda")
        scgr.scgr_get_descriptors(self.ctx, which, out, None)
        return out.cpu().numpy()

    def curv64(self, which):
        n = self.n if which == 0 else self.m
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        scgr.scgr_get_curvature64(self.ctx, which, out)
        return out.cpu().numpy()

    def set_curvature(self, which, a):
        scgr.scgr_set_curvature(self.ctx, which, torch.from_numpy(np.asarray(a, np.float64)).cuda())

    def forces(self):
        f4 = torch.empty((self.m, 4), dtype=torch.float32, device="cuda")
        scgr.scgr_forces(self.ctx, f4)
        return f4.cpu().numpy()

    def run(self, iters):
        scgr.scgr_run(self.ctx, iters)
        return scgr.scgr_get_result(self.ctx)

    def moved(self):
        out = torch.empty((self.m, 3), dtype=torch.float32, device="cuda")
        scgr.scgr_get_moved(self.ctx, out)
        return out.cpu().numpy()

    def sigma(self):
        return scgr.scgr_get_sigma(self.ctx)
