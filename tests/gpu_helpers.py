"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI.

check() asserts a measured error against its tolerance and, when the
environment variable SCGR_PARITY_LOG names a file, appends the measurement
to it (one JSON object per line: test id, quantity, value, tolerance), so
that a GPU run states the error of every result against the FP64 oracle
(tests/parity_report.py tabulates the log).

check_rows() adds the per-row view of a force check: a relative L2 over many
rows can hide a single row whose sum cancels, so every checked row i must meet

    |f_got,i - f_i| <= C_ROW * 2^-24 * (B_i + |Y_i - c| W_i + Ae_i) + U_i,

with the oracle's term-magnitude sums (oracle.force_row_magnitudes) in the
frame centred on the reference mean c, where the kernel accumulates
sum_j w_ij X_j and sum_j w_ij and forms f_i as their difference:
B_i + |Y_i - c| W_i bounds both sums, and Ae_i = sum_j |w_ij r_ij| e_ij carries
the rounding of each pair's float32 exponent (absolute error ~ 2^-24 e_ij,
e_ij the exponent's size).  The logged ratio is therefore an effective
condition number kappa'_i = (B_i + |Y_i - c| W_i + Ae_i) / |f_i| times
2^-24 times the stated C_ROW, and kappa'_i is at least the condition number
kappa_i = sum_j |w_ij r_ij| / |f_i| of the Eq. 5 sum (triangle inequality),
which is logged beside it.  C_ROW = 64 covers the pair-weight rounding (ex2,
sqrt, a few products: < 8 ulp), the float32 tile sums under Kahan
compensation across tiles, and the squared distance evaluated as
|X'|^2 + |Y'|^2 - 2 X'.Y' (absolute error ~ 2^-24 (|X'|^2 + |Y'|^2), which
enters f_i only through w_ij r_ij).  U_i is the float32 underflow allowance:
the factor 2^(log2 aX - (a_hat_X - a_hat_Y)^2) of each pair is flushed to 0
below 2^-126, an absolute error of at most aY_i 2^-126 d_ij^(p-1) per pair
weight, so U_i = aY_i 2^-126 N dmax_i^p (aY_i read as 1 for g = s) with
dmax_i = |Y_i - c| + max_j |X_j - c|.  Rows whose oracle force is below
2^24 U_i lie outside float32's range and are counted, not compared by their
relative error.  W_i is checked the same way with its own sums
(W_i + We_i, allowance N aY_i 2^-126 dmax_i^(p-1))."""
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
    Returns (worst per-row relative error of f over the rows inside float32's
    range, worst kappa_i over those rows)."""
    import oracle as O
    got4 = np.asarray(got4, np.float64)
    f_ref = np.asarray(f_ref, np.float64)
    W_ref = np.asarray(W_ref, np.float64)
    Y = np.asarray(Y, np.float64)
    X = np.asarray(X, np.float64)
    c = X.mean(axis=0)
    rows_idx = np.arange(len(Y)) if rows is None else np.asarray(rows)
    mg = O.force_row_magnitudes(Y, X, aY, aX, sigma, p, g_mode, rows_idx, centre=c)
    ydist = np.linalg.norm(Y[rows_idx] - c, axis=1)
    dmax = ydist + float(np.max(np.linalg.norm(X - c, axis=1)))
    afac = np.asarray(aY, np.float64)[rows_idx] if g_mode == 1 else np.ones(len(rows_idx))
    U_f = afac * 2.0 ** -126 * len(X) * dmax ** p
    U_W = afac * 2.0 ** -126 * len(X) * dmax ** (p - 1.0)
    scale_f = mg["B"] + ydist * mg["W"] + mg["Ae"]
    fn = np.linalg.norm(f_ref, axis=1)
    err = np.linalg.norm(got4[:, :3] - f_ref, axis=1)
    live = scale_f > 0
    c_f = np.maximum(err[live] - U_f[live], 0.0) / (EPS32 * scale_f[live])
    check(f"{what}: per-row f error / (2^-24 kappa'_i |f_i|), worst row", float(c_f.max()) if c_f.size else 0.0, C_ROW)
    inside = fn >= 2.0 ** 24 * U_f
    check(f"{what}: rows below float32 range (not compared relatively)", int(np.count_nonzero(~inside & (fn > 0))),
          float("inf"))
    rel = err[inside] / fn[inside]
    kappa = mg["A"][inside] / fn[inside]
    check(f"{what}: per-row relative error of f_i, worst row", float(rel.max()) if rel.size else 0.0, float("inf"))
    if rel.size:
        check(f"{what}: row condition kappa_i of the worst row", float(kappa[int(np.argmax(rel))]), float("inf"))
    check(f"{what}: row condition kappa_i, largest", float(kappa.max()) if kappa.size else 0.0, float("inf"))
    check(f"{what}: row condition kappa_i, median", float(np.median(kappa)) if kappa.size else 0.0, float("inf"))
    scale_W = mg["W"] + mg["We"]
    wl = scale_W > 0
    errW = np.abs(got4[:, 3] - W_ref)
    c_W = np.maximum(errW[wl] - U_W[wl], 0.0) / (EPS32 * scale_W[wl])
    check(f"{what}: per-row W error / (2^-24 (W_i + We_i)), worst row", float(c_W.max()) if c_W.size else 0.0, C_ROW)
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
