"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI.

check() asserts a measured error against its tolerance and, when the
environment variable SCGR_PARITY_LOG names a file, appends the measurement
to it (one JSON object per line: test id, quantity, value, tolerance), so
that a GPU run states the error of every result against the FP64 oracle
(tests/parity_report.py tabulates the log)."""
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
