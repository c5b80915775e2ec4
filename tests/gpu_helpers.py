"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI."""
import math

import numpy as np
import torch

from paper_1902_01061_gb300 import scgr


def rot_err_deg(Ra, Rb):
    c = (np.trace(np.asarray(Ra).T @ np.asarray(Rb)) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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
