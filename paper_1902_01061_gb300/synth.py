"""Seeded synthetic point clouds shaped like the paper's registration workloads.

The paper evaluates on scanned models (Stanford bunny, Armadillo, a human scan)
and Kinect captures (Sec. V), none of which are available here.  This module
builds stand-ins: points sampled uniformly by area on the outer surface of a
union of overlapping ellipsoids, a template that is a similarity transform of
the reference (row-vector convention, Y = s * X @ R + t, as in Eq. 9), plus
the paper's perturbations: Gaussian noise, uniform outliers, a removed part
(Sec. V "18% consecutive points deleted") and a dense structured outlier
cluster (Sec. V, Fig. 4).

This module holds none of the registration method's arithmetic.  It feeds both
the CPU oracle and the CUDA path, and nothing else is shared between them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1902010610


def rotation_matrix(axis, angle_deg: float) -> np.ndarray:
    """Right-multiplied rotation (row vectors: y = x @ R) about `axis`."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    th = math.radians(angle_deg)
    kx, ky, kz = axis
    K = np.array([[0.0, -kz, ky], [kz, 0.0, -kx], [-ky, kx, 0.0]])
    Rcol = np.eye(3) + math.sin(th) * K + (1.0 - math.cos(th)) * (K @ K)
    return Rcol.T  # x @ Rcol.T == (Rcol @ x^T)^T


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


@dataclass
class EllipsoidUnion:
    centres: np.ndarray   # K x 3
    axes: np.ndarray      # K x 3 semi-axes
    rots: np.ndarray      # K x 3 x 3, local -> world (row vectors: w = l @ rot + c)

    @staticmethod
    def random(rng: np.random.Generator, k: int) -> "EllipsoidUnion":
        centres = rng.uniform(-0.5, 0.5, size=(k, 3))
        axes = rng.uniform(0.3, 1.0, size=(k, 3))
        rots = np.stack([random_rotation(rng) for _ in range(k)])
        return EllipsoidUnion(centres, axes, rots)

    def _inside(self, p: np.ndarray, e: int) -> np.ndarray:
        loc = (p - self.centres[e]) @ self.rots[e].T
        return np.sum((loc / self.axes[e]) ** 2, axis=1) < 1.0 - 1e-9

    def sample_surface(self, rng: np.random.Generator, n: int) -> np.ndarray:
        """n points uniform by area on the union's outer surface."""
        K = len(self.axes)
        areas = np.array([_ellipsoid_area(a) for a in self.axes])
        out = []
        have = 0
        while have < n:
            batch = max(4 * (n - have), 4096)
            comp = rng.choice(K, size=batch, p=areas / areas.sum())
            pts = np.empty((batch, 3))
            keep = np.zeros(batch, dtype=bool)
            for e in range(K):
                sel = np.nonzero(comp == e)[0]
                if sel.size == 0:
                    continue
                a, b, c = self.axes[e]
                u = rng.standard_normal((sel.size, 3))
                u /= np.linalg.norm(u, axis=1, keepdims=True)
                # area element of the sphere->ellipsoid map, relative to its max
                gelem = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
                acc = rng.uniform(size=sel.size) * max(a * b, a * c, b * c) < gelem
                loc = u * self.axes[e]
                pts[sel] = loc @ self.rots[e] + self.centres[e]
                keep[sel] = acc
                for o in range(K):
                    if o != e:
                        keep[sel] &= ~self._inside(pts[sel], o)
            good = pts[keep]
            out.append(good)
            have += len(good)
        allp = np.concatenate(out)
        pick = rng.permutation(len(allp))[:n]
        return allp[np.sort(pick)]


def _ellipsoid_area(ax) -> float:
    # Knud Thomsen's approximation; only used to split samples between ellipsoids
    a, b, c = ax
    q = 1.6075
    return 4.0 * math.pi * (((a * b) ** q + (a * c) ** q + (b * c) ** q) / 3.0) ** (1.0 / q)


def bbox_diag(P: np.ndarray) -> float:
    return float(np.linalg.norm(P.max(axis=0) - P.min(axis=0)))


@dataclass
class Pair:
    """One registration problem.  X: reference (N x 3), Y0: template (M x 3),
    both float32.  The inlier part of the template satisfies
    Y0 ~= s_gt * X[corr] @ R_gt + t_gt, so the registration that maps Y0 back
    onto X is s = 1/s_gt, R = R_gt^T, t = -t_gt @ R_gt^T / s_gt."""
    name: str
    X: np.ndarray
    Y0: np.ndarray
    R_gt: np.ndarray
    t_gt: np.ndarray
    s_gt: float
    corr: np.ndarray | None = None   # template row -> reference row (inliers), -1 for outliers
    iterations: int = 100
    meta: dict = field(default_factory=dict)

    def inverse_pose(self):
        R = self.R_gt.T
        s = 1.0 / self.s_gt
        t = -(self.t_gt @ R) * s
        return R, t, s


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def tiny(seed: int | None = None, n: int = 1000) -> Pair:
    """1,000-point reference on a 3-ellipsoid union; template rotated 50 deg
    about x, translated (0.2,-0.1,0.3), scaled 1.2, N(0,0.005) noise."""
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    surf = EllipsoidUnion.random(rng, 3)
    X = surf.sample_surface(rng, n)
    R = rotation_matrix([1, 0, 0], 50.0)
    t = np.array([0.2, -0.1, 0.3])
    s = 1.2
    Y0 = s * X @ R + t + rng.normal(0.0, 0.005, size=X.shape)
    return Pair("tiny-1k", _f32(X), _f32(Y0), R, t, s, np.arange(n), 100)


def mild(seed: int | None = None, n: int = 1000, angle: float = 15.0) -> Pair:
    """Like `tiny` with a gentler transform (15 deg about a fixed axis,
    translation (0.1,0,0), scale 1.1): the must-converge recovery case."""
    rng = np.random.default_rng(SEED_BASE + 11 if seed is None else seed)
    surf = EllipsoidUnion.random(rng, 3)
    X = surf.sample_surface(rng, n)
    R = rotation_matrix([0.3, 0.9, 0.2], angle)
    t = np.array([0.1, 0.0, 0.0])
    s = 1.1
    Y0 = s * X @ R + t + rng.normal(0.0, 0.002, size=X.shape)
    return Pair(f"mild-{n}", _f32(X), _f32(Y0), R, t, s, np.arange(n), 100)


def scale_case(seed: int | None = None, n: int = 35000) -> Pair:
    """35,000-point 5-ellipsoid reference; template rotated 90 deg about a
    random axis, scaled 0.8, 20% removed by a half-space slab, then 10% uniform
    outliers in the template's bounding box (M = 0.8 n + 0.08 n)."""
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    surf = EllipsoidUnion.random(rng, 5)
    X = surf.sample_surface(rng, n)
    R = rotation_matrix(random_unit(rng), 90.0)
    s = 0.8
    t = rng.uniform(-0.2, 0.2, size=3)
    Y = s * X @ R + t
    u = random_unit(rng)
    proj = Y @ u
    nkeep = n - int(round(0.2 * n))
    keep = np.sort(np.argsort(proj, kind="stable")[:nkeep])
    Y = Y[keep]
    lo, hi = Y.min(axis=0), Y.max(axis=0)
    nout = int(round(0.1 * nkeep))
    out = rng.uniform(lo, hi, size=(nout, 3))
    Y0 = np.concatenate([Y, out])
    corr = np.concatenate([keep, -np.ones(nout, dtype=np.int64)])
    return Pair(f"scale-{n}", _f32(X), _f32(Y0), R, t, s, corr, 200)


def diff_case(seed: int | None = None, n: int = 50000) -> Pair:
    """n x n points, 5-ellipsoid surface, template rotated 30 deg, noise with
    standard deviation 0.01 of the bounding-box diagonal."""
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    surf = EllipsoidUnion.random(rng, 5)
    X = surf.sample_surface(rng, n)
    R = rotation_matrix(random_unit(rng), 30.0)
    s = 1.0
    t = rng.uniform(-0.1, 0.1, size=3)
    Y0 = s * X @ R + t + rng.normal(0.0, 0.01 * bbox_diag(X), size=X.shape)
    return Pair(f"diff-{n}", _f32(X), _f32(Y0), R, t, s, np.arange(n), 1)


def large_case(seed: int | None = None, n: int = 1_000_000, n_out_frac: float = 0.15) -> Pair:
    """1M-point 8-ellipsoid reference; template = an independent surface
    sample of 0.85 n points, rotated 60 deg, scaled 1.1, plus 0.15 n points
    uniform in an axis-aligned box of side 0.15 x bbox diagonal placed
    against one face of the bounding box (a dense structured outlier)."""
    rng = np.random.default_rng(SEED_BASE + 5 if seed is None else seed)
    surf = EllipsoidUnion.random(rng, 8)
    X = surf.sample_surface(rng, n)
    n_out = int(round(n_out_frac * n))
    Ys = surf.sample_surface(rng, n - n_out)
    R = rotation_matrix(random_unit(rng), 60.0)
    s = 1.1
    t = rng.uniform(-0.2, 0.2, size=3)
    Y = s * Ys @ R + t
    lo, hi = Y.min(axis=0), Y.max(axis=0)
    side = 0.15 * bbox_diag(Y)
    face_axis = int(rng.integers(3))
    corner = lo + rng.uniform(0, 1, size=3) * (hi - lo - side)
    corner[face_axis] = hi[face_axis]          # against the +face, outside it
    box = corner + rng.uniform(0, side, size=(n_out, 3))
    Y0 = np.concatenate([Y, box])
    corr = -np.ones(n, dtype=np.int64)
    return Pair(f"large-{n}", _f32(X), _f32(Y0), R, t, s, corr, 50,
                meta={"n_outliers": n_out})


def batch_case(seed: int | None = None, npairs: int = 512, lo: int = 500, hi: int = 20000):
    """npairs independent problems, reference sizes log-uniform in [lo, hi],
    each template a transformed copy (random rotation up to 90 deg, scale in
    [0.7, 1.4]) with 0-15% uniform outliers in its bounding box."""
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    pairs = []
    for b in range(npairs):
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        surf = EllipsoidUnion.random(rng, int(rng.integers(3, 6)))
        X = surf.sample_surface(rng, n)
        R = rotation_matrix(random_unit(rng), float(rng.uniform(0.0, 90.0)))
        s = float(rng.uniform(0.7, 1.4))
        t = rng.uniform(-0.2, 0.2, size=3)
        Y = s * X @ R + t
        nout = int(round(rng.uniform(0.0, 0.15) * n))
        lo3, hi3 = Y.min(axis=0), Y.max(axis=0)
        Y0 = np.concatenate([Y, rng.uniform(lo3, hi3, size=(nout, 3))])
        corr = np.concatenate([np.arange(n), -np.ones(nout, dtype=np.int64)])
        pairs.append(Pair(f"batch{b}-{n}", _f32(X), _f32(Y0), R, t, s, corr, 100))
    return pairs


def subsample(P: np.ndarray, m: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(P), size=m, replace=False))
    return idx
