"""FP64 CPU oracle: shape-constrained gravitational registration, step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the product
path may import this module.

Notation follows the paper (arXiv 1902.01061):
  X  : reference cloud, N x 3 (row vectors), points X_j
  Y  : template cloud at iteration t, M x 3, points Y_i;  Y0 = Y(0)
  a  : per-point curvature descriptor (Sec. III-A, Sec. IV)
  s  : shape similarity, Eq. 3;  g(s): Eq. 10 or g = s (Sec. IV)
  h  : distance law, Eq. 4 / Eq. 11, h(d) = d^p
  f  : force on a template point, Eq. 5
  d  : template displacement, Eq. 5.5
  R  : Kabsch rotation, Eq. 6;  c: scale, Sec. III-B / Eq. 8
  G  : gravitational constant schedule, Eq. 12

Readings where the paper is silent, ambiguous or garbled:
  R1  kNN key: float32 (dx*dx + dy*dy) + dz*dz, every operation rounded
      separately (no fused multiply-add), self included, ties to lower index.
  R2  "curvature" (the cited definition is missing): surface variation
      lambda_min / (lambda_1 + lambda_2 + lambda_3) of the covariance of the
      k nearest neighbours (k = 16), in [0, 1/3]; a negative rounding residue
      of lambda_min is clamped to 0, and a zero trace gives 0.
  R3  sigma of Eq. 3 (unspecified): population standard deviation of the
      reference curvatures; 1 if that is below 1e-12.  User-overridable.
  R4  n_ij = (Y_i - X_j) / ||Y_i - X_j||; with the minus sign of Eq. 5 the
      force pulls Y_i toward X_j.
  R5  Eq. 11 is circular as printed; h(d) = d^p with p >= 1.  Default p = 1:
      under these readings larger p drifts away from alignment (for p > 1 the
      geometric term alone prefers crossed principal axes), matching the
      paper's remark that lower p registers better.
  R6  step size (Eq. 5.5 with unit masses, v = 0): each template point is
      displaced by delta_i = kappa * f_i and the template translation is
      d = mean(delta_i) = kappa * F / M.  Normalized mode (default):
      kappa = eta0 * (G/G1) * M / W with W = sum_i W_i, W_i = sum_j g h / d,
      which makes d = eta0 (G/G1) F / W scale-free.  Literal mode:
      kappa = G * time^2.
  R7  Eq. 12 with 0-based iteration t: G(t) = 0.1 G1 + 0.9 G1 / (1 + e^-(t - E/2));
      E = number of iterations of the run unless given.
  R8  scale c = sqrt(eX / eY) (std-dev ratio; a ratio of variances is a
      squared length ratio).  eX, eY: largest eigenvalues of the 1/n
      covariances of the reference and of the current template.
  R9  Eq. 8 with a scalar c is Y' = c (Y(t) - mu); Eq. 9 then adds mu and d.
  R10 the "after" cloud of Eq. 6 is the per-point displaced template
      Y + delta, mean-subtracted (a pure translation would give R = I).
  R11 if the second singular value of C^ is below 1e-12 of the first, the
      rotation increment is the identity (flagged as degenerate).
  R12 a coincident pair (d = 0) contributes nothing to f (limit for p >= 1).
  R14 template descriptors are computed once on Y0 (the descriptor is
      invariant under similarity transforms).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


@dataclass
class Params:
    k: int = 16             # neighbours per descriptor (R2)
    p: float = 1.0          # distance exponent, Eq. 11 (R5)
    sigma: float = 0.0      # RBF spread of Eq. 3; <= 0 selects R3
    g_mode: int = 1         # 0: g = s (equal weight, Sec. IV); 1: g = aX aY s (Eq. 10)
    G1: float = 1.0e4       # Eq. 12 (Sec. IV value)
    E: int = 0              # Eq. 12 horizon; <= 0: the run's iteration count (R7)
    step_mode: int = 0      # 0: normalized step (R6); 1: literal Eq. 5.5
    eta0: float = 0.5       # normalized step fraction (R6)
    time: float = 1.0       # literal-mode time step of Eq. 5.5
    scale_mode: int = 0     # 0: c = sqrt(eX/eY) (R8); 1: c = eX/eY as printed; 2: c = 1
    neigh_mode: int = 0     # 0: k nearest neighbours (R2); 1: radius radius_scale*sqrt(e) (Sec. IV)
    radius_scale: float = 1.0


# ----------------------------------------------------------------- descriptors

def knn(P, k: int) -> np.ndarray:
    """k nearest neighbours of every point of P among P (self included).

    Reading R1: the key is the float32 value (dx*dx + dy*dy) + dz*dz with
    every operation rounded on its own; the neighbours are the first k points
    of the order (key, index).  numpy float32 ufuncs round each operation
    separately and never fuse, so the keys below are exactly that value.
    Returns int32 [n, k], each row sorted by (key, index).
    """
    P = np.ascontiguousarray(P, dtype=np.float32)
    n = len(P)
    if k > n:
        raise ValueError("k > n")
    out = np.empty((n, k), dtype=np.int32)
    px, py, pz = P[:, 0], P[:, 1], P[:, 2]
    chunk = max(1, (1 << 22) // max(n, 1))
    for q0 in range(0, n, chunk):
        q1 = min(n, q0 + chunk)
        dx = P[q0:q1, 0:1] - px[None, :]
        dy = P[q0:q1, 1:2] - py[None, :]
        dz = P[q0:q1, 2:3] - pz[None, :]
        key = (dx * dx + dy * dy) + dz * dz
        # value of the k-th smallest key; every point with a key <= it is a
        # candidate, and the (key, index) order picks k of them
        kth = np.partition(key, k - 1, axis=1)[:, k - 1]
        for r in range(q1 - q0):
            cand = np.nonzero(key[r] <= kth[r])[0]           # ascending index
            order = np.argsort(key[r, cand], kind="stable")  # ties keep index order
            out[q0 + r] = cand[order[:k]]
    return out


def curvature(P, nbr: np.ndarray) -> np.ndarray:
    """Per-point curvature a (Sec. III-A, Sec. IV; reading R2).

    For point p with neighbour set Q (its k nearest, p included):
    mu = mean(Q), C = (1/k) sum (q - mu)(q - mu)^T in float64, and
    a = lambda_min(C) / (lambda_1 + lambda_2 + lambda_3).
    """
    Q = np.asarray(P, dtype=np.float64)[nbr]            # n, k, 3
    k = Q.shape[1]
    mu = Q.mean(axis=1)
    D = Q - mu[:, None, :]
    C = np.einsum("nki,nkj->nij", D, D) / k
    lam = np.linalg.eigvalsh(C)                          # ascending
    tr = np.trace(C, axis1=1, axis2=2)                   # = lambda_1 + lambda_2 + lambda_3
    lmin = np.maximum(lam[:, 0], 0.0)
    a = np.zeros(len(Q))
    pos = tr > 0
    a[pos] = lmin[pos] / tr[pos]
    return a


def curvature_radius(P, radius_scale: float = 1.0) -> np.ndarray:
    """Curvature over the radius neighbourhood of Sec. IV: every point whose
    distance from p is at most radius_scale * sqrt(e), e the largest
    eigenvalue of the cloud's 1/n covariance.  Membership is decided on the
    float32 key of R1 against float32(radius_scale^2 e) (same precision as the
    GPU); the covariance of the members (1/|N|) is float64."""
    P32 = np.ascontiguousarray(P, dtype=np.float32)
    P64 = P32.astype(np.float64)
    _, _, e = cloud_stats(P64)
    r2 = np.float32(radius_scale * radius_scale * e)
    a = np.zeros(len(P32))
    for i in range(len(P32)):
        dx = P32[i, 0] - P32[:, 0]
        dy = P32[i, 1] - P32[:, 1]
        dz = P32[i, 2] - P32[:, 2]
        key = (dx * dx + dy * dy) + dz * dz
        Q = P64[key <= r2]
        D = Q - Q.mean(axis=0)
        C = D.T @ D / len(Q)
        tr = np.trace(C)
        a[i] = max(np.linalg.eigvalsh(C)[0], 0.0) / tr if tr > 0 else 0.0
    return a


def sigma_auto(aX) -> float:
    """Reading R3: population std of the reference curvatures (1 if ~0)."""
    sd = float(np.std(np.asarray(aX, dtype=np.float64)))
    return sd if sd >= 1e-12 else 1.0


def cloud_stats(P):
    """Mean, 1/n covariance and its largest eigenvalue (Sec. III-B)."""
    P = np.asarray(P, dtype=np.float64)
    mu = P.mean(axis=0)
    D = P - mu
    C = D.T @ D / len(P)
    return mu, C, float(np.linalg.eigvalsh(C)[-1])


def descriptors(X, Y0, prm: Params, sigma_scale: float = 1.0):
    """The one-time descriptor pass: neighbourhoods (k nearest, or the radius
    of Sec. IV), curvature of both clouds, sigma (times sigma_scale)."""
    if prm.neigh_mode == 1:
        nX = nY = None
        aX = curvature_radius(X, prm.radius_scale)
        aY = curvature_radius(Y0, prm.radius_scale)
    else:
        nX = knn(X, prm.k)
        nY = knn(Y0, prm.k)
        aX = curvature(X, nX)
        aY = curvature(Y0, nY)
    sigma = (prm.sigma if prm.sigma > 0 else sigma_auto(aX)) * sigma_scale
    return dict(knnX=nX, knnY=nY, aX=aX, aY=aY, sigma=sigma)


# ----------------------------------------------------------------- forces

def _pair_terms(Yi, X, aYi, aX, sigma, p, g_mode):
    """For a block of template rows: r_ij, d_ij and g_ij (Eq. 3, Eq. 10)."""
    r = Yi[:, None, :] - X[None, :, :]                   # r^{Yi} - r^{Xj}
    d = np.sqrt(np.sum(r * r, axis=2))
    s = np.exp(-((aX[None, :] - aYi[:, None]) ** 2) / sigma ** 2)   # Eq. 3
    if g_mode == 1:
        g = aX[None, :] * aYi[:, None] * s               # Eq. 10
    else:
        g = s                                            # g = s (Sec. IV)
    return r, d, g


def forces_rows(Y, X, aY, aX, sigma, p, g_mode, rows=None):
    """Eq. 5 without the factor G, for template rows `rows` (all if None):

        f_i = - sum_j g(s_ij) h(||Y_i - X_j||) n_ij,  h(d) = d^p,
        n_ij = (Y_i - X_j) / ||Y_i - X_j||  (R4, R5; R12 at d = 0),

    and the per-row weight W_i = sum_j g(s_ij) d_ij^(p-1) used by the
    normalized step (R6).  Sums run over j in order, in float64.
    """
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    aY = np.asarray(aY, dtype=np.float64)
    aX = np.asarray(aX, dtype=np.float64)
    rows = np.arange(len(Y)) if rows is None else np.asarray(rows)
    f = np.zeros((len(rows), 3))
    W = np.zeros(len(rows))
    chunk = max(1, (1 << 21) // max(len(X), 1))
    for c0 in range(0, len(rows), chunk):
        rr = rows[c0:c0 + chunk]
        r, d, g = _pair_terms(Y[rr], X, aY[rr], aX, sigma, p, g_mode)
        h = d ** p                                       # Eq. 11 (R5)
        with np.errstate(invalid="ignore", divide="ignore"):
            n = np.where(d[..., None] > 0, r / d[..., None], 0.0)   # R4, R12
            hd = np.where(d > 0, d ** (p - 1.0), 1.0 if p == 1.0 else 0.0)
        f[c0:c0 + len(rr)] = -np.sum((g * h)[..., None] * n, axis=1)
        W[c0:c0 + len(rr)] = np.sum(g * hd, axis=1)
    return f, W


def forces(Y, X, aY, aX, sigma, p, g_mode):
    return forces_rows(Y, X, aY, aX, sigma, p, g_mode, None)


def force_row_magnitudes(Y, X, aY, aX, sigma, p, g_mode, rows=None, centre=None):
    """Magnitudes of the terms of the Eq. 5 sum, for judging how well each
    row's force is conditioned.  For template row i with pair weight
    w_ij = g(s_ij) d_ij^(p-1) and r_ij = Y_i - X_j (the same terms as
    `forces_rows`), returns a dict of per-row sums over j, in float64:

      A  = sum_j |w_ij r_ij|            (Euclidean norm of each term)
      B  = sum_j w_ij |X_j - centre|    (centre: 3-vector, default the origin)
      W  = sum_j w_ij
      Ae = sum_j |w_ij r_ij| e_ij,  We = sum_j w_ij e_ij,

    with e_ij = -ln(g_ij / aY_i) = (aX_j - aY_i)^2 / sigma^2 - ln aX_j for
    g = aX aY s (Eq. 10), and e_ij = -ln s_ij = (aX_j - aY_i)^2 / sigma^2 for
    g = s: the size of the exponent of the pair's pose-independent factor.

    kappa_i = A_i / |f_i| is the condition number of the sum that gives f_i.
    B_i + |Y_i - centre| W_i bounds the size of the two sums sum_j w_ij X_j
    and Y_i sum_j w_ij when f_i is formed as their difference in a frame
    with that centre, and Ae_i, We_i measure how an absolute error in each
    pair's exponent (relative error e_ij times that of the exponent) reaches
    f_i and W_i."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    aY = np.asarray(aY, dtype=np.float64)
    aX = np.asarray(aX, dtype=np.float64)
    c = np.zeros(3) if centre is None else np.asarray(centre, dtype=np.float64)
    rows = np.arange(len(Y)) if rows is None else np.asarray(rows)
    out = {key: np.zeros(len(rows)) for key in ("A", "B", "W", "Ae", "We")}
    xdist = np.sqrt(np.sum((X - c) ** 2, axis=1))
    with np.errstate(divide="ignore"):
        lnaX = np.where(aX > 0, np.log(np.where(aX > 0, aX, 1.0)), -np.inf)
    chunk = max(1, (1 << 21) // max(len(X), 1))
    for c0 in range(0, len(rows), chunk):
        rr = rows[c0:c0 + chunk]
        r, d, g = _pair_terms(Y[rr], X, aY[rr], aX, sigma, p, g_mode)
        with np.errstate(invalid="ignore", divide="ignore"):
            w = np.where(d > 0, g * d ** (p - 1.0), g if p == 1.0 else 0.0)   # R12
        e = (aX[None, :] - aY[rr][:, None]) ** 2 / sigma ** 2                  # Eq. 3
        if g_mode == 1:
            e = e - lnaX[None, :]                                             # Eq. 10: the aX factor
        e = np.where(w > 0, e, 0.0)                                           # zero terms carry no error
        wd = w * d                                                            # |w r| = w d
        sl = slice(c0, c0 + len(rr))
        out["A"][sl] = np.sum(wd, axis=1)
        out["B"][sl] = w @ xdist
        out["W"][sl] = np.sum(w, axis=1)
        out["Ae"][sl] = np.sum(wd * e, axis=1)
        out["We"][sl] = np.sum(w * e, axis=1)
    return out


def potential(Y, X, aY, aX, sigma, p, g_mode) -> float:
    """U = sum_i sum_j g(s_ij) d_ij^(p+1) / (p+1); its gradient with respect to
    Y_i is -f_i of Eq. 5 (descriptors held fixed)."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    aY = np.asarray(aY, dtype=np.float64)
    aX = np.asarray(aX, dtype=np.float64)
    U = 0.0
    chunk = max(1, (1 << 21) // max(len(X), 1))
    for c0 in range(0, len(Y), chunk):
        _, d, g = _pair_terms(Y[c0:c0 + chunk], X, aY[c0:c0 + chunk], aX, sigma, p, g_mode)
        U += float(np.sum(g * d ** (p + 1.0)) / (p + 1.0))
    return U


def potential_grad(Y, X, aY, aX, sigma, p, g_mode):
    """dU/dY (M x 3) = -f (Eq. 5)."""
    f, _ = forces(Y, X, aY, aX, sigma, p, g_mode)
    return -f


def force_vjp(Y, X, aY, aX, sigma, p, g_mode, v):
    """(d f_i / d Y_i)^T v_i for the force of Eq. 5 (descriptors fixed): with
    r = Y_i - X_j, d = |r| and w = g d^(p-1), f_i = -sum_j w r gives
    d f_i / d Y_i = -sum_j [w I + r (dw/dY_i)^T], dw/dY_i = g (p-1) d^(p-3) r."""
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    out = np.zeros((len(Y), 3))
    for i in range(len(Y)):
        r, d, g = _pair_terms(Y[i:i + 1], X, np.asarray(aY, dtype=np.float64)[i:i + 1],
                              np.asarray(aX, dtype=np.float64), sigma, p, g_mode)
        r, d, g = r[0], d[0], g[0]
        live = d > 0
        w = np.where(live, g * np.where(live, d, 1.0) ** (p - 1.0), g if p == 1.0 else 0.0)
        dw = np.where(live, g * (p - 1.0) * np.where(live, d, 1.0) ** (p - 3.0), 0.0)
        J = -(w.sum() * np.eye(3) + (r * dw[:, None]).T @ r)
        out[i] = J.T @ np.asarray(v, dtype=np.float64)[i]
    return out


def rodrigues(omega):
    """Row-vector rotation for axis-angle omega: y = x @ R, with
    R = exp([omega]_x)^T."""
    w = np.asarray(omega, dtype=np.float64)
    th = float(np.linalg.norm(w))
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-12:
        Rc = np.eye(3) + K + 0.5 * K @ K
    else:
        Rc = np.eye(3) + math.sin(th) / th * K + (1.0 - math.cos(th)) / th ** 2 * (K @ K)
    return Rc.T


def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def _drodrigues(omega):
    """d exp([omega]_x) / d omega_k for k = 0..2 (column-vector form), by the
    closed form of Gallego & Yezzi (2015):
    dR/dw_k = (w_k [w]_x + [w x ((I - R) e_k)]_x) R / |w|^2, and [e_k]_x at 0."""
    w = np.asarray(omega, dtype=np.float64)
    th2 = float(w @ w)
    E = np.eye(3)
    if th2 < 1e-24:
        return [_skew(E[k]) for k in range(3)]
    Rc = rodrigues(w).T
    out = []
    for k in range(3):
        v = np.cross(w, (np.eye(3) - Rc) @ E[k])
        out.append((w[k] * _skew(w) + _skew(v)) @ Rc / th2)
    return out


def pose_potential_and_grad(pose7, Y0, X, aY, aX, sigma, p, g_mode):
    """U(pose) for Y = s * Y0 @ R(omega) + t, pose7 = (omega, t, s), and its
    gradient: dU/dt = sum_i G_i, dU/ds = sum_i G_i . (Y0_i R),
    dU/dR = s Y0^T G, dU/domega_k = <dU/dR, dR/domega_k>, with G = dU/dY = -f
    and dR/domega_k the transpose of the column-form derivative.
    Also returns dU/dY0 = s G R^T."""
    pose7 = np.asarray(pose7, dtype=np.float64)
    w, t, s = pose7[:3], pose7[3:6], float(pose7[6])
    Y0 = np.asarray(Y0, dtype=np.float64)
    R = rodrigues(w)
    Y = s * Y0 @ R + t
    U = potential(Y, X, aY, aX, sigma, p, g_mode)
    G = potential_grad(Y, X, aY, aX, sigma, p, g_mode)
    g_t = G.sum(axis=0)
    g_s = float(np.sum(G * (Y0 @ R)))
    dUdR = s * Y0.T @ G
    g_w = np.array([np.sum(dUdR * dRc.T) for dRc in _drodrigues(w)])
    grad = np.concatenate([g_w, g_t, [g_s]])
    gY0 = s * G @ R.T
    return U, grad, gY0


# ----------------------------------------------------------------- pose update

def g_schedule(t, G1: float, E: float) -> float:
    """Eq. 12 with 0-based iteration t (reading R7)."""
    z = -(t - E / 2.0)
    logistic = 0.0 if z > 700.0 else 1.0 / (1.0 + math.exp(z))   # e^z overflows past ~709
    return 0.1 * G1 + 0.9 * G1 * logistic


def kabsch(Chat):
    """Eq. 6: C^ = U^ S^ V^T, d = sign det(V^ U^T), R = V^ diag(1,1,d) U^T.
    Returns (R, degenerate) with R11 for rank < 2."""
    U, S, Vt = np.linalg.svd(Chat)
    if not (S[0] > 0) or S[1] <= 1e-12 * S[0]:
        return np.eye(3), True
    V = Vt.T
    dd = 1.0 if np.linalg.det(V @ U.T) >= 0 else -1.0
    return V @ np.diag([1.0, 1.0, dd]) @ U.T, False


def scale_factor(eX: float, eY: float, mode: int = 0) -> float:
    """Sec. III-B: c from the largest covariance eigenvalues (reading R8)."""
    if mode == 2:
        return 1.0
    ratio = eX / eY
    return math.sqrt(ratio) if mode == 0 else ratio


def polar(R):
    """Nearest orthogonal matrix (polar factor) U V^T of R = U S V^T."""
    U, _, Vt = np.linalg.svd(R)
    return U @ Vt


def step_once(Y, X, desc, prm: Params, it: int, E: int, eX: float):
    """One iteration of the method on the current template Y (Eq. 5-12).

    Returns (Y_next, info) with info holding the increment (c, R_inc, d),
    the forces and the step size."""
    M = len(Y)
    G = g_schedule(it, prm.G1, E)                                   # Eq. 12
    f, Wi = forces(Y, X, desc["aY"], desc["aX"], desc["sigma"], prm.p, prm.g_mode)  # Eq. 5 / G
    F = f.sum(axis=0)
    W = float(Wi.sum())
    if prm.step_mode == 0:
        kappa = prm.eta0 * (G / prm.G1) * M / W if W > 0 else 0.0  # R6
    else:
        kappa = G * prm.time ** 2                                   # Eq. 5.5, m = 1, v = 0
    delta = kappa * f                                               # per-point displacement
    dvec = delta.mean(axis=0)                                       # Eq. 5.5: kappa F / M
    mu = Y.mean(axis=0)
    Yc = Y - mu
    YD = Yc + delta - dvec                                          # R10
    Chat = YD.T @ Yc                                                # Eq. 6
    Rinc, degenerate = kabsch(Chat)
    _, _, eY = cloud_stats(Y)
    c = scale_factor(eX, eY, prm.scale_mode)                        # Sec. III-B (R8)
    Ynext = c * Yc @ Rinc + mu + dvec                               # Eq. 8, Eq. 9 (R9)
    sym = 0.5 * (Chat + Chat.T)
    info = dict(G=G, F=F, W=W, kappa=kappa, d=dvec, mu=mu, c=c, Rinc=Rinc,
                degenerate=degenerate, Chat=Chat, f=f, Wi=Wi,
                lam_min_sym=float(np.linalg.eigvalsh(sym)[0]))
    return Ynext, info


def nearest(Q, X):
    """Nearest point of X for every query of Q under the float32 key of R1,
    ties to the lower index: (index, key)."""
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    idx = np.empty(len(Q), dtype=np.int32)
    key = np.empty(len(Q), dtype=np.float32)
    for i in range(len(Q)):
        dx = Q[i, 0] - X[:, 0]
        dy = Q[i, 1] - X[:, 1]
        dz = Q[i, 2] - X[:, 2]
        k = (dx * dx + dy * dy) + dz * dz
        j = int(np.argmin(k))              # first minimum: the lowest index among ties
        idx[i], key[i] = j, k[j]
    return idx, key


def change_mask(moved, X, threshold: float):
    """Change detection after registration (abstract, Sec. V): a moved
    template point is 'changed' if its nearest reference point is farther
    than the threshold (decided on the float32 key against threshold^2)."""
    _, key = nearest(moved, X)
    return (key > np.float32(threshold * threshold)).astype(np.uint8), np.sqrt(key.astype(np.float32))


def register_pyramid(X, Y0, prm: Params, levels):
    """Pyramidal schedule (Sec. IV): `levels` = [(iterations, k, radius_scale,
    sigma_scale), ...].  Each level recomputes the descriptors of both clouds
    with its neighbourhood and sigma, then continues the iterations from the
    current template (Eq. 9) and the current position in the Eq. 12 schedule
    (E = all levels' iterations unless prm.E is set)."""
    X64 = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y0, dtype=np.float64).copy()
    total = sum(lv[0] for lv in levels)
    E = prm.E if prm.E > 0 else total
    _, _, eX = cloud_stats(X64)
    s, R, t = 1.0, np.eye(3), np.zeros(3)
    it = 0
    for iters, k, rscale, sscale in levels:
        lp = replace(prm, k=k, radius_scale=rscale)
        desc = descriptors(X, Y0, lp, sigma_scale=sscale)
        for _ in range(iters):
            Y, info = step_once(Y, X64, desc, lp, it, E, eX)
            c, Rinc, mu, dvec = info["c"], info["Rinc"], info["mu"], info["d"]
            t = c * (t - mu) @ Rinc + mu + dvec
            R = polar(R @ Rinc)
            s = c * s
            it += 1
    return dict(R=R, t=t, s=s, Y=Y, iterations=it, E=E)


def partial_sums(Y, X, desc, prm: Params, rows):
    """Sums over the template rows `rows` at the current template Y: total
    force F (3), total weight W and the moment T = sum_i f_i (Y_i - ybar)^T
    (3x3, ybar the mean of the whole template).  Adding the sums of a
    partition of the rows gives the totals of one iteration (Eq. 5, 5.5, 6)."""
    Y = np.asarray(Y, dtype=np.float64)
    f, Wi = forces_rows(Y, X, desc["aY"], desc["aX"], desc["sigma"], prm.p, prm.g_mode, rows)
    ybar = Y.mean(axis=0)
    T = f.T @ (Y[rows] - ybar)
    return np.concatenate([f.sum(axis=0), [Wi.sum()], T.reshape(9)])


def update_from_totals(Y, totals, prm: Params, it: int, E: int, eX: float):
    """The update of `step_once` computed from the 13 totals of
    `partial_sums`: with Y_D = Y_c + delta - d, C^ = Y_D^T Y_c = Y_c^T Y_c + kappa T."""
    Y = np.asarray(Y, dtype=np.float64)
    totals = np.asarray(totals, dtype=np.float64)
    F, W, T = totals[:3], float(totals[3]), totals[4:].reshape(3, 3)
    M = len(Y)
    G = g_schedule(it, prm.G1, E)
    if prm.step_mode == 0:
        kappa = prm.eta0 * (G / prm.G1) * M / W if W > 0 else 0.0
    else:
        kappa = G * prm.time ** 2
    dvec = kappa * F / M
    mu = Y.mean(axis=0)
    Yc = Y - mu
    Chat = Yc.T @ Yc + kappa * T
    Rinc, degenerate = kabsch(Chat)
    _, _, eY = cloud_stats(Y)
    c = scale_factor(eX, eY, prm.scale_mode)
    return c * Yc @ Rinc + mu + dvec, dict(c=c, Rinc=Rinc, mu=mu, d=dvec, degenerate=degenerate)


def register_from_partials(X, Y0, prm: Params, iterations: int, desc, row_blocks, map_partials=map):
    """`register` with each iteration's totals (F, W, T; Eq. 5, 5.5, 6) added
    from `partial_sums` over a partition of the template rows, in block order,
    and the update taken by `update_from_totals`.  `map_partials(fn, args)`
    evaluates fn(args[b]) = partial_sums(Y, X, desc, prm, row_blocks[b]) for
    every block; the builtin map runs them in turn, a process pool's map runs
    them in parallel with the same result.  Returns R, t, s and the template,
    composed as in `register`."""
    X64 = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y0, dtype=np.float64).copy()
    E = prm.E if prm.E > 0 else iterations
    _, _, eX = cloud_stats(X64)
    s, R, t = 1.0, np.eye(3), np.zeros(3)
    for it in range(iterations):
        parts = list(map_partials(_partials_task, [(Y, X64, desc, prm, rows) for rows in row_blocks]))
        totals = np.zeros(13)
        for part in parts:                                          # block order
            totals = totals + part
        Ynext, info = update_from_totals(Y, totals, prm, it, E, eX)
        c, Rinc, mu, dvec = info["c"], info["Rinc"], info["mu"], info["d"]
        t = c * (t - mu) @ Rinc + mu + dvec
        R = polar(R @ Rinc)
        s = c * s
        Y = Ynext
    return dict(R=R, t=t, s=s, Y=Y, iterations=iterations, E=E)


def _partials_task(args):
    Y, X, desc, prm, rows = args
    return partial_sums(Y, X, desc, prm, rows)


def register(X, Y0, prm: Params | None = None, iterations: int = 100, desc=None,
             keep_history: bool = False, record_forces_at=()):
    """Run the method: descriptors once (R14), then `iterations` updates.

    The template is iterated literally by Eq. 9, and the composed similarity
    (s, R, t) with Y(t) = s Y0 R + t is tracked beside it:
    s <- c s, R <- polar(R R_inc), t <- c (t - mu) R_inc + mu + d.
    """
    prm = prm or Params()
    X64 = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y0, dtype=np.float64).copy()
    if desc is None:
        desc = descriptors(X, Y0, prm)
    E = prm.E if prm.E > 0 else iterations
    _, _, eX = cloud_stats(X64)
    s, R, t = 1.0, np.eye(3), np.zeros(3)
    hist = []
    forces_at = {}
    for it in range(iterations):
        Ynext, info = step_once(Y, X64, desc, prm, it, E, eX)
        if it in record_forces_at:
            forces_at[it] = (info["f"].copy(), info["Wi"].copy())
        c, Rinc, mu, dvec = info["c"], info["Rinc"], info["mu"], info["d"]
        t = c * (t - mu) @ Rinc + mu + dvec
        R = polar(R @ Rinc)
        s = c * s
        Y = Ynext
        if keep_history:
            hist.append(dict(it=it, s=s, R=R.copy(), t=t.copy(), G=info["G"], W=info["W"],
                             kappa=info["kappa"], F=info["F"].copy(), c=c,
                             degenerate=info["degenerate"], lam_min_sym=info["lam_min_sym"]))
    return dict(R=R, t=t, s=s, Y=Y, desc=desc, history=hist, forces_at=forces_at,
                iterations=iterations, E=E, params=replace(prm))
