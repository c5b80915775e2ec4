"""Pins of the oracle's force (Eq. 5 with Eq. 3, Eq. 10, Eq. 11; readings
R4, R5, R12) and potential: a hand-worked two-point case, the p = 1 closed
forms, Newton's third law, equivariances, homogeneity and finite differences."""
import math

import numpy as np
import pytest

import oracle as O


def rand_case(seed, n=40, m=30):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 3))
    Y = rng.normal(size=(m, 3)) + np.array([0.5, -0.2, 0.1])
    aX = rng.uniform(0.0, 0.3, n)
    aY = rng.uniform(0.0, 0.3, m)
    return X, Y, aX, aY


def test_two_point_hand_case():
    # X at the origin, Y at (1,0,0), equal curvature a: s = 1, g = a^2 (Eq. 10),
    # h(1) = 1, n = (1,0,0): f = -a^2 (1,0,0), W = a^2
    a = 0.2
    X = np.zeros((1, 3)); Y = np.array([[1.0, 0, 0]])
    f, W = O.forces(Y, X, np.array([a]), np.array([a]), 0.1, 2.0, 1)
    np.testing.assert_allclose(f, [[-a * a, 0, 0]], rtol=1e-15)
    np.testing.assert_allclose(W, [a * a], rtol=1e-15)
    # p = 3 at distance 2 along -y: h = 8, n = (0,-1,0): f = +8 a^2 (0,1,0), W = a^2 * 4
    Y2 = np.array([[0.0, -2.0, 0]])
    f, W = O.forces(Y2, X, np.array([a]), np.array([a]), 0.1, 3.0, 1)
    np.testing.assert_allclose(f, [[0, 8 * a * a, 0]], rtol=1e-15)
    np.testing.assert_allclose(W, [4 * a * a], rtol=1e-15)
    # different curvatures: aX = 0.1, aY = 0.3, sigma = 0.2 -> s = e^-1 (Eq. 3)
    f, W = O.forces(Y, X, np.array([0.3]), np.array([0.1]), 0.2, 2.0, 1)
    np.testing.assert_allclose(f, [[-0.03 * math.exp(-1.0), 0, 0]], rtol=1e-14)
    f0, _ = O.forces(Y, X, np.array([0.3]), np.array([0.1]), 0.2, 2.0, 0)   # g = s
    np.testing.assert_allclose(f0, [[-math.exp(-1.0), 0, 0]], rtol=1e-14)


def test_coincident_pair_contributes_nothing():
    X = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    Y = np.array([[1.0, 2.0, 3.0]])
    a = np.array([0.1, 0.1])
    for p in (1.0, 2.0, 1.5):
        f, W = O.forces(Y, X, a[:1], a, 0.05, p, 1)
        f_only, W_only = O.forces(Y, X[1:], a[:1], a[1:], 0.05, p, 1)
        np.testing.assert_allclose(f, f_only, rtol=1e-15)
        extra = 0.01 if p == 1.0 else 0.0     # d^(p-1) at d = 0 is 1 for p = 1, else 0
        np.testing.assert_allclose(W, W_only + extra, rtol=1e-15)


def test_p1_equal_similarity_closed_form():
    # p = 1, g = s = 1 (equal curvatures): f_i = -sum_j (Y_i - X_j) = -N (Y_i - xbar)
    X, Y, _, _ = rand_case(1)
    a = np.full(len(X), 0.1); b = np.full(len(Y), 0.1)
    f, W = O.forces(Y, X, b, a, 0.3, 1.0, 0)
    np.testing.assert_allclose(f, -len(X) * (Y - X.mean(axis=0)), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(W, np.full(len(Y), float(len(X))), rtol=1e-14)


def test_p1_moment_closed_form():
    # p = 1 general: f_i = -aY_i (Y_i S0_i - S1_i), S0_i = sum_j aX_j s_ij, S1_i = sum_j aX_j s_ij X_j
    X, Y, aX, aY = rand_case(2)
    sigma = 0.07
    S = np.exp(-np.subtract.outer(aY, aX) ** 2 / sigma ** 2)      # [m, n]
    S0 = S @ aX
    S1 = (S * aX[None, :]) @ X
    expect = -aY[:, None] * (Y * S0[:, None] - S1)
    f, W = O.forces(Y, X, aY, aX, sigma, 1.0, 1)
    np.testing.assert_allclose(f, expect, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(W, aY * S0, rtol=1e-12)


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0, 1.5])
def test_newton_third_law(p):
    X, Y, aX, aY = rand_case(3)
    fY, _ = O.forces(Y, X, aY, aX, 0.1, p, 1)
    fX, _ = O.forces(X, Y, aX, aY, 0.1, p, 1)
    np.testing.assert_allclose(fY.sum(axis=0), -fX.sum(axis=0), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("p", [2.0, 1.5])
def test_translation_and_rotation_equivariance(p):
    X, Y, aX, aY = rand_case(4)
    f, W = O.forces(Y, X, aY, aX, 0.1, p, 1)
    tau = np.array([3.0, -7.0, 0.25])
    f2, W2 = O.forces(Y + tau, X + tau, aY, aX, 0.1, p, 1)
    np.testing.assert_allclose(f2, f, rtol=1e-11, atol=1e-12)
    Q, _ = np.linalg.qr(np.random.default_rng(9).normal(size=(3, 3)))
    f3, W3 = O.forces(Y @ Q, X @ Q, aY, aX, 0.1, p, 1)
    np.testing.assert_allclose(f3, f @ Q, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(W3, W, rtol=1e-12)


@pytest.mark.parametrize("p", [1.0, 2.0, 3.0, 1.5])
def test_homogeneity_in_scale(p):
    X, Y, aX, aY = rand_case(5)
    f, W = O.forces(Y, X, aY, aX, 0.1, p, 1)
    lam = 1.7
    f2, W2 = O.forces(lam * Y, lam * X, aY, aX, 0.1, p, 1)
    np.testing.assert_allclose(f2, lam ** p * f, rtol=1e-11)
    np.testing.assert_allclose(W2, lam ** (p - 1) * W, rtol=1e-11)


def test_forces_rows_subset():
    X, Y, aX, aY = rand_case(6)
    f, W = O.forces(Y, X, aY, aX, 0.1, 2.0, 1)
    rows = np.array([3, 0, 17])
    fr, Wr = O.forces_rows(Y, X, aY, aX, 0.1, 2.0, 1, rows)
    np.testing.assert_array_equal(fr, f[rows])
    np.testing.assert_array_equal(Wr, W[rows])


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
def test_force_is_minus_potential_gradient(p):
    X, Y, aX, aY = rand_case(7, n=25, m=6)
    f, _ = O.forces(Y, X, aY, aX, 0.1, p, 1)
    h = 1e-5
    for i in range(len(Y)):
        for c in range(3):
            Yp = Y.copy(); Yp[i, c] += h
            Ym = Y.copy(); Ym[i, c] -= h
            fd = (O.potential(Yp, X, aY, aX, 0.1, p, 1) - O.potential(Ym, X, aY, aX, 0.1, p, 1)) / (2 * h)
            assert abs(fd + f[i, c]) <= 1e-6 * max(1.0, abs(f[i, c]))
    np.testing.assert_array_equal(O.potential_grad(Y, X, aY, aX, 0.1, p, 1), -f)


def test_pose_gradient_matches_finite_differences():
    X, Y0, aX, aY = rand_case(8, n=30, m=12)
    pose = np.array([0.3, -0.2, 0.5, 0.1, 0.2, -0.3, 1.2])
    U, g, gY0 = O.pose_potential_and_grad(pose, Y0, X, aY, aX, 0.1, 2.0, 1)
    h = 1e-6
    for q in range(7):
        pp = pose.copy(); pp[q] += h
        pm = pose.copy(); pm[q] -= h
        Up = O.pose_potential_and_grad(pp, Y0, X, aY, aX, 0.1, 2.0, 1)[0]
        Um = O.pose_potential_and_grad(pm, Y0, X, aY, aX, 0.1, 2.0, 1)[0]
        assert abs((Up - Um) / (2 * h) - g[q]) <= 1e-6 * max(1.0, abs(g[q]))
    # template coordinates
    for i in (0, 5):
        for c in range(3):
            Yp = Y0.copy(); Yp[i, c] += h
            Ym = Y0.copy(); Ym[i, c] -= h
            Up = O.pose_potential_and_grad(pose, Yp, X, aY, aX, 0.1, 2.0, 1)[0]
            Um = O.pose_potential_and_grad(pose, Ym, X, aY, aX, 0.1, 2.0, 1)[0]
            assert abs((Up - Um) / (2 * h) - gY0[i, c]) <= 1e-6 * max(1.0, abs(gY0[i, c]))


def test_pose_gradient_at_zero_rotation():
    X, Y0, aX, aY = rand_case(12, n=20, m=8)
    pose = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    _, g, _ = O.pose_potential_and_grad(pose, Y0, X, aY, aX, 0.1, 2.0, 1)
    h = 1e-6
    for q in range(3):
        pp = pose.copy(); pp[q] += h
        pm = pose.copy(); pm[q] -= h
        fd = (O.pose_potential_and_grad(pp, Y0, X, aY, aX, 0.1, 2.0, 1)[0]
              - O.pose_potential_and_grad(pm, Y0, X, aY, aX, 0.1, 2.0, 1)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(g[q]))


@pytest.mark.parametrize("p", [1.0, 2.0, 1.5])
def test_force_vjp_matches_central_differences(p):
    X, Y, aX, aY = rand_case(10, n=25, m=5)
    v = np.random.default_rng(11).normal(size=(5, 3))
    got = O.force_vjp(Y, X, aY, aX, 0.1, p, 1, v)
    h = 1e-6
    for i in range(len(Y)):
        J = np.zeros((3, 3))
        for c in range(3):
            Yp = Y.copy(); Yp[i, c] += h
            Ym = Y.copy(); Ym[i, c] -= h
            fp, _ = O.forces_rows(Yp, X, aY, aX, 0.1, p, 1, [i])
            fm, _ = O.forces_rows(Ym, X, aY, aX, 0.1, p, 1, [i])
            J[:, c] = (fp[0] - fm[0]) / (2 * h)
        np.testing.assert_allclose(got[i], J.T @ v[i], rtol=1e-6, atol=1e-9)


def test_row_magnitudes_hand_cases():
    # one reference point: the sum has a single term, so A = |f| (kappa = 1)
    a = 0.2
    X = np.array([[0.0, 0.0, 0.0]])
    Y = np.array([[0.0, 3.0, 4.0]])                    # d = 5
    mg = O.force_row_magnitudes(Y, X, np.array([a]), np.array([a]), 0.1, 2.0, 1, centre=np.array([1.0, 0.0, 0.0]))
    f, Wf = O.forces(Y, X, np.array([a]), np.array([a]), 0.1, 2.0, 1)
    assert mg["A"][0] == pytest.approx(np.linalg.norm(f[0]), rel=1e-15)
    assert mg["A"][0] == pytest.approx(a * a * 5.0 * 5.0, rel=1e-15)     # w = a^2 d, |r| = d
    assert mg["W"][0] == pytest.approx(Wf[0], rel=1e-15)
    assert mg["B"][0] == pytest.approx(a * a * 5.0 * 1.0, rel=1e-15)     # |X - centre| = 1
    # equal curvatures: s = 1, so e = -ln aX (g = aX aY s) or 0 (g = s)
    assert mg["We"][0] == pytest.approx(mg["W"][0] * -math.log(a), rel=1e-14)
    assert mg["Ae"][0] == pytest.approx(mg["A"][0] * -math.log(a), rel=1e-14)
    m0 = O.force_row_magnitudes(Y, X, np.array([a]), np.array([a]), 0.1, 2.0, 0)
    assert m0["We"][0] == 0.0 and m0["Ae"][0] == 0.0
    # aX = 0.1, aY = 0.3, sigma = 0.2: e = 1 - ln 0.1 (Eq. 3 exponent and the aX factor)
    m1 = O.force_row_magnitudes(Y, X, np.array([0.3]), np.array([0.1]), 0.2, 2.0, 1)
    assert m1["We"][0] / m1["W"][0] == pytest.approx(1.0 - math.log(0.1), rel=1e-14)
    # two equal pulls from opposite sides: f = 0, A = 2 w d (kappa infinite)
    X2 = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]])
    Y2 = np.zeros((1, 3))
    aa = np.array([a, a])
    f2, _ = O.forces(Y2, X2, np.array([a]), aa, 0.1, 1.5, 1)
    m2 = O.force_row_magnitudes(Y2, X2, np.array([a]), aa, 0.1, 1.5, 1)
    assert np.linalg.norm(f2) == 0.0
    assert m2["A"][0] == pytest.approx(2 * a * a, rel=1e-15)


def test_row_magnitudes_match_term_list():
    # brute force over the pair terms, written out per pair with math.*
    X, Y, aX, aY = rand_case(11, n=9, m=4)
    sigma, p = 0.08, 1.5
    c = np.array([0.3, -0.1, 0.2])
    mg = O.force_row_magnitudes(Y, X, aY, aX, sigma, p, 1, rows=np.array([2, 0]), centre=c)
    for out_i, i in enumerate((2, 0)):
        sums = dict(A=0.0, B=0.0, W=0.0, Ae=0.0, We=0.0)
        for j in range(len(X)):
            r = [Y[i][q] - X[j][q] for q in range(3)]
            d = math.sqrt(r[0] ** 2 + r[1] ** 2 + r[2] ** 2)
            expo = (aX[j] - aY[i]) ** 2 / sigma ** 2
            g = aX[j] * aY[i] * math.exp(-expo)
            w = g * d ** (p - 1.0)
            e = expo - math.log(aX[j])
            sums["A"] += w * d
            sums["B"] += w * math.sqrt(sum((X[j][q] - c[q]) ** 2 for q in range(3)))
            sums["W"] += w
            sums["Ae"] += w * d * e
            sums["We"] += w * e
        for key, value in sums.items():
            assert mg[key][out_i] == pytest.approx(value, rel=1e-13), key
