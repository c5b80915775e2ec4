"""Pins of the pose update: Eq. 12 schedule, Kabsch (Eq. 6), scale model
(Sec. III-B, R8), polar factor, the fixed point at the aligned pose and the
consistency of the composed pose with the literal Eq. 9 iteration."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1902_01061_gb300 import synth


def rot(axis, deg):
    return synth.rotation_matrix(axis, deg)


def test_g_schedule_closed_form():
    G1, E = 1e4, 400
    assert O.g_schedule(200, G1, E) == pytest.approx(0.55 * G1, rel=1e-15)
    assert O.g_schedule(0, G1, E) == pytest.approx(0.1 * G1, rel=1e-12)
    assert O.g_schedule(399, G1, E) == pytest.approx(G1, rel=1e-12)
    # logistic step: G(E/2 + 1) - 0.1 G1 = 0.9 G1 / (1 + e^-1)
    assert O.g_schedule(201, G1, E) == pytest.approx(0.1 * G1 + 0.9 * G1 / (1 + math.exp(-1)), rel=1e-15)


def test_kabsch_recovers_known_rotation():
    rng = np.random.default_rng(1)
    Yc = rng.normal(size=(50, 3)); Yc -= Yc.mean(axis=0)
    Q = rot([0.2, -0.5, 0.8], 73.0)
    R, deg = O.kabsch((Yc @ Q).T @ Yc)
    assert not deg
    np.testing.assert_allclose(R, Q, atol=1e-12)


def test_kabsch_planar_cloud_needs_sign_fix():
    rng = np.random.default_rng(2)
    Yc = np.c_[rng.normal(size=(30, 2)), np.zeros(30)]; Yc -= Yc.mean(axis=0)
    Q = rot([1.0, 1.0, 0.3], 120.0)
    R, deg = O.kabsch((Yc @ Q).T @ Yc)
    assert not deg
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(Yc @ R, Yc @ Q, atol=1e-12)


def test_kabsch_reflection_gives_proper_rotation():
    # axis pairs: Yc^T Yc = diag(18, 8, 2); the mirrored "after" cloud gives
    # C^ = diag(18, 8, -2), whose unconstrained fit is the mirror itself
    Yc = np.array([[3.0, 0, 0], [-3.0, 0, 0], [0, 2.0, 0], [0, -2.0, 0], [0, 0, 1.0], [0, 0, -1.0]])
    P = np.diag([1.0, 1.0, -1.0])
    R, _ = O.kabsch((Yc @ P).T @ Yc)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(R, np.eye(3), atol=1e-12)   # best proper fit of a z-mirror


def test_kabsch_degenerate_rank_one():
    t = np.linspace(-1, 1, 11)
    Yc = np.c_[t, 2 * t, 3 * t]
    R, deg = O.kabsch(Yc.T @ Yc)
    assert deg
    np.testing.assert_array_equal(R, np.eye(3))


def test_scale_factor_and_polar():
    assert O.scale_factor(4.0, 1.0, 0) == pytest.approx(2.0)
    assert O.scale_factor(4.0, 1.0, 1) == pytest.approx(4.0)
    assert O.scale_factor(4.0, 1.0, 2) == 1.0
    Q = rot([0.3, 0.1, -0.9], 40.0)
    np.testing.assert_allclose(O.polar(Q), Q, atol=1e-15)
    A = Q @ (np.eye(3) + 1e-3 * np.array([[0, 1, 2], [1, 0, 3], [2, 3, 0]]))   # symmetric stretch
    np.testing.assert_allclose(O.polar(A), Q, atol=1e-12)


def small_pair(n=300, seed=4):
    rng = np.random.default_rng(seed)
    surf = synth.EllipsoidUnion.random(rng, 3)
    return surf.sample_surface(rng, n).astype(np.float32)


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_fixed_point_at_alignment(p):
    X = small_pair()
    prm = O.Params(p=p)
    res = O.register(X, X.copy(), prm, iterations=6, keep_history=True)
    np.testing.assert_allclose(res["R"], np.eye(3), atol=1e-12)
    np.testing.assert_allclose(res["t"], 0.0, atol=1e-12)
    assert res["s"] == pytest.approx(1.0, abs=1e-12)
    for h in res["history"]:
        assert np.abs(h["F"]).max() < 1e-9 * max(1.0, h["W"])


def test_scaled_copy_recovered_in_one_step():
    X = small_pair(seed=5)
    lam = 1.7
    res = O.register(X, (lam * X.astype(np.float64)).astype(np.float32), O.Params(), iterations=1)
    assert res["s"] == pytest.approx(1.0 / lam, rel=1e-6)    # float32 rounding of the scaled input


def test_composed_pose_matches_literal_iteration():
    case = synth.mild(n=400)
    res = O.register(case.X, case.Y0, O.Params(p=1.0), iterations=12)
    Ypose = res["s"] * case.Y0.astype(np.float64) @ res["R"] + res["t"]
    np.testing.assert_allclose(Ypose, res["Y"], atol=1e-10)
    np.testing.assert_allclose(res["R"] @ res["R"].T, np.eye(3), atol=1e-13)


def test_rodrigues_is_the_matrix_exponential_in_row_vector_form():
    """rodrigues(w) = exp([w]_x)^T (so that y = x @ R rotates x by |w| about
    w, right-handed), against scipy's matrix exponential and a hand case;
    near zero the series branch agrees with the closed form."""
    from scipy.linalg import expm
    rng = np.random.default_rng(3)
    for w in [np.array([0.0, 0.0, math.pi / 2]), rng.normal(size=3), 1e-3 * rng.normal(size=3), 2.5 * rng.normal(size=3)]:
        K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
        R = O.rodrigues(w)
        np.testing.assert_allclose(R, expm(K).T, atol=1e-13)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
    # +90 degrees about z takes x to y in the row-vector convention
    np.testing.assert_allclose(np.array([1.0, 0.0, 0.0]) @ O.rodrigues([0.0, 0.0, math.pi / 2]), [0.0, 1.0, 0.0],
                               atol=1e-15)
    w = np.array([3e-13, -1e-13, 2e-13])
    K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    np.testing.assert_allclose(O.rodrigues(w), (np.eye(3) + K).T, atol=1e-20)


def test_cloud_stats_closed_form():
    """Mean, 1/n covariance and largest eigenvalue (Sec. III-B) of the six
    points centre +- a e_x, +- b e_y, +- c e_z: covariance diag(a^2, b^2, c^2)/3;
    and numpy's biased covariance on a random cloud."""
    a, b, c = 2.0, 0.5, 1.0
    centre = np.array([0.3, -1.0, 4.0])
    P = centre + np.array([[a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0], [0, 0, c], [0, 0, -c]])
    mu, C, lam = O.cloud_stats(P)
    np.testing.assert_allclose(mu, centre, atol=1e-15)
    np.testing.assert_allclose(C, np.diag([a * a, b * b, c * c]) / 3.0, atol=1e-15)
    assert lam == pytest.approx(a * a / 3.0, rel=1e-14)
    Q = np.random.default_rng(4).normal(size=(200, 3)) @ np.diag([1.0, 2.0, 0.5])
    _, C2, lam2 = O.cloud_stats(Q)
    np.testing.assert_allclose(C2, np.cov(Q.T, bias=True), atol=1e-14)
    assert lam2 == pytest.approx(np.linalg.eigvalsh(np.cov(Q.T, bias=True))[-1], rel=1e-13)
