"""Pins of the curvature descriptor (Sec. III-A, Sec. IV; reading R2:
a = lambda_min / trace of the 1/k neighbourhood covariance) and sigma (R3)."""
import numpy as np
import pytest

import oracle as O


def curv_all(P):
    P = np.asarray(P, dtype=np.float64)
    nb = np.tile(np.arange(len(P)), (len(P), 1))
    return O.curvature(P, nb)


def test_planar_neighbourhood_is_zero():
    rng = np.random.default_rng(0)
    P = np.c_[rng.uniform(-1, 1, (20, 2)), np.zeros(20)]
    np.testing.assert_allclose(curv_all(P), 0.0, atol=1e-15)


def test_collinear_neighbourhood_is_zero():
    t = np.linspace(-1, 1, 9)
    P = np.c_[t, 2 * t, -t]
    np.testing.assert_allclose(curv_all(P), 0.0, atol=1e-15)


def test_axis_star_is_one_third():
    P = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    # covariance = (2/7) I, isotropic: lambda_min / trace = 1/3
    np.testing.assert_allclose(curv_all(P), 1.0 / 3.0, rtol=1e-14)


def test_box_corners_one_fourteenth():
    P = np.array([[x, y, z] for x in (-1, 1) for y in (-2, 2) for z in (-3, 3)], float)
    # covariance = diag(1, 4, 9): a = 1 / 14
    np.testing.assert_allclose(curv_all(P), 1.0 / 14.0, rtol=1e-14)


def test_axis_pairs_general_lengths():
    a, b, c = 0.7, 1.9, 0.4
    P = np.array([[a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0], [0, 0, c], [0, 0, -c]])
    # covariance = diag(a^2, b^2, c^2) / 3
    np.testing.assert_allclose(curv_all(P), c * c / (a * a + b * b + c * c), rtol=1e-13)


def test_similarity_invariance():
    rng = np.random.default_rng(5)
    P = rng.normal(size=(40, 3))
    nb = O.knn(P.astype(np.float32), 8)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    a0 = O.curvature(P, nb)
    a1 = O.curvature(2.5 * P @ Q + np.array([3.0, -1.0, 0.5]), nb)
    np.testing.assert_allclose(a1, a0, rtol=1e-10, atol=1e-14)


def test_sigma_population_std():
    # two-valued population {0, 0.2} in equal parts: std = 0.1 exactly
    a = np.array([0.0, 0.2] * 50)
    assert abs(O.sigma_auto(a) - 0.1) < 1e-15
    assert O.sigma_auto(np.full(10, 0.05)) == 1.0      # degenerate spread -> 1


def test_radius_curvature_hand_cases():
    # axis star, e = 2/7; a radius of 1.2 (between 1 and sqrt 2): the centre sees all 7 points -> 1/3, each
    # outer point sees itself and the centre (two points, collinear) -> 0
    P = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    a = O.curvature_radius(P, radius_scale=1.2 / np.sqrt(2.0 / 7.0))
    assert a[0] == pytest.approx(1.0 / 3.0, rel=1e-12)
    np.testing.assert_allclose(a[1:], 0.0, atol=1e-15)
    # a radius large enough for the whole cloud reproduces the whole-cloud kNN curvature
    rng = np.random.default_rng(3)
    Q = (rng.normal(size=(30, 3)) * np.array([3.0, 1.0, 0.2])).astype(np.float32)   # inputs are float32
    big = O.curvature_radius(Q, radius_scale=100.0)
    ref = O.curvature(Q, np.tile(np.arange(30), (30, 1)))
    np.testing.assert_allclose(big, ref, rtol=1e-10)


def test_radius_curvature_planar_cloud_is_zero():
    rng = np.random.default_rng(4)
    P = np.c_[rng.uniform(-1, 1, (60, 2)), np.zeros(60)]
    np.testing.assert_allclose(O.curvature_radius(P), 0.0, atol=1e-15)
