"""One pose update on the GPU from given totals (scgr_step_apply) against the
oracle's update from the same totals (Eq. 5.5, Eq. 6, Eq. 8, Eq. 9).  The
totals are chosen so that C^ = S_yy + kappa T takes each branch of the
Kabsch step: det C^ > 0 with a moderate condition number (the polar factor
by Newton's iteration in float32 with two float64 corrections, including a
170 degree rotation), a condition number near 1e4 (beyond the float32
iteration's limit of about 1e3: Newton's iteration in float64), det C^ < 0
(the reflection fix of Eq. 6 through the SVD), and a nearly rank-2 C^
(beyond the float64 iteration's limit: the SVD)."""
import numpy as np
import pytest

import oracle as O
from paper_1902_01061_gb300 import scgr, synth
from tests.gpu_helpers import Gpu, check

pytestmark = pytest.mark.gpu

E = 10


@pytest.fixture(scope="module", autouse=True)
def _lib(scgr_lib):
    return scgr_lib


def rotation(axis, deg):
    a = np.asarray(axis, np.float64)
    return synth.rotation_matrix(a / np.linalg.norm(a), deg)


def chat_target(Syy, kind):
    U, S, Vt = np.linalg.svd(Syy)
    if kind == "rotated":          # C^ = Q H with a proper Q: det > 0
        return rotation([0.3, -0.5, 0.8], 35.0) @ Syy
    if kind == "identity":         # T = 0: C^ = S_yy, R_inc = I
        return Syy.copy()
    if kind == "reflected":        # det < 0: the third axis flips
        return rotation([1.0, 2.0, -0.5], 20.0) @ Syy @ np.diag([1.0, 1.0, -1.0])
    if kind == "rank2":            # smallest singular value 1e-9 of the largest
        return rotation([0.0, 1.0, 1.0], 50.0) @ U @ np.diag([S[0], S[1], 1e-9 * S[0]]) @ Vt
    if kind == "halfturn":         # a polar factor far from the identity
        return rotation([-0.2, 0.7, 0.4], 170.0) @ Syy
    if kind == "cond3e2":          # within the float32 iteration's range
        return rotation([0.6, 0.1, -0.3], 25.0) @ U @ np.diag([S[0], 0.4 * S[0], S[0] / 300.0]) @ Vt
    if kind == "cond1e4":          # beyond it: the float64 iteration
        return rotation([0.6, 0.1, -0.3], 25.0) @ U @ np.diag([S[0], 0.4 * S[0], 1e-4 * S[0]]) @ Vt
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["identity", "rotated", "halfturn", "cond3e2", "cond1e4", "reflected", "rank2"])
def test_step_from_totals_matches_oracle(kind):
    case = synth.mild(n=700)
    Y = case.Y0.astype(np.float64)
    M = len(Y)
    prm = O.Params(E=E)
    W = float(M)                                         # kappa = eta0 G / G1
    kappa = prm.eta0 * O.g_schedule(0, prm.G1, E) / prm.G1 * M / W
    Yc = Y - Y.mean(axis=0)
    Syy = Yc.T @ Yc
    Ch = chat_target(Syy, kind)
    T = (Ch - Syy) / kappa
    F = np.array([0.3, -0.2, 0.1]) * W
    tot = np.concatenate([F, [W], T.reshape(9)])
    if kind == "reflected":
        assert np.linalg.det(Ch) < 0
    eX = O.cloud_stats(case.X)[2]
    Ynew, info = O.update_from_totals(Y, tot, prm, 0, E, eX)
    with Gpu(case.X, case.Y0, E=E) as g:
        scgr.scgr_step_apply(g.ctx, tot)
        R, t, s = scgr.scgr_get_result(g.ctx).as_numpy()
        moved = g.moved()
    t_ref = -info["c"] * info["mu"] @ info["Rinc"] + info["mu"] + info["d"]
    np.testing.assert_allclose(R, info["Rinc"], atol=1e-9)
    check(f"Kabsch step ({kind}): max |R - R_oracle|", np.abs(R - info["Rinc"]).max(), 1e-9)
    assert abs(np.linalg.det(R) - 1.0) <= 1e-12
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
    assert s == pytest.approx(info["c"], rel=1e-10)
    np.testing.assert_allclose(t, t_ref, atol=1e-9 * (1.0 + np.abs(t_ref).max()))
    np.testing.assert_allclose(moved, Ynew, rtol=0, atol=2e-6 * np.abs(Ynew).max())
