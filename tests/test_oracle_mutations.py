"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in
the oracle (on the CPU, by patching one of its functions) and runs the pins
that should expose it; at least one must fail."""
import math

import numpy as np
import pytest

import oracle.scgr_oracle as M
from tests import test_oracle_curvature as TC
from tests import test_oracle_forces as TF
from tests import test_oracle_knn as TK
from tests import test_oracle_pose as TP
from tests import test_oracle_register as TR


def _pair_terms_sign(Yi, X, aYi, aX, sigma, p, g_mode):
    r, d, g = ORIG["_pair_terms"](Yi, X, aYi, aX, sigma, p, g_mode)
    return -r, d, g                                   # n_ij pointing the wrong way


def _pair_terms_no_square(Yi, X, aYi, aX, sigma, p, g_mode):
    r, d, _ = ORIG["_pair_terms"](Yi, X, aYi, aX, sigma, p, g_mode)
    s = np.exp(-np.abs(aX[None, :] - aYi[:, None]) / sigma ** 2)   # |.| instead of |.|^2 in Eq. 3
    g = aX[None, :] * aYi[:, None] * s if g_mode == 1 else s
    return r, d, g


def _pair_terms_drop_aY(Yi, X, aYi, aX, sigma, p, g_mode):
    r, d, g = ORIG["_pair_terms"](Yi, X, aYi, aX, sigma, p, g_mode)
    if g_mode == 1:
        g = g / np.where(aYi[:, None] > 0, aYi[:, None], 1.0)      # Eq. 10 without aY
    return r, d, g


def _forces_rows_exponent(Y, X, aY, aX, sigma, p, g_mode, rows=None):
    return ORIG["forces_rows"](Y, X, aY, aX, sigma, p - 1.0 if p > 1.0 else p + 1.0, g_mode, rows)  # h = d^(p-1)


def _curvature_lmax(P, nbr):
    Q = np.asarray(P, dtype=np.float64)[nbr]
    D = Q - Q.mean(axis=1)[:, None, :]
    C = np.einsum("nki,nkj->nij", D, D) / Q.shape[1]
    lam = np.linalg.eigvalsh(C)
    tr = np.trace(C, axis1=1, axis2=2)
    return np.where(tr > 0, lam[:, -1] / np.where(tr > 0, tr, 1), 0.0)   # largest eigenvalue


def _curvature_no_centre(P, nbr):
    Q = np.asarray(P, dtype=np.float64)[nbr]
    C = np.einsum("nki,nkj->nij", Q, Q) / Q.shape[1]                    # mean not subtracted
    lam = np.linalg.eigvalsh(C)
    tr = np.trace(C, axis1=1, axis2=2)
    return np.where(tr > 0, np.maximum(lam[:, 0], 0) / np.where(tr > 0, tr, 1), 0.0)


def _kabsch_transposed(Chat):
    return ORIG["kabsch"](np.asarray(Chat).T)


def _kabsch_no_reflection_fix(Chat):
    U, S, Vt = np.linalg.svd(Chat)
    return Vt.T @ U.T, False


def _knn_ties_high(P, k):
    P = np.ascontiguousarray(P, dtype=np.float32)
    out = np.empty((len(P), k), dtype=np.int32)
    for q in range(len(P)):
        d = P[q] - P
        key = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        order = np.lexsort((-np.arange(len(P)), key))                # ties to the higher index
        out[q] = order[:k]
    return out


def _knn_fma_key(P, k):
    P64 = np.asarray(P, dtype=np.float64)
    out = np.empty((len(P), k), dtype=np.int32)
    for q in range(len(P)):
        key = np.sum((P64[q] - P64) ** 2, axis=1).astype(np.float32)    # key not rounded per operation
        out[q] = np.lexsort((np.arange(len(P)), key))[:k]
    return out


def _scale_no_sqrt(eX, eY, mode=0):
    return eX / eY if mode != 2 else 1.0


def _g_schedule_sign(t, G1, E):
    return 0.1 * G1 + 0.9 * G1 / (1.0 + math.exp(min(700.0, (t - E / 2.0))))


def _rodrigues_column_form(omega):
    return ORIG["rodrigues"](omega).T                 # column-vector matrix used in a row-vector product


def _cloud_stats_unbiased(P):
    P = np.asarray(P, dtype=np.float64)
    mu = P.mean(axis=0)
    D = P - mu
    C = D.T @ D / (len(P) - 1)                        # 1/(n-1) instead of the 1/n of Sec. III-B
    return mu, C, float(np.linalg.eigvalsh(C)[-1])


def _pyramid_variant(position_reset=False, sigma_from_template=False, descriptors_on_moved=False):
    """register_pyramid with one level-switch mistake planted (a copy of the
    oracle's loop; the shared steps are the oracle's own functions)."""
    from dataclasses import replace as dc_replace

    def run(X, Y0, prm, levels):
        X64 = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y0, dtype=np.float64).copy()
        total = sum(lv[0] for lv in levels)
        E = prm.E if prm.E > 0 else total
        _, _, eX = M.cloud_stats(X64)
        s, R, t = 1.0, np.eye(3), np.zeros(3)
        it = 0
        for iters, k, rscale, sscale in levels:
            lp = dc_replace(prm, k=k, radius_scale=rscale)
            desc = M.descriptors(X, Y.astype(np.float32) if descriptors_on_moved else Y0, lp, sigma_scale=sscale)
            if sigma_from_template:
                desc["sigma"] = M.sigma_auto(desc["aY"]) * sscale
            if position_reset:
                it = 0
            for _ in range(iters):
                Y, info = M.step_once(Y, X64, desc, lp, it, E, eX)
                c, Rinc, mu, dvec = info["c"], info["Rinc"], info["mu"], info["d"]
                t = c * (t - mu) @ Rinc + mu + dvec
                R = M.polar(R @ Rinc)
                s = c * s
                it += 1
        return dict(R=R, t=t, s=s, Y=Y, iterations=it, E=E)
    return run


ORIG = {name: getattr(M, name) for name in
        ("_pair_terms", "forces_rows", "curvature", "kabsch", "knn", "scale_factor", "g_schedule", "rodrigues",
         "cloud_stats", "register_pyramid")}

CASES = {
    "force sign": ("_pair_terms", _pair_terms_sign, [TF.test_two_point_hand_case]),
    "similarity without square": ("_pair_terms", _pair_terms_no_square, [TF.test_two_point_hand_case]),
    "g without aY": ("_pair_terms", _pair_terms_drop_aY, [TF.test_two_point_hand_case, TF.test_p1_moment_closed_form]),
    "distance exponent": ("forces_rows", _forces_rows_exponent,
                          [TF.test_two_point_hand_case, TF.test_p1_equal_similarity_closed_form]),
    "largest eigenvalue": ("curvature", _curvature_lmax, [TC.test_box_corners_one_fourteenth]),
    "uncentred covariance": ("curvature", _curvature_no_centre, [TC.test_planar_neighbourhood_is_zero,
                                                                 TC.test_similarity_invariance]),
    "Kabsch transposed": ("kabsch", _kabsch_transposed, [TP.test_kabsch_recovers_known_rotation]),
    "Kabsch without reflection fix": ("kabsch", _kabsch_no_reflection_fix,
                                      [TP.test_kabsch_reflection_gives_proper_rotation]),
    "kNN ties to the higher index": ("knn", _knn_ties_high, [TK.test_knn_ties_go_to_lower_index]),
    "kNN key not rounded per operation": ("knn", _knn_fma_key, [TK.test_knn_matches_scalar_bruteforce_random,
                                                                 TK.test_knn_key_is_rounded_per_operation]),
    "scale without square root": ("scale_factor", _scale_no_sqrt, [TP.test_scale_factor_and_polar]),
    "schedule sign": ("g_schedule", _g_schedule_sign, [TP.test_g_schedule_closed_form]),
    "axis-angle rotation transposed": ("rodrigues", _rodrigues_column_form,
                                       [TP.test_rodrigues_is_the_matrix_exponential_in_row_vector_form]),
    "unbiased covariance": ("cloud_stats", _cloud_stats_unbiased, [TP.test_cloud_stats_closed_form]),
    "pyramid: Eq. 12 position reset per level": ("register_pyramid", _pyramid_variant(position_reset=True),
                                                 [TR.test_pyramid_two_equal_levels_equal_one_long_level]),
    "pyramid: sigma from the template curvatures": ("register_pyramid", _pyramid_variant(sigma_from_template=True),
                                                    [TR.test_pyramid_sigma_scale_multiplies_reference_std]),
    "pyramid: descriptors of the moved template": ("register_pyramid", _pyramid_variant(descriptors_on_moved=True),
                                                   [TR.test_pyramid_second_level_uses_its_own_descriptors]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_planted_mistake_is_caught(name, monkeypatch):
    target, mutant, pins = CASES[name]
    monkeypatch.setattr(M, target, mutant)
    import oracle
    if hasattr(oracle, target):
        monkeypatch.setattr(oracle, target, mutant)
    caught = 0
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError):
            caught += 1
    assert caught >= 1, f"no pin caught: {name}"
