"""Whole-loop pins of the oracle: the paper's constants, and recovery of a
known synthetic similarity transform (the must-converge 15-degree case).
The paper gives no numeric convergence figure for its method, so the
thresholds here are this project's acceptance bar, not the paper's."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1902_01061_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def paper_constants():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def rot_err_deg(Ra, Rb):
    c = (np.trace(Ra.T @ Rb) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def test_defaults_follow_paper_constants():
    k = paper_constants()
    prm = O.Params()
    assert prm.G1 == k["G1"]
    E = k["E"]
    assert O.g_schedule(-1e3, prm.G1, E) / prm.G1 == pytest.approx(k["G_ratio_start"])
    assert O.g_schedule(E + 1e3, prm.G1, E) / prm.G1 == pytest.approx(k["G_ratio_end"])


def test_recovers_mild_transform():
    case = synth.mild()
    res = O.register(case.X, case.Y0, O.Params(), iterations=case.iterations)
    R, t, s = case.inverse_pose()
    assert rot_err_deg(res["R"], R) < 5.0          # from 15 degrees
    assert res["s"] == pytest.approx(s, rel=5e-3)
    rmse = float(np.sqrt(np.mean(np.sum((res["Y"] - case.X) ** 2, axis=1))))
    assert rmse < 0.02 * synth.bbox_diag(case.X)


def test_paper_rotation_reduced():
    # Fig. 1 setting: 50 degrees about x.  Under the readings the method
    # reduces the error but does not finish within 100 iterations; this pins
    # the direction of travel and the one-step scale recovery.
    case = synth.tiny()
    assert paper_constants()["fig1_rotation_deg"] == 50
    res = O.register(case.X, case.Y0, O.Params(eta0=0.7), iterations=case.iterations)
    R, t, s = case.inverse_pose()
    assert rot_err_deg(res["R"], R) < 25.0
    assert res["s"] == pytest.approx(s, rel=5e-3)


def test_pyramid_single_level_equals_register():
    case = synth.mild(n=300)
    prm = O.Params()
    a = O.register_pyramid(case.X, case.Y0, prm, [(8, 16, 1.0, 1.0)])
    b = O.register(case.X, case.Y0, prm, iterations=8)
    np.testing.assert_allclose(a["Y"], b["Y"], atol=1e-12)
    assert a["s"] == pytest.approx(b["s"], rel=1e-14)


def test_pyramid_two_equal_levels_equal_one_long_level():
    """Two identical levels of n iterations equal one level of 2n: the
    template (Eq. 9) and the position in the Eq. 12 schedule carry over from
    one level to the next (E = all levels' iterations)."""
    case = synth.mild(n=250)
    prm = O.Params(p=2.0)
    a = O.register_pyramid(case.X, case.Y0, prm, [(5, 16, 1.0, 1.0), (5, 16, 1.0, 1.0)])
    b = O.register(case.X, case.Y0, prm, iterations=10)
    np.testing.assert_allclose(a["Y"], b["Y"], atol=1e-12)
    np.testing.assert_allclose(a["R"], b["R"], atol=1e-12)
    np.testing.assert_allclose(a["t"], b["t"], atol=1e-12)
    assert a["s"] == pytest.approx(b["s"], rel=1e-14)
    assert a["E"] == b["E"] == 10


def test_pyramid_sigma_scale_multiplies_reference_std():
    """A level with sigma_scale = lam runs with sigma = lam * (population std
    of the reference curvatures) of that level's neighbourhood (Sec. IV with
    reading R3): the same as a plain run with that sigma given explicitly."""
    case = synth.mild(n=250)
    prm = O.Params(p=2.0)
    lam = 0.6
    aX = O.curvature(case.X, O.knn(case.X, 12))
    a = O.register_pyramid(case.X, case.Y0, prm, [(6, 12, 1.0, lam)])
    b = O.register(case.X, case.Y0, O.Params(p=2.0, k=12, sigma=lam * O.sigma_auto(aX)), iterations=6)
    np.testing.assert_allclose(a["Y"], b["Y"], atol=1e-12)
    assert a["s"] == pytest.approx(b["s"], rel=1e-14)


def test_pyramid_second_level_uses_its_own_descriptors():
    """Level 2 continues level 1's template with descriptors recomputed on the
    input clouds (R14) for its own k and sigma: its first update equals one
    step of the method from level 1's template with those descriptors, at
    schedule position n1 of the horizon n1 + n2."""
    case = synth.mild(n=250)
    prm = O.Params(p=2.0)
    n1 = 4
    two = O.register_pyramid(case.X, case.Y0, prm, [(n1, 16, 1.0, 1.0), (1, 8, 1.0, 0.7)])
    # level 1 alone with the horizon of the two-level run
    lv1 = O.register(case.X, case.Y0, O.Params(p=2.0, E=n1 + 1), iterations=n1)
    d8 = O.descriptors(case.X, case.Y0, O.Params(p=2.0, k=8), sigma_scale=0.7)
    eX = O.cloud_stats(case.X)[2]
    Y2, _ = O.step_once(lv1["Y"], np.asarray(case.X, np.float64), d8, O.Params(p=2.0, k=8), n1, n1 + 1, eX)
    np.testing.assert_allclose(two["Y"], Y2, atol=1e-12)
