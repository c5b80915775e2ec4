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
