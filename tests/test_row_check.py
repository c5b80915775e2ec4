"""The per-row force check of the GPU tests (tests/gpu_helpers.check_rows),
exercised on the CPU: it accepts the oracle's own forces rounded to float32,
accepts rows whose true force lies below float32's range when the GPU path
returns 0 for them (its weights flush to zero there), and rejects a single
row perturbed far beyond its condition-scaled bound while the relative L2
over all rows would still pass."""
import numpy as np
import pytest

import oracle as O
from paper_1902_01061_gb300 import synth
from tests.gpu_helpers import check_rows, rel_l2


@pytest.fixture(scope="module")
def ragged():
    sc = synth.scale_case()
    X = sc.X[synth.subsample(sc.X, 800, 3)]
    Y0 = sc.Y0[synth.subsample(sc.Y0, 700, 4)]
    d = O.descriptors(X, Y0, O.Params(p=2.0))
    f, W = O.forces(Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)
    return X, Y0, d, f, W


def test_float32_rounded_oracle_passes(ragged):
    X, Y0, d, f, W = ragged
    got = np.c_[f, W].astype(np.float32)
    check_rows("oracle rounded to float32", got, f, W, Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)


def test_underflowing_rows_may_read_zero(ragged):
    X, Y0, d, f, W = ragged
    aY = d["aY"].copy()
    aY[5] = 0.33                       # far from every reference curvature: the similarity underflows
    f2, W2 = O.forces(Y0, X, aY, d["aX"], d["sigma"], 2.0, 1)
    assert 0 < np.linalg.norm(f2[5]) < 1e-38
    got = np.c_[f2, W2].astype(np.float32)
    got[5] = 0.0
    check_rows("underflowing row read as 0", got, f2, W2, Y0, X, aY, d["aX"], d["sigma"], 2.0, 1)


def test_one_bad_row_is_caught(ragged):
    X, Y0, d, f, W = ragged
    got = np.c_[f, W].astype(np.float64)
    i = int(np.argmax(np.linalg.norm(f, axis=1) < np.median(np.linalg.norm(f, axis=1))))
    got[i, :3] *= 1.0 + 3e-4           # a 3e-4 relative error in one row
    assert rel_l2(got[:, :3], f) < 1e-5
    with pytest.raises(AssertionError):
        check_rows("one bad row", got, f, W, Y0, X, d["aY"], d["aX"], d["sigma"], 2.0, 1)
