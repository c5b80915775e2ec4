"""The FP32-pipe exponential of the force kernel (ex2_neg_poly2 in force.cu),
emulated step by step in float32 on the CPU: Cody-Waite reduction by adding
1.5 * 2^23, the degree-5 polynomial of csrc/ex2_poly.cuh by fused
multiply-adds, and the exponent added to the float's bit pattern.  Its
relative error against the exact 2^-e stays below 2^-22 on [0, 125.5), it is
exactly 0 from 125.5 up (and at +inf, the padding weight), and the committed
coefficients are the ones the generator script fits."""
import importlib.util
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1902_01061_gb300", "csrc")


def header_coefficients():
    text = open(os.path.join(CSRC, "ex2_poly.cuh")).read()
    deg = int(re.search(r"EX2_POLY_DEGREE = (\d+);", text).group(1))
    return [np.float32(float(re.search(rf"EX2_POLY_C{k} = ([-+0-9.eE]+)f;", text).group(1))) for k in range(deg + 1)]


def fma32(a, b, c):
    # one rounding: the float32 product is exact in float64
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def ex2_neg_poly(e):
    e = np.asarray(e, np.float32)
    R = np.float32(12582912.0)
    with np.errstate(invalid="ignore", over="ignore"):
        t = (R - e).astype(np.float32)
        nf = (t - R).astype(np.float32)
        g = (e + nf).astype(np.float32)
        c = header_coefficients()
        q = np.full_like(g, c[-1])
        for ck in c[-2::-1]:
            q = fma32(q, g, np.full_like(g, ck))
        bits = (q.view(np.uint32).astype(np.uint64) + (t.view(np.uint32).astype(np.uint64) << np.uint64(23)))
        r = (bits & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where(e < np.float32(125.5), r, np.float32(0.0))


def test_relative_error_below_2_pow_minus_22():
    rng = np.random.default_rng(3)
    e = np.concatenate([np.linspace(0.0, 125.49, 2_000_001, dtype=np.float32),
                        rng.uniform(0.0, 125.5, 1_000_000).astype(np.float32),
                        np.arange(0, 126, dtype=np.float32), np.arange(0, 125, dtype=np.float32) + 0.5])
    e = e[e < 125.5]
    got = ex2_neg_poly(e).astype(np.float64)
    want = np.exp2(-e.astype(np.float64))
    rel = np.abs(got / want - 1.0)
    assert rel.max() < 2.0 ** -22, rel.max()


def test_zero_from_the_underflow_threshold_and_for_padding():
    e = np.array([125.5, 126.0, 130.0, 1e6, np.inf], np.float32)
    assert np.all(ex2_neg_poly(e) == 0.0)
    assert ex2_neg_poly(np.array([0.0], np.float32))[0] == pytest.approx(1.0, rel=2e-7)


def test_header_matches_generator():
    spec = importlib.util.spec_from_file_location("ex2_poly_fit", os.path.join(CSRC, "ex2_poly_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    c, E = mod.remez()
    assert E < 1e-7
    np.testing.assert_array_equal(c.astype(np.float32), np.array(header_coefficients(), np.float32))
