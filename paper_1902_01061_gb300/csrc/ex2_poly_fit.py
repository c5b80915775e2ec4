"""Fit the polynomial of the FMA-pipe exponential used by the force kernel
and write it to ex2_poly.cuh (run from any directory:
``python paper_1902_01061_gb300/csrc/ex2_poly_fit.py``).

The force kernel needs 2^-e for e >= 0 (the similarity-and-aX factor of the
pair weight).  Besides the special-function unit's ex2, it can evaluate a
part of these on the FP32 pipe by Cody-Waite range reduction,
e = n + g with n = round(e) and g in [-1/2, 1/2], 2^-e = 2^-n 2^-g,
where 2^-g comes from a polynomial and 2^-n is added to the float's exponent
field.  The polynomial here is the degree-5 minimax approximation of 2^-g on
[-1/2, 1/2] in relative error, found by the Remez exchange algorithm in
float64 and then rounded to float32 coefficients.
"""
import os

import numpy as np

DEGREE = 5
LO, HI = -0.5, 0.5


def target(x):
    return np.exp2(-x)


def remez(deg=DEGREE, iters=30):
    """Minimax polynomial c_0 + c_1 x + ... of 2^-x on [LO, HI], weight 1/2^-x
    (relative error).  Returns (coefficients, levelled error)."""
    n = deg + 2
    k = np.arange(n)
    x = 0.5 * (LO + HI) + 0.5 * (HI - LO) * np.cos(np.pi * k[::-1] / (n - 1))   # Chebyshev extrema
    dense = np.linspace(LO, HI, 200001)
    for _ in range(iters):
        # p(x_i) - f(x_i) = (-1)^i E f(x_i): unknowns c_0..c_deg, E
        A = np.zeros((n, n))
        for i in range(n):
            A[i, :deg + 1] = x[i] ** np.arange(deg + 1)
            A[i, deg + 1] = -((-1) ** i) * target(x[i])
        sol = np.linalg.solve(A, target(x))
        c, E = sol[:deg + 1], sol[deg + 1]
        err = (np.polyval(c[::-1], dense) - target(dense)) / target(dense)
        # new reference: the extremum of each sign-alternating run of the error
        sgn = np.sign(err)
        breaks = np.nonzero(np.diff(sgn) != 0)[0] + 1
        runs = np.split(np.arange(len(dense)), breaks)
        ext = [r[np.argmax(np.abs(err[r]))] for r in runs if len(r)]
        if len(ext) < n:
            break
        # keep n alternating extrema with the largest errors
        while len(ext) > n:
            drop = 0 if abs(err[ext[0]]) < abs(err[ext[-1]]) else len(ext) - 1
            ext.pop(drop)
        x = dense[np.array(ext)]
    return c, abs(E)


def f32_horner(c32, g):
    """float32 Horner evaluation with one rounding per fused multiply-add
    (float64 intermediate: the product of two float32 values is exact)."""
    p = np.full_like(g, c32[-1], dtype=np.float32)
    for ck in c32[-2::-1]:
        p = (p.astype(np.float64) * g.astype(np.float64) + np.float64(ck)).astype(np.float32)
    return p


def main():
    c, E = remez()
    c32 = c.astype(np.float32)
    g = np.linspace(LO, HI, 400001).astype(np.float32)
    rel = np.abs(f32_horner(c32, g).astype(np.float64) / target(g.astype(np.float64)) - 1.0)
    lines = [
        "// Generated by ex2_poly_fit.py: degree-%d minimax polynomial of 2^-g on [-1/2, 1/2]" % DEGREE,
        "// (relative error), Remez exchange in float64, coefficients rounded to float32.",
        "// Levelled error of the float64 fit: %.3e; float32 Horner evaluation, max relative" % E,
        "// error on a 400,001-point grid: %.3e." % rel.max(),
        "#pragma once",
        "namespace scgr {",
        "constexpr int EX2_POLY_DEGREE = %d;" % DEGREE,
    ]
    for k, v in enumerate(c32):
        lines.append("constexpr float EX2_POLY_C%d = %sf;" % (k, np.format_float_scientific(v, unique=True)))
    lines.append("}  // namespace scgr")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ex2_poly.cuh")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(out, E, rel.max())


if __name__ == "__main__":
    main()
