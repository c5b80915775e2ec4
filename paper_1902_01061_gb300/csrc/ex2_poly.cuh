// Generated by ex2_poly_fit.py: degree-5 minimax polynomial of 2^-g on [-1/2, 1/2]
// (relative error), Remez exchange in float64, coefficients rounded to float32.
// Levelled error of the float64 fit: 7.494e-08; float32 Horner evaluation, max relative
// error on a 400,001-point grid: 2.121e-07.
#pragma once
namespace scgr {
constexpr int EX2_POLY_DEGREE = 5;
constexpr float EX2_POLY_C0 = 1.0000001e+00f;
constexpr float EX2_POLY_C1 = -6.9314694e-01f;
constexpr float EX2_POLY_C2 = 2.402212e-01f;
constexpr float EX2_POLY_C3 = -5.550713e-02f;
constexpr float EX2_POLY_C4 = 9.675541e-03f;
constexpr float EX2_POLY_C5 = -1.3276472e-03f;
}  // namespace scgr
