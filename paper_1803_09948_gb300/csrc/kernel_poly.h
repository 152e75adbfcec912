// Generated by gen_kernel_poly.py -- do not edit.
// C(u) = cos(sqrt u), S(u) = sin(sqrt u)/sqrt u on 0 <= u <= 2.500, power basis in u.
// float32 Horner max abs error: C 1.60e-07, S 9.16e-08.
#pragma once
#define HFMM_POLY_UMAX 2.500000000e+00f
#define HFMM_POLY_C_DEG 4
#define HFMM_POLY_S_DEG 4
#define HFMM_POLY_C_INIT {9.999999499e-01f, -4.999989971e-01f, 4.166345081e-02f, -1.385271084e-03f, 2.313129436e-05f}
#define HFMM_POLY_S_INIT {9.999999954e-01f, -1.666665748e-01f, 8.333038945e-03f, -1.980817435e-04f, 2.603169116e-06f}
