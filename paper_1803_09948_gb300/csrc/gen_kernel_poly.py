"""Writes kernel_poly.h: polynomial fits used by the near-field (P2P) kernel.

With u = (k R)^2 the Helmholtz kernel splits into two even functions,
    exp(i k R) / R = k * ( C(u) / sqrt(u) + i S(u) ),
    C(u) = cos(sqrt u),   S(u) = sin(sqrt u) / sqrt u,
both entire in u, so on a bounded interval 0 <= u <= U low-degree polynomials
in u reproduce them to single precision with no range reduction and no
square root: one rsqrt and two Horner chains per source-target pair.

The coefficients are Chebyshev interpolants at Chebyshev points of [0, U]
(near-minimax), converted to the power basis in u.  The degree is the
smallest whose fit error (evaluated in float64) is below FIT_TARGET; the
float32 Horner evaluation then sits at the rounding floor (about 1.6e-7 for
C near u = U, where cos(sqrt u) passes close to zero; one degree more would
not move it, and costs an FMA per source-target pair).

Run:  python gen_kernel_poly.py   (rewrites kernel_poly.h next to this file)
"""
from __future__ import annotations

import os

import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as P

U_MAX = 2.5          # (kR)^2 <= 2.5, i.e. kR <= 1.58 rad
FIT_TARGET = 1e-7    # max abs error of the fit itself (exact arithmetic), at float32 rounding


def f_cos(u):
    return np.cos(np.sqrt(u))


def f_sinc(u):
    r = np.sqrt(u)
    out = np.ones_like(u)
    nz = r > 0
    out[nz] = np.sin(r[nz]) / r[nz]
    return out


def fit(fun, deg):
    # Chebyshev points on [0, U] -> interpolant -> power basis in u
    x = np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    u = 0.5 * U_MAX * (x + 1.0)
    cheb = C.chebfit(x, fun(u), deg)
    # p(x) with x = 2u/U - 1  ->  coefficients in u
    px = C.cheb2poly(cheb)
    coeff_u = np.zeros(deg + 1)
    lin = np.array([-1.0, 2.0 / U_MAX])
    term = np.array([1.0])
    for c in px:
        coeff_u[: term.size] += c * term
        term = P.polymul(term, lin)
    return coeff_u


def horner32(coeff, u):
    acc = np.float32(coeff[-1])
    u = u.astype(np.float32)
    for c in coeff[-2::-1]:
        acc = (acc * u + np.float32(c)).astype(np.float32)
    return acc


def best(fun):
    u = np.linspace(0.0, U_MAX, 20001)
    for deg in range(3, 12):
        c = fit(fun, deg)
        if np.max(np.abs(P.polyval(u, c) - fun(u))) < FIT_TARGET:
            return c, np.max(np.abs(horner32(c, u).astype(np.float64) - fun(u)))
    raise RuntimeError("no degree met the target")


def main():
    cc, ec = best(f_cos)
    cs, es = best(f_sinc)
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_kernel_poly.py -- do not edit.",
        "// C(u) = cos(sqrt u), S(u) = sin(sqrt u)/sqrt u on 0 <= u <= %.3f, power basis in u." % U_MAX,
        "// float32 Horner max abs error: C %.2e, S %.2e." % (ec, es),
        "#pragma once",
        "#define HFMM_POLY_UMAX %.9ef" % U_MAX,
        "#define HFMM_POLY_C_DEG %d" % (cc.size - 1),
        "#define HFMM_POLY_S_DEG %d" % (cs.size - 1),
        "#define HFMM_POLY_C_INIT {%s}" % ", ".join("%.9ef" % v for v in cc),
        "#define HFMM_POLY_S_INIT {%s}" % ", ".join("%.9ef" % v for v in cs),
        "",
    ]
    with open(os.path.join(here, "kernel_poly.h"), "w") as f:
        f.write("\n".join(lines))
    print("C degree", cc.size - 1, "err", ec, "| S degree", cs.size - 1, "err", es)


if __name__ == "__main__":
    main()
