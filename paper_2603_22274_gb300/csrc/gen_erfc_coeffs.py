"""Writes erfc_coeffs.h: this library's own fit of the scaled complementary
error function used by the FP32 pair kernels.

    erfc(t) ~= u * Q(u) * exp(-t^2),   u = 1 / (1 + P_SUB * t),   0 <= t <= T_MAX

Q is a degree-7 polynomial in u from Chebyshev interpolation (400 nodes) of
erfc(t) exp(t^2) / u on the u-interval [1/(1 + P_SUB T_MAX), 1], converted to
monomial coefficients for Horner evaluation. Evaluated in binary32 this gives
a maximum relative error of about 4e-7 on [0, 3.3] (Horner or Estrin). The
kernels share the factor exp(-t^2) with the force term, so erfc costs one
reciprocal and about ten multiply(-add)s per pair.

Run:  python gen_erfc_coeffs.py > erfc_coeffs.h
"""
import sys

import numpy as np
from numpy.polynomial import chebyshev as Ch
from scipy.special import erfcx

P_SUB = 0.5
T_MAX = 3.6
DEG = 7
NODES = 400


def fit():
    ulo = 1.0 / (1.0 + P_SUB * T_MAX)
    xs = np.cos(np.pi * (np.arange(NODES) + 0.5) / NODES)
    u = ulo + (xs + 1) / 2 * (1 - ulo)
    t = (1 / u - 1) / P_SUB
    q = erfcx(t) / u
    c = Ch.chebfit(2 * (u - ulo) / (1 - ulo) - 1, q, DEG)
    p = np.polynomial.Polynomial(Ch.cheb2poly(c))
    mono = p(np.polynomial.Polynomial([-(1 + ulo) / (1 - ulo), 2 / (1 - ulo)]))
    return mono.coef


def main(out=sys.stdout):
    c = fit()
    out.write("// Generated by gen_erfc_coeffs.py: erfc(t) ~= u*Q(u)*exp(-t*t), u = 1/(1+%.1f t),\n"
              % P_SUB)
    out.write("// Q(u) = sum_k ABFE_ERFC_Qk u^k, valid for 0 <= t <= %.1f (own Chebyshev fit).\n" % T_MAX)
    out.write("#pragma once\n")
    out.write("#define ABFE_ERFC_PSUB %.1ff\n" % P_SUB)
    out.write("#define ABFE_ERFC_TMAX %.1f\n" % T_MAX)
    out.write("#define ABFE_ERFC_DEG %d\n" % DEG)
    for k, v in enumerate(c):
        out.write("#define ABFE_ERFC_Q%d (%.9ef)\n" % (k, v))


if __name__ == "__main__":
    main()
