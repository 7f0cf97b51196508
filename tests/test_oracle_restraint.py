"""Pins of the restraint standard-state correction: the dihedral integral's
Bessel closed form, the distance integral's erf closed form, and the stiff
limit, where the harmonic (Boresch et al. 2003) expression becomes exact."""
import math

import pytest
from scipy.special import erf, i0e

from oracle.restraint import V0_NM3, boresch_correction, z_angle, z_dihedral, z_distance

KT = 0.00831446261815324 * 300.0


def test_dihedral_integral_is_bessel():
    for k in (4.184, 41.84, 334.72):
        x = k / KT
        # int_-pi^pi exp(-x (1 - cos p)) dp = 2 pi exp(-x) I0(x) = 2 pi i0e(x)
        assert z_dihedral(KT, k) == pytest.approx(2 * math.pi * i0e(x), rel=1e-11)


def test_distance_integral_closed_form():
    for r0, k in ((0.6, 4184.0), (0.3, 836.8), (0.05, 400.0)):
        a = 0.5 * k / KT
        s = math.sqrt(a)
        # int_0^inf r^2 exp(-a (r - r0)^2) dr
        closed = (math.sqrt(math.pi) * (1 + 2 * a * r0 ** 2) * (1 + erf(s * r0)) / (4 * a ** 1.5)
                  + r0 * math.exp(-a * r0 ** 2) / (2 * a))
        assert z_distance(KT, r0, k) == pytest.approx(closed, rel=1e-10)


def test_stiff_limit_is_the_harmonic_formula():
    """Boresch et al. (2003): the release of the restraint costs
    -kT ln[8 pi^2 V0 sqrt(k_r k_tA k_tB k_pA k_pB k_pC) / (r0^2 sin tA sin tB (2 pi kT)^3)];
    applying it is the negative, and that is the large-k limit of the exact value."""
    r0, th = 0.6, (1.4, 1.9)
    errs = []
    for scale in (1.0, 10.0, 100.0):
        kr, kt, kp = 4184.0 * scale, 41.84 * scale, 41.84 * scale
        harm = -KT * math.log(8 * math.pi ** 2 * V0_NM3 * math.sqrt(kr * kt * kt * kp ** 3)
                              / (r0 ** 2 * math.sin(th[0]) * math.sin(th[1]) * (2 * math.pi * KT) ** 3))
        errs.append(abs(boresch_correction(KT, r0, th, kr, kt, kp) - (-harm)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.02 * KT


def test_angle_integral_limits():
    # very stiff: sin(theta0) sqrt(2 pi kT / k); floppy (k -> 0): int_0^pi sin = 2
    th0, k = 1.2, 1e6
    assert z_angle(KT, th0, k) == pytest.approx(math.sin(th0) * math.sqrt(2 * math.pi * KT / k), rel=1e-4)
    assert z_angle(KT, th0, 1e-9) == pytest.approx(2.0, rel=1e-9)
