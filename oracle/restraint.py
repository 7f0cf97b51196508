"""Reference standard-state correction of the Boresch restraint (TEST INFRASTRUCTURE).

The paper adds the free energy of the restraints in the decoupled state,
computed analytically ("Restraints"), to the simulated legs; its closed form is
cited, not printed. This restates the quantity from its definition: with the
ligand decoupled, the restraint acts only on the six external coordinates
(distance r, angles theta_A, theta_B, dihedrals phi_A, phi_B, phi_C) whose
volume element is r^2 sin(theta_A) sin(theta_B) dr dtheta_A dtheta_B dphi_A dphi_B dphi_C,
so its partition function factorises into one-dimensional integrals, and

    dG = -kT ln( Z_r Z_thetaA Z_thetaB Z_phi^3 / (V0 8 pi^2) ),
    Z_r = int_0^inf r^2 exp(-(k_r/2)(r-r0)^2/kT) dr,
    Z_theta = int_0^pi sin(theta) exp(-(k_theta/2)(theta-theta0)^2/kT) dtheta,
    Z_phi = int_-pi^pi exp(-k_phi (1 - cos phi)/kT) dphi,

V0 = 1/(C0 N_A) = 1.66054 nm^3 at C0 = 1 mol/L, and 8 pi^2 the orientational
volume. The integrals are taken with scipy's adaptive quadrature (a library
step).
"""
from __future__ import annotations

import math

from scipy.integrate import quad

V0_NM3 = 1.0e24 / (6.02214076e23 * 1.0e3)    # 1 / (1 mol/L x N_A) in nm^3 = 1.66054


def z_distance(kT, r0, k_r):
    s = math.sqrt(kT / k_r)
    lo, hi = max(0.0, r0 - 40 * s), r0 + 40 * s
    f = lambda r: r * r * math.exp(-0.5 * k_r * (r - r0) ** 2 / kT)
    return quad(f, lo, hi, points=[r0], epsabs=0.0, epsrel=1e-13, limit=400)[0]


def z_angle(kT, theta0, k_theta):
    f = lambda t: math.sin(t) * math.exp(-0.5 * k_theta * (t - theta0) ** 2 / kT)
    return quad(f, 0.0, math.pi, points=[theta0], epsabs=0.0, epsrel=1e-13, limit=400)[0]


def z_dihedral(kT, k_phi):
    f = lambda p: math.exp(-k_phi * (1.0 - math.cos(p)) / kT)
    return quad(f, -math.pi, math.pi, points=[0.0], epsabs=0.0, epsrel=1e-13, limit=400)[0]


def boresch_correction(kT, r0, theta0, k_r, k_theta, k_phi):
    """Free energy (kJ/mol) of applying the restraint to the decoupled ligand at 1 mol/L."""
    Z = (z_distance(kT, r0, k_r) * z_angle(kT, theta0[0], k_theta) * z_angle(kT, theta0[1], k_theta)
         * z_dihedral(kT, k_phi) ** 3)
    return -kT * math.log(Z / (V0_NM3 * 8.0 * math.pi ** 2))
