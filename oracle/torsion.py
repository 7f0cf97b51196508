"""Reference periodic torsions of rotatable ligand bonds (TEST INFRASTRUCTURE).

The paper scales the periodic torsional potentials of the ligand's rotatable
bonds linearly with the alchemical parameter ("Double annihilation protocol").
Reading taken: the torsions are scaled by lambda_v, the parameter of the
steric (vdW) stage, so that they are fully on until the vdW stage and off in
the annihilated state; when the ligand is decoupled (ligand_mode 1, the
ligand's internal interactions kept) they stay at full strength.

    U_T(x; lambda) = s(lambda) sum_t k_t [1 + cos(n_t phi_t - phi0_t)],
    s = lambda_v (annihilation) or 1 (decoupling),

phi_t the dihedral angle of atoms (a, b, c, d) about the b-c bond, with
b1 = x_b - x_a, b2 = x_c - x_b, b3 = x_d - x_c (nearest images) and
phi = atan2(|b2| b1 . (b2 x b3), (b1 x b2) . (b2 x b3)) (IUPAC sign: positive
for a clockwise rotation of the far bond seen along b-c).

Forces are minus the gradient by the chain rule through atan2: with
y = |b2| b1 . (b2 x b3) and x = (b1 x b2) . (b2 x b3)
= (b1.b2)(b2.b3) - (b1.b3)(b2.b2), d phi = (x dy - y dx) / (x^2 + y^2), and the
b-vector gradients map onto the atoms as a: -g1, b: g1 - g2, c: g2 - g3, d: g3.
Plain numpy in FP64, all torsions at once.
"""
from __future__ import annotations

import numpy as np


def _bvecs(s, pos):
    idx = np.asarray(s.torsions, dtype=np.int64).reshape(-1, 4)
    x = np.asarray(s.pos if pos is None else pos, dtype=np.float64)
    box = np.asarray(s.box, dtype=np.float64)

    def sep(i, j):
        d = x[idx[:, j]] - x[idx[:, i]]
        return d - box * np.round(d / box)

    return idx, sep(0, 1), sep(1, 2), sep(2, 3)


def dihedrals(s, pos=None):
    """The dihedral angle phi_t (radians, in (-pi, pi]) of every torsion."""
    _, b1, b2, b3 = _bvecs(s, pos)
    n1, n2 = np.cross(b1, b2), np.cross(b2, b3)
    y = np.linalg.norm(b2, axis=1) * np.einsum("ij,ij->i", b1, n2)
    xx = np.einsum("ij,ij->i", n1, n2)
    return np.arctan2(y, xx)


def torsions(s, lam_v, pos=None, forces=True, ligand_mode=0):
    """(U_T unscaled, forces of s(lambda) U_T or None, dU/dlambda_v).

    U_T unscaled = sum_t k_t [1 + cos(n_t phi_t - phi0_t)]; the state's energy
    is s(lambda) U_T and its lambda_v derivative U_T (annihilation) or 0."""
    x = np.asarray(s.pos if pos is None else pos, dtype=np.float64)
    m = len(np.asarray(s.torsions).reshape(-1, 4))
    if m == 0:
        return 0.0, (np.zeros_like(x) if forces else None), 0.0
    k = np.asarray(s.torsion_k, dtype=np.float64)
    n = np.asarray(s.torsion_n, dtype=np.float64)
    p0 = np.asarray(s.torsion_phi0, dtype=np.float64)
    idx, b1, b2, b3 = _bvecs(s, x)
    n1, n2 = np.cross(b1, b2), np.cross(b2, b3)
    lb2 = np.linalg.norm(b2, axis=1)
    y = lb2 * np.einsum("ij,ij->i", b1, n2)
    xx = np.einsum("ij,ij->i", n1, n2)
    phi = np.arctan2(y, xx)
    U = float(np.sum(k * (1.0 + np.cos(n * phi - p0))))
    scale = float(lam_v) if ligand_mode == 0 else 1.0
    dudl = U if ligand_mode == 0 else 0.0
    if not forces:
        return U, None, dudl
    # d U_t / d phi_t, times the state's scale
    dUdphi = -scale * k * n * np.sin(n * phi - p0)
    d12 = np.einsum("ij,ij->i", b1, b2)[:, None]
    d23 = np.einsum("ij,ij->i", b2, b3)[:, None]
    d13 = np.einsum("ij,ij->i", b1, b3)[:, None]
    d22 = np.einsum("ij,ij->i", b2, b2)[:, None]
    # y = |b2| b1.(b2 x b3): gradients with respect to b1, b2, b3
    t = np.einsum("ij,ij->i", b1, n2)[:, None]
    dy1 = lb2[:, None] * n2
    dy2 = (b2 / lb2[:, None]) * t + lb2[:, None] * np.cross(b3, b1)
    dy3 = lb2[:, None] * n1
    # x = (b1.b2)(b2.b3) - (b1.b3)(b2.b2)
    dx1 = b2 * d23 - b3 * d22
    dx2 = b1 * d23 + b3 * d12 - 2.0 * b2 * d13
    dx3 = b2 * d12 - b1 * d22
    den = (xx * xx + y * y)[:, None]
    g1 = (xx[:, None] * dy1 - y[:, None] * dx1) / den
    g2 = (xx[:, None] * dy2 - y[:, None] * dx2) / den
    g3 = (xx[:, None] * dy3 - y[:, None] * dx3) / den
    F = np.zeros_like(x)
    c = -dUdphi[:, None]                       # force = -dU/dphi * dphi/dx
    np.add.at(F, idx[:, 0], c * (-g1))
    np.add.at(F, idx[:, 1], c * (g1 - g2))
    np.add.at(F, idx[:, 2], c * (g2 - g3))
    np.add.at(F, idx[:, 3], c * g3)
    return U, F, dudl
