"""Pins of the oracle's rotatable-bond torsions (oracle/torsion.py) against
geometry fixed by construction, closed-form values at special angles, finite
differences, lambda endpoints, rigid-motion invariance and periodic images.
None of these calls the CUDA path."""
import math

import numpy as np
import pytest

import abfe_synth as S
import oracle as O
from oracle.torsion import dihedrals, torsions


def _quad(phi, box=10.0, shift=(5.0, 5.0, 5.0)):
    """b at the origin, c on +z, a on +x, d rotated by phi about the b->c axis
    (counter-clockwise seen from +z, i.e. clockwise looking from b to c)."""
    a = np.array([1.0, 0.0, 0.0])
    b = np.zeros(3)
    c = np.array([0.0, 0.0, 1.0])
    d = np.array([math.cos(phi), math.sin(phi), 1.0])
    return np.stack([a, b, c, d]) + np.asarray(shift)


def _system(pos, k, n, phi0, box=10.0, lig=True):
    m = len(pos)
    s = S.System("t", np.full(3, float(box)), np.asarray(pos, float), np.zeros((m, 3)),
                 np.ones(m), np.zeros(m), np.zeros(m), np.zeros(m),
                 np.full(m, 1 if lig else 0, np.uint8), np.zeros((0, 2), np.int32),
                 np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0))
    s.torsions = np.array([[0, 1, 2, 3]], np.int32)
    s.torsion_k = np.array([k], float)
    s.torsion_n = np.array([n], np.int32)
    s.torsion_phi0 = np.array([phi0], float)
    return s


@pytest.mark.parametrize("deg", [0.0, 60.0, 90.0, 180.0, -120.0, -45.0])
def test_dihedral_of_constructed_geometry(deg):
    phi = math.radians(deg)
    s = _system(_quad(phi), 1.0, 1, 0.0)
    got = dihedrals(s)[0]
    # +-180 degrees are the same angle
    assert math.isclose(math.cos(got), math.cos(phi), abs_tol=1e-12)
    assert math.isclose(math.sin(got), math.sin(phi), abs_tol=1e-12)


@pytest.mark.parametrize("deg,n,phi0,val", [
    (180.0, 1, 0.0, 0.0),          # trans: 1 + cos(180) = 0
    (0.0, 1, 0.0, 2.0),            # cis: 1 + cos(0) = 2
    (90.0, 1, 0.0, 1.0),           # 1 + cos(90) = 1
    (90.0, 2, math.pi, 2.0),       # 1 + cos(180 - 180) = 2
    (-90.0, 1, math.pi / 2, 0.0),  # 1 + cos(-90 - 90) = 0
])
def test_energy_at_special_angles(deg, n, phi0, val):
    k = 2.5
    s = _system(_quad(math.radians(deg)), k, n, phi0)
    U, _, _ = torsions(s, 1.0, forces=False)
    assert U == pytest.approx(k * val, abs=1e-12)


def test_threefold_phase_pi_values():
    """n = 3, phi0 = pi: minima at 0 and +-120 degrees (1 + cos(-pi) = 0),
    maxima at 60 and 180 degrees (1 + cos(0) = 2)."""
    k = 1.7
    for deg, val in ((0.0, 0.0), (120.0, 0.0), (-120.0, 0.0), (60.0, 2.0), (180.0, 2.0)):
        s = _system(_quad(math.radians(deg)), k, 3, math.pi)
        assert torsions(s, 1.0, forces=False)[0] == pytest.approx(k * val, abs=1e-12)


def _chain_system(seed=3, box=3.0):
    rng = np.random.default_rng(seed)
    lig = S.make_ligand(rng, 20)   # torsions only across angles <= 135 degrees: 7 of 17 bonds
    pos = lig["xyz"] + box / 2
    m = len(pos)
    s = S.System("chain", np.full(3, box), pos, np.zeros((m, 3)), np.ones(m), np.zeros(m),
                 np.zeros(m), np.zeros(m), np.ones(m, np.uint8), np.zeros((0, 2), np.int32),
                 np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0))
    s.torsions, s.torsion_k, s.torsion_n, s.torsion_phi0 = S.ligand_torsions(lig, 0, p_rotatable=1.0)
    return s


@pytest.mark.parametrize("lam_v", [1.0, 0.37])
def test_forces_are_minus_gradient(lam_v):
    s = _chain_system()
    assert len(s.torsions) >= 5
    U, F, _ = torsions(s, lam_v)
    h = 1e-6
    for i in range(s.n):
        for a in range(3):
            xp, xm = s.pos.copy(), s.pos.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -lam_v * (torsions(s, 1.0, pos=xp, forces=False)[0] -
                           torsions(s, 1.0, pos=xm, forces=False)[0]) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_lambda_endpoints_and_modes():
    s = _chain_system()
    U1, F1, d1 = torsions(s, 1.0)
    U0, F0, d0 = torsions(s, 0.0)
    assert U0 == U1 and d0 == d1 == U1          # unscaled energy and its lambda_v derivative
    assert np.abs(F0).max() == 0.0               # annihilated: no torsion force
    # decoupling keeps the ligand's internal terms: full forces, no lambda dependence
    Ud, Fd, dd = torsions(s, 0.0, ligand_mode=1)
    assert dd == 0.0
    np.testing.assert_allclose(Fd, F1, rtol=0, atol=0)
    # the state helper: lambda_v U_T when annihilating, U_T when decoupling
    P = dict(ligand_mode=0)
    assert O.torsion_state(s, P, 0.25, forces=False)[0] == pytest.approx(0.25 * U1, rel=1e-15)
    assert O.torsion_state(s, dict(ligand_mode=1), 0.25, forces=False)[0] == U1


def test_rigid_motion_invariance_net_force_and_torque():
    s = _chain_system()
    U, F, _ = torsions(s, 1.0)
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).max()
    c = s.pos.mean(0)
    torque = np.cross(s.pos - c, F).sum(0)
    assert np.abs(torque).max() < 1e-10 * np.abs(F).max()
    th = 0.7
    rot = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    moved = (s.pos - c) @ rot.T + c + np.array([0.1, -0.2, 0.05])
    assert torsions(s, 1.0, pos=moved, forces=False)[0] == pytest.approx(U, rel=1e-12)


def test_periodic_images():
    """A torsion whose atoms straddle the box edge: wrapping the coordinates
    into the box leaves the angle and the energy unchanged."""
    box = 2.0
    q = _quad(math.radians(75.0), shift=(1.6, 1.7, 1.3))
    s = _system(q, 3.0, 2, 0.4, box=box)
    U0 = torsions(s, 1.0, forces=False)[0]
    wrapped = np.mod(q, box)
    assert (wrapped != q).any()
    assert torsions(s, 1.0, pos=wrapped, forces=False)[0] == pytest.approx(U0, rel=1e-12)


def test_generated_torsions_shared_by_both_legs():
    lig = S.make_ligand(np.random.default_rng(11), 30)
    a = S.ligand_torsions(lig, 0)
    b = S.ligand_torsions(lig, 100)
    np.testing.assert_array_equal(a[0] + 100, b[0])
    for u, v in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(u, v)
    c = S.complex_leg(9, n_atoms=9000, core_diameter=2.2, n_lig=20)
    assert len(c.torsions) > 0 and c.is_ligand[c.torsions].all()


def test_ukn_lambda_part_includes_torsions():
    """u_k from whole-state energies minus the lambda part is the same at every
    state (the torsions move with lambda_v into the lambda part)."""
    s = S.solvent_leg(6, n_lig=20, box=2.2, n_atoms=1100)
    assert len(s.torsions) > 0
    P = S.params_for(1.0, 3.12)
    sch = S.schedule_solvent_k30()
    full = O.ukn(s, P, sch) * P["kT"]
    part = O.ukn_lambda_part(s, P, sch)
    rest = full - part
    assert np.ptp(rest) < 1e-9 * np.abs(rest).max()
    # and the torsion term is lambda dependent there
    Ut = torsions(s, 1.0, forces=False)[0]
    assert Ut > 0
