"""The seeded input generators (abfe_synth) keep the properties that long MD runs
of the synthetic systems rely on: no water H can fall into a deep well next to
a small, strongly charged atom, and no periodic torsion spans a bond angle that
can straighten to 180 degrees (where a dihedral's gradient diverges)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import abfe_synth as S  # noqa: E402


def _angles_deg(xyz):
    b1 = xyz[:-2] - xyz[1:-1]
    b2 = xyz[2:] - xyz[1:-1]
    c = (b1 * b2).sum(1) / (np.linalg.norm(b1, axis=1) * np.linalg.norm(b2, axis=1))
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def _h_well(q, sig, eps):
    """Deepest pair energy of a water H (q 0.417 e, sigma 0.1 nm, eps 0.1 kJ/mol)
    with an atom, Lorentz-Berthelot mixing, over 0.05..0.4 nm."""
    r = np.linspace(0.05, 0.4, 3501)
    sm = 0.5 * (sig + S.H_LJ_MD[0])
    em = np.sqrt(eps * S.H_LJ_MD[1])
    u = 4 * em * ((sm / r) ** 12 - (sm / r) ** 6) + S.COULOMB_K * S.WATER_Q_H * q / r
    return u.min()


def test_core_types_within_the_ligand_ranges():
    c = S.complex_leg(9, n_atoms=9000, core_diameter=2.2, n_lig=20)
    core = ~c.is_ligand.astype(bool)
    core[c.info["n_core"]:] = False
    assert core.sum() == c.info["n_core"]
    assert c.sigma[core].min() >= 0.25 - 1e-6 and c.sigma[core].max() <= 0.39 + 1e-6
    assert np.abs(c.charge[core]).max() <= 0.82
    # no core atom gives a water H a well much deeper than a water O does
    o_well = _h_well(S.WATER_Q_O, S.WATER_SIG_O, S.WATER_EPS_O)
    worst = min(_h_well(q, s, e) for q, s, e in
                zip(c.charge[core], c.sigma[core], c.epsilon[core]))
    assert worst > 1.25 * o_well, (worst, o_well)


def test_torsions_only_across_bent_angles_held_by_13_bonds():
    for s in (S.complex_leg(9, n_atoms=9000, core_diameter=2.2, n_lig=30),
              S.solvent_leg(6, n_lig=40, box=3.0, n_atoms=2800)):
        lig = np.where(s.is_ligand)[0]
        # the chain made whole (stored positions are wrapped into the box)
        x = s.pos[lig].copy()
        for a in range(1, len(x)):
            d = x[a] - x[a - 1]
            x[a] = x[a - 1] + d - s.box * np.round(d / s.box)
        ang = _angles_deg(x)                      # angle at chain atom a = 1 .. n-2
        assert len(s.torsions) > 0
        for q in np.asarray(s.torsions) - lig[0]:
            # a torsion (a, b, c, d) spans the angles at b and c
            assert ang[q[1] - 1] <= 135.0 + 1e-9 and ang[q[2] - 1] <= 135.0 + 1e-9
        # every 1-3 pair of the chain is a harmonic bond at its starting length
        bonds = {tuple(sorted(b)): k for k, b in enumerate(np.asarray(s.bonds))}
        for a in range(len(lig) - 2):
            key = (lig[a], lig[a + 2])
            assert key in bonds
            k = bonds[key]
            assert abs(s.bond_r0[k] - np.linalg.norm(x[a + 2] - x[a])) < 1e-6
            assert s.bond_k[k] == S.K_LIGAND_13
        # and stays excluded
        ex = {tuple(sorted(e)) for e in np.asarray(s.excl)}
        assert all((lig[a], lig[a + 2]) in ex for a in range(len(lig) - 2))
