"""Pins of the oracle's alchemical waters (oracle/alchemical_water.py) against
neutrality along the path, endpoint charges, the paper's per-water range,
finite differences in lambda_q, and the u_kn lambda part against whole-state
energies. None of these calls the CUDA path."""
import numpy as np
import pytest

import abfe_synth as S
import oracle as O
from oracle import alchemical_water as AW


@pytest.fixture(scope="module")
def leg():
    s = S.solvent_leg(6, n_lig=20, box=2.4, n_atoms=1400)
    return S.charged_leg(s, +1.0), S.params_for(1.0, 3.12)


def test_generator_choice_follows_the_paper_range():
    s = S.solvent_leg(6, n_lig=20, box=2.4, n_atoms=1400)
    for q, n in ((+1.0, 2), (-1.0, 3), (+2.0, 4), (-2.0, 5), (0.5, 1)):
        t = S.charged_leg(s, q)
        assert len(t.alch_water) == n == AW.count_for(q)
        assert np.all((t.alch_water_dq >= -0.4 - 1e-6) & (t.alch_water_dq <= 0.6 + 1e-6))
        assert abs(t.alch_water_dq.sum() - q) < 1e-5
        lig = t.is_ligand.astype(bool)
        assert abs(t.charge[lig].sum() - q) < 1e-4
        assert abs(t.charge.sum()) < 1e-4                 # neutral physical state
        assert not lig[t.alch_water].any()


@pytest.mark.parametrize("lam_q", [1.0, 0.7, 0.3, 0.0])
def test_box_stays_neutral(leg, lam_q):
    s, P = leg
    q = AW.charges_at(s, lam_q)
    lig = s.is_ligand.astype(bool)
    total = lam_q * q[lig].sum() + q[~lig].sum()
    assert abs(total) < 1e-4


def test_endpoint_charges(leg):
    s, P = leg
    np.testing.assert_array_equal(AW.charges_at(s, 1.0), s.charge)
    q0 = AW.charges_at(s, 0.0)
    np.testing.assert_allclose(q0[s.alch_water] - s.charge[s.alch_water], s.alch_water_dq)


@pytest.mark.parametrize("lq,lv", [(0.8, 1.0), (0.35, 1.0), (0.0, 0.6)])
def test_dudlq_by_differences(leg, lq, lv):
    """dU/dlambda_q with the alchemical waters' charges moving with lambda_q."""
    s, P = leg
    h = 1e-6
    U = lambda a: O.nonbonded(s, P, a, lv, forces=False)["E"].sum()
    r = O.nonbonded(s, P, lq, lv, forces=False)
    lo, hi = max(lq - h, 0.0), min(lq + h, 1.0)
    fd = (U(hi) - U(lo)) / (hi - lo)
    assert r["dudl_q"] == pytest.approx(fd, rel=1e-6, abs=1e-5)
    assert abs(AW.dudlq_waters(s, P, lq)) > 1e-3        # the waters' part matters here


def test_forces_with_waters_are_minus_gradient(leg):
    s, P = leg
    lq, lv = 0.4, 1.0
    F = O.nonbonded(s, P, lq, lv)["F"]
    h = 1e-6
    for i in list(s.alch_water[:1]) + [0, 5]:
        for k in range(3):
            xp, xm = s.pos.copy(), s.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(O.nonbonded(s, P, lq, lv, forces=False, pos=xp)["E"].sum()
                   - O.nonbonded(s, P, lq, lv, forces=False, pos=xm)["E"].sum()) / (2 * h)
            assert F[i, k] == pytest.approx(fd, rel=2e-5, abs=2e-3)


def test_ukn_lambda_part_with_waters(leg):
    s, P = leg
    sch = S.schedule_solvent_k30()
    full = O.ukn(s, P, sch) * P["kT"]
    part = O.ukn_lambda_part(s, P, sch)
    rest = full - part
    assert np.ptp(rest) < 1e-9 * np.abs(rest).max()
    # the waters' pair energy does depend on lambda_q
    assert abs(AW.water_pair_energy(s, P, 0.0) - AW.water_pair_energy(s, P, 1.0)) > 1e-3
