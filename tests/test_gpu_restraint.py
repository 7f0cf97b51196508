"""The library's restraint standard-state correction (abfe_boresch_correction,
host arithmetic behind the C ABI) against the oracle's adaptive quadrature of
the same integrals, to 1e-9 kJ/mol, and its argument checks."""
import numpy as np
import pytest

from oracle.restraint import boresch_correction as oracle_correction

pytestmark = pytest.mark.gpu

KT = 0.00831446261815324 * 300.0


@pytest.fixture(scope="module")
def G():
    import paper_2603_22274_gb300 as G
    G.lib()
    return G


@pytest.mark.parametrize("r0,th,kr,kt,kp", [
    (0.6, (1.45, 1.7), 4184.0, 41.84, 41.84),          # the workloads' constants
    (0.5, (0.9, 2.3), 836.8, 334.72, 334.72),          # the paper's constants in kJ/mol, nm, rad
    (0.25, (0.3, 2.9), 200.0, 5.0, 2.0),                # soft, angles near the poles
])
def test_boresch_correction_matches_oracle(G, r0, th, kr, kt, kp):
    got = G.boresch_correction(KT, r0, th, kr, kt, kp)
    ref = oracle_correction(KT, r0, th, kr, kt, kp)
    assert abs(got - ref) <= 1e-9, (got, ref)


def test_boresch_correction_rejects_bad_arguments(G):
    with pytest.raises(G.AbfeError):
        G.boresch_correction(KT, 0.6, (0.0, 1.0), 4184.0, 41.84, 41.84)
    with pytest.raises(G.AbfeError):
        G.boresch_correction(KT, -0.1, (1.0, 1.0), 4184.0, 41.84, 41.84)
