"""Reciprocal-space Ewald (smooth PME) on the device against the FP64 oracle's
SPME on the same grid and B-spline order, with the self energy and the
excluded-pair correction: forces, total energies, dU/dlambda_q and u_kn, and
determinism. The oracle's SPME is itself pinned to the Ewald k-space sum and
the rock-salt Madelung constant (tests/test_oracle_pme.py)."""
import numpy as np
import pytest

import abfe_synth as S
import oracle as O
from oracle.pme import exclusion_correction, scaled_charges, self_energy, spme
from paper_2603_22274_gb300 import ENERGY_NAMES

pytestmark = pytest.mark.gpu

E_TOTAL = ENERGY_NAMES.index("total")
E_RECIP = ENERGY_NAMES.index("recip")


def grid_for(box, spacing, order):
    """Smallest 2^a 3^b 5^c >= max(2 order, L / spacing) per edge (the library's rule)."""
    def smooth(k):
        for f in (2, 3, 5):
            while k % f == 0:
                k //= f
        return k == 1
    out = []
    for L in box:
        k = max(2 * order, int(np.ceil(L / spacing - 1e-9)))
        while not smooth(k):
            k += 1
        out.append(k)
    return tuple(out)


def recip_terms(s, P, lam_q, pos, parts=False):
    q = scaled_charges(s, lam_q)
    grid = grid_for(s.box, P["pme_spacing"], P["pme_order"])
    Er, Fr = spme(pos, q, s.box, P["ewald_beta"], grid, P["pme_order"], P["coulomb_k"])
    Es = self_energy(q, P["ewald_beta"], P["coulomb_k"])
    Ex, Fx = exclusion_correction(pos, q, s.box, s.excl, P["ewald_beta"], P["coulomb_k"])
    if parts:
        return Er + Es + Ex, Fr + Fx, abs(Er) + abs(Es) + abs(Ex)
    return Er + Es + Ex, Fr + Fx


def state_ref(s, P, lam, pos):
    """Total energy, forces, the reciprocal-side energy, and the magnitude scale
    of the summed terms (the total of a small system cancels large parts)."""
    lr, lq, lv = lam
    o = O.nonbonded(s, P, lq, lv, pos=pos)
    ub, fb = O.bonds(s, pos=pos)
    ut, ft, _ = O.torsion_state(s, P, lv, pos=pos)
    E = o["E"].sum() + ub + ut
    F = o["F"] + fb + ft
    scale = np.abs(o["E"]).sum() + abs(ub) + abs(ut)
    if s.boresch is not None:
        UB, FB, _ = O.boresch(s, lr, pos=pos)
        E += lr * UB
        F = F + FB
    Er, Fr, sr = recip_terms(s, P, lq, pos, parts=True)
    return E + Er, F + Fr, Er, scale + sr


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    O.build()
    return G


def _tiny(order=4, spacing=0.1):
    s = S.tiny(S.BASE_SEED + 1)
    sch = S.schedule_k12()
    P = dict(S.params_for(0.9, 3.47, skin=0.0), pme_order=order, pme_spacing=spacing)
    states = np.array([0, 2, 4, 8], np.int32)       # lambda_q = 1, 0.5, 0 and a vdW state
    return S.Workload("tiny-pme", [s], np.zeros(len(states), np.int32), [sch],
                      np.zeros(len(states), np.int32), states, P)


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


@pytest.mark.parametrize("order", [4, 6])
def test_pme_forces_energies_match_oracle(G, order):
    w = _tiny(order)
    s, sch = w.systems[0], w.schedules[0]
    eng = G.engine_for_workload(w)
    F, E, D = eng.compute()
    X = eng.positions()
    for r in range(w.n_replicas):
        lam = sch.state(int(w.state_of_replica[r]))
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Eo, Fo, Er, sc = state_ref(s, w.params, lam, X[a:b])
        assert rel_rms(F[a:b], Fo) <= 1e-5, (r, rel_rms(F[a:b], Fo))
        assert abs(E[r, E_TOTAL] - Eo) <= 1e-6 * sc, (r, E[r, E_TOTAL], Eo, sc)
        assert abs(E[r, E_RECIP] - Er) <= 1e-6 * sc, (r, E[r, E_RECIP], Er, sc)
    eng.close()


def test_pme_dudl_and_ukn(G):
    """FP64 pair path on the tiny system (its 0.15 nm contacts put FP32 u_kn
    rows at the 1e-2 kJ/mol level with or without PME), so that what is checked
    at 1e-3 kJ/mol is the reciprocal part of u_kn and dU/dlambda_q."""
    w = _tiny()
    s, sch, P = w.systems[0], w.schedules[0], w.params
    eng = G.engine_for_workload(w, precision=1)
    U, dU, Dd = eng.eval_ukn()
    X = eng.positions()
    for r in range(w.n_replicas):
        a, b = eng.offsets[r], eng.offsets[r + 1]
        pos = X[a:b]
        refs = [state_ref(s, P, sch.state(k), pos) for k in range(sch.K)]
        ref = np.array([x[0] for x in refs])
        sc = max(x[3] for x in refs)
        du = dU[r, :sch.K]
        # u_kn's lambda part: differences between states are what MBAR uses
        got = du - du[0]
        exp_ = ref - ref[0]
        assert np.abs(got - exp_).max() <= 1e-3, np.abs(got - exp_).max()
        assert np.abs(U[r, :sch.K] * P["kT"] - ref).max() <= 1e-6 * sc
        # dU/dlambda_q: the oracle's nonbonded part plus the reciprocal polynomial's slope
        lam = sch.state(int(w.state_of_replica[r]))
        o = O.nonbonded(s, P, lam[1], lam[2], forces=False, pos=pos)
        # the reciprocal-side energy is exactly quadratic in lambda_q: its slope
        # from the values at 0, 1/2 and 1
        e0, e5, e1 = (recip_terms(s, P, x, pos)[0] for x in (0.0, 0.5, 1.0))
        cq = 2.0 * (e1 - 2.0 * e5 + e0)
        slope = (e1 - e0 - cq) + 2.0 * cq * lam[1]
        dq = o["dudl_q"] + slope
        assert abs(Dd[r, 1] - dq) <= 1e-5 * abs(dq) + 1e-3, (r, Dd[r, 1], dq)
    eng.close()


def test_pme_deterministic_and_md_finite(G):
    w = _tiny()
    eng = G.engine_for_workload(w)
    F1, E1, _ = eng.compute()
    F2, E2, _ = eng.compute()
    assert np.array_equal(F1, F2) and np.array_equal(E1, E2)
    eng.step(20, dt=0.0005, gamma=5.0, seed=3)
    F3, E3, _ = eng.compute()
    assert np.isfinite(F3).all() and np.isfinite(E3).all()
    eng.close()


def test_pme_mid_system_sampled(G):
    """6,000-atom system (3.9 nm box, 40^3-class grid): forces on every atom and
    total energy at two states."""
    s = S.complex_leg(S.BASE_SEED + 7, n_atoms=6000, core_diameter=1.8, n_lig=24)
    sch = S.schedule_k42()
    P = dict(S.params_for(1.0, 3.12, skin=0.1), pme_order=4, pme_spacing=0.1)
    states = np.array([8, 14], np.int32)
    w = S.Workload("mid-pme", [s], np.zeros(2, np.int32), [sch], np.zeros(2, np.int32), states, P)
    eng = G.engine_for_workload(w)
    F, E, D = eng.compute()
    U, dU, Dd = eng.eval_ukn()
    X = eng.positions()
    ks = [0, 8, 10, 14, 20, 30, 41]
    for r in range(2):
        lam = sch.state(int(states[r]))
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Eo, Fo, Er, sc = state_ref(s, P, lam, X[a:b])
        assert rel_rms(F[a:b], Fo) <= 1e-5
        assert abs(E[r, E_TOTAL] - Eo) <= 1e-6 * sc
        # u_kn differences between states (FP32 pair path at a realistic density)
        ref = np.array([state_ref(s, P, sch.state(k), X[a:b])[0] for k in ks])
        got = dU[r, ks]
        assert np.abs((got - got[0]) - (ref - ref[0])).max() <= 1e-3
    eng.close()


def test_pme_rejects_decouple_mode(G):
    w = _tiny()
    w.params["ligand_mode"] = 1
    with pytest.raises(G.AbfeError):
        G.engine_for_workload(w)


def _nve_drift(G, pme):
    s = S.complex_leg(S.BASE_SEED + 7, n_atoms=6000, core_diameter=1.8, n_lig=24)
    sch = S.schedule_k42()
    P = dict(S.params_for(1.0, 3.12, skin=0.1))
    if pme:
        P.update(pme_order=4, pme_spacing=0.1)
    w = S.Workload("nve", [s], np.zeros(1, np.int32), [sch], np.zeros(1, np.int32),
                   np.array([14], np.int32), P)
    eng = G.engine_for_workload(w)
    eng.step(200, dt=0.0005, gamma=20.0, seed=1)       # relax the synthetic start
    m = np.asarray(s.mass, np.float64)

    def total():
        _, E, _ = eng.compute()
        v = eng.velocities()
        return E[0, E_TOTAL] + 0.5 * float((m[:, None] * v ** 2).sum())

    e0 = total()
    eng.step(400, dt=0.0005, gamma=0.0, seed=2)        # gamma = 0: velocity Verlet
    e1 = total()
    eng.close()
    return abs(e1 - e0), e0


def test_pme_conserves_energy_like_real_space(G):
    """Velocity Verlet with and without the reciprocal terms: the drift of the
    total energy over 400 steps of 0.5 fs stays at the real-space level (the
    SPME forces are the exact gradient of the SPME energy)."""
    d0, e0 = _nve_drift(G, False)
    d1, e1 = _nve_drift(G, True)
    print("NVE drift kJ/mol: real space", d0, "with PME", d1, "totals", e0, e1)
    n_dof = 3 * 6000
    kT = 0.00831446261815324 * 300.0
    assert d1 <= max(5.0 * d0, 1e-3 * n_dof * kT / 2), (d0, d1)


def test_pme_mixed_grids_in_one_batch(G):
    """Two systems with different grids in one context, their windows
    interleaved: 2.6 nm box (24^3 grid at 0.12 nm) and 3.1 nm box (27^3: odd
    edge, radix-3 stages only, a ragged second tile of 16 lines). The FFT tiles,
    the convolution's multi-chunk blocks (which here straddle two windows) and
    the FP64 lambda_q split all index across windows of different grids."""
    sa = S.solvent_leg(S.BASE_SEED + 31, n_lig=16, box=2.6)
    sb = S.solvent_leg(S.BASE_SEED + 32, n_lig=16, box=3.1)
    sch = S.schedule_solvent_k30()
    P = dict(S.params_for(1.0, 3.12, skin=0.1), pme_order=4, pme_spacing=0.12)
    assert grid_for(sa.box, 0.12, 4) == (24, 24, 24) and grid_for(sb.box, 0.12, 4) == (27, 27, 27)
    sys_of = np.array([0, 1, 0, 1], np.int32)
    states = np.array([0, 5, 14, 29], np.int32)
    w = S.Workload("mixed-pme", [sa, sb], sys_of, [sch], np.zeros(4, np.int32), states, P)
    eng = G.engine_for_workload(w)
    F, E, D = eng.compute()
    U, dU, Dd = eng.eval_ukn()
    X = eng.positions()
    ks = [0, 3, 5, 8, 14, 29]
    for r in range(w.n_replicas):
        s = w.systems[int(sys_of[r])]
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Eo, Fo, Er, sc = state_ref(s, P, sch.state(int(states[r])), X[a:b])
        assert rel_rms(F[a:b], Fo) <= 1e-5, (r, rel_rms(F[a:b], Fo))
        assert abs(E[r, E_TOTAL] - Eo) <= 1e-6 * sc, (r, E[r, E_TOTAL], Eo, sc)
        assert abs(E[r, E_RECIP] - Er) <= 1e-6 * sc, (r, E[r, E_RECIP], Er, sc)
        ref = np.array([state_ref(s, P, sch.state(k), X[a:b])[0] for k in ks])
        got = dU[r, ks]
        assert np.abs((got - got[0]) - (ref - ref[0])).max() <= 1e-3, (r, got - got[0], ref - ref[0])
    eng.close()


def test_pme_two_contexts_with_different_grids(G):
    """A context with larger grids keeps working after a context with smaller
    grids was created in the same process (kernel attributes are per process)."""
    s = S.complex_leg(S.BASE_SEED + 7, n_atoms=6000, core_diameter=1.8, n_lig=24)
    sch = S.schedule_k42()
    P = dict(S.params_for(1.0, 3.12, skin=0.1), pme_order=4, pme_spacing=0.1)
    big = G.engine_for_workload(S.Workload("mid-pme", [s], np.zeros(1, np.int32), [sch],
                                           np.zeros(1, np.int32), np.array([8], np.int32), P))
    F1, E1, _ = big.compute()
    small = G.engine_for_workload(_tiny())
    small.compute()
    F2, E2, _ = big.compute()
    assert np.array_equal(F1, F2) and np.array_equal(E1, E2)
    small.close()
    big.close()
