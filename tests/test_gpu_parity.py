"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated for FP32 pair arithmetic):
  forces: relative RMS error <= 1e-5 over all atoms of a replica;
  per-state total energy: relative error <= 1e-6 of |E_total| (where the total
    is a near-cancellation of large terms, relative to the sum of the
    components' magnitudes, stated per test);
  u_kn: the lambda-dependent part U_k - U_indep within 1e-3 kJ/mol per entry;
  dU/dlambda: relative error <= 1e-5 (absolute 1e-4 kJ/mol floor).
The oracle is evaluated at the positions the engine reports (the engine stores
FP32 coordinates and wraps them into the box at list builds).
"""
import os
import tempfile

import numpy as np
import pytest

import abfe_synth as S
import oracle as O
from paper_2603_22274_gb300 import ENERGY_NAMES

E_TOTAL = ENERGY_NAMES.index("total")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    return G


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


E_TORS = ENERGY_NAMES.index("torsion")


def oracle_state(s, P, lam, X):
    """FP64 oracle of one replica at positions X: forces, energy parts (the
    first eight components, then the rotatable-bond torsions), dU/dlambda."""
    lr, lq, lv = lam
    o = O.nonbonded(s, P, lq, lv, pos=X)
    ub, fb = O.bonds(s, pos=X)
    ut, ft, dt = O.torsion_state(s, P, lv, pos=X)
    F = o["F"] + fb + ft
    UB = 0.0
    if s.boresch is not None:
        UB, FB, _ = O.boresch(s, lr, pos=X)
        F = F + FB
    E = np.r_[o["E"], ub, lr * UB, ut]
    return F, E, np.array([UB, o["dudl_q"], o["dudl_v"] + dt])


def check_replicas(eng, w, ftol=1e-5, etol=1e-6, etol_mode="total", dtol=1e-5, dabs=1e-4):
    F, E, D = eng.compute()
    X = eng.positions()
    worst = {}
    for r in range(eng.R):
        s = w.systems[w.system_of_replica[r]]
        sch = w.schedules[w.schedule_of_replica[r]]
        lam = sch.state(int(w.state_of_replica[r]))
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Fr, Er, Dr = oracle_state(s, w.params, lam, X[a:b])
        fr = rel_rms(F[a:b], Fr)
        assert fr <= ftol, (r, fr)
        scale = abs(Er.sum()) if etol_mode == "total" else np.abs(Er).sum()
        de = abs(E[r, E_TOTAL] - Er.sum())
        assert de <= etol * scale + 1e-6, (r, E[r], Er, de, scale)
        assert np.all(np.abs(E[r, :8] - Er[:8]) <= etol * scale + 1e-6), (r, E[r, :8] - Er[:8])
        assert abs(E[r, E_TORS] - Er[8]) <= 1e-9 * abs(Er[8]) + 1e-9, (r, E[r, E_TORS], Er[8])
        assert np.all(np.abs(D[r] - Dr) <= dtol * np.abs(Dr) + dabs), (r, D[r], Dr)
        worst[r] = (fr, de / max(scale, 1e-300))
    return worst


def check_ukn(eng, w, tol=1e-3):
    U, dU, Dd = eng.eval_ukn()
    X = eng.positions()
    for r in range(eng.R):
        s = w.systems[w.system_of_replica[r]]
        sch = w.schedules[w.schedule_of_replica[r]]
        a, b = eng.offsets[r], eng.offsets[r + 1]
        ref = O.ukn_lambda_part(s, w.params, sch, pos=X[a:b])
        if w.params.get("ligand_mode", 0) == 1:
            # decoupling: the ligand's own pairs are lambda independent and
            # belong to U_indep, not to the lambda-dependent part
            e = O.nonbonded(s, w.params, 1.0, 1.0, forces=False, pos=X[a:b])["energy"]
            ref = ref - e["liglig_lj"] - e["liglig_c"]
        err = np.abs(dU[r, :sch.K] - ref).max()
        assert err <= tol, (r, err)
        if r > 1:
            continue
        # full reduced potential: E_indep + dU over kT
        full = O.ukn(s, w.params, sch, pos=X[a:b])
        assert np.abs(U[r, :sch.K] - full).max() <= 1e-6 * np.abs(full).max() + tol / w.params["kT"]
    return U, dU


# ----------------------------------------------------------------------- tiny system

def test_tiny_fp64_all_states(G):
    w = S.workload_tiny()
    eng = G.engine_for_workload(w, precision=1)
    check_replicas(eng, w, ftol=1e-5, etol=1e-6)
    check_ukn(eng, w)
    eng.close()


def test_tiny_fp32_forces_and_energies(G):
    """The tiny case is an FP64 configuration; run in FP32 as a stress test its
    0.15 nm solute-water contacts make dU/dlambda_q a sum of +-230 kJ/mol pair
    terms cancelling to ~0.4, so its absolute floor is 1e-3 kJ/mol."""
    w = S.workload_tiny()
    eng = G.engine_for_workload(w, precision=0)
    check_replicas(eng, w, ftol=1e-5, etol=1e-6, etol_mode="components", dabs=1e-3)
    eng.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_ligand_modes(G, mode):
    w = S.workload_tiny()
    w.params = dict(w.params, ligand_mode=mode)
    eng = G.engine_for_workload(w, precision=1)
    check_replicas(eng, w)
    check_ukn(eng, w)
    eng.close()


def test_tiny_pair_set_matches_brute_force(G):
    """Every in-cutoff pair found through the cluster list, per atom; pairs whose
    distance lies within 1e-5 nm of the cutoff may go either way in FP32."""
    w = S.workload_tiny()
    eng = G.engine_for_workload(w, precision=0)
    c, per_atom = eng.count_pairs(per_atom=True)
    X = eng.positions()
    s = w.systems[0]
    rc = w.params["cutoff"]
    for r in (0, 7):
        a, b = eng.offsets[r], eng.offsets[r + 1]
        ref = O.neighbor_counts(s, rc, pos=X[a:b])
        lo = O.neighbor_counts(s, rc - 1e-5, pos=X[a:b])
        hi = O.neighbor_counts(s, rc + 1e-5, pos=X[a:b])
        got = per_atom[a:b]
        assert np.all((got >= lo) & (got <= hi))
        exact = lo == hi
        assert np.array_equal(got[exact], ref[exact])
        total = int(c[r].sum())
        assert int(lo.sum()) // 2 <= total <= int(hi.sum()) // 2


# ----------------------------------------------------------------------- mid-size complex

@pytest.fixture(scope="module")
def mid():
    c = S.complex_leg(77, n_atoms=6000, core_diameter=2.0, n_lig=30)
    sch = S.schedule_k42()
    st = np.array([0, 5, 9, 20, 31, 41], np.int32)
    return S.Workload("mid-6000", [c], np.zeros(len(st), np.int32), [sch],
                      np.zeros(len(st), np.int32), st, S.params_for(1.0, 3.12))


@pytest.mark.parametrize("group", [1, 2, 4])
def test_mid_fp32_parity(G, mid, group):
    eng = G.engine_for_workload(mid)
    eng.set_tuning(group=group, max_entries=32)
    # this small system's total is a near-cancellation: energy tolerance is
    # relative to the sum of the components' magnitudes
    check_replicas(eng, mid, etol_mode="components")
    check_ukn(eng, mid)
    eng.close()


def test_mid_fp64_parity(G, mid):
    eng = G.engine_for_workload(mid, precision=1)
    check_replicas(eng, mid, ftol=1e-6, etol=1e-9, etol_mode="components", dtol=1e-9)
    check_ukn(eng, mid, tol=1e-6)
    eng.close()


def test_batch_of_uneven_systems_matches_single(G):
    """Replicas of different systems in one context give bit-identical results
    to the same replica alone."""
    a = S.complex_leg(5, n_atoms=4500, core_diameter=1.6, n_lig=24)
    b = S.solvent_leg(6, n_lig=40, box=3.0, n_atoms=2800)
    sch = S.schedule_k42()
    sol = S.schedule_solvent_k30()
    P = S.params_for(1.0, 3.12)
    wb = S.Workload("ab", [a, b], np.array([0, 1, 0, 1], np.int32), [sch, sol],
                    np.array([0, 1, 0, 1], np.int32), np.array([3, 4, 25, 17], np.int32), P)
    eb = G.engine_for_workload(wb)
    Fb, Eb, Db = eb.compute()
    check_replicas(eb, wb, etol_mode="components")
    for r in range(4):
        wa = S.Workload("one", [wb.systems[wb.system_of_replica[r]]], np.zeros(1, np.int32),
                        [wb.schedules[wb.schedule_of_replica[r]]], np.zeros(1, np.int32),
                        np.array([wb.state_of_replica[r]], np.int32), P)
        e1 = G.engine_for_workload(wa)
        F1, E1, D1 = e1.compute()
        assert np.array_equal(F1, Fb[eb.offsets[r]:eb.offsets[r + 1]])
        assert np.array_equal(D1[0], Db[r])
        e1.close()
    eb.close()


def test_inner_list_between_prunes(G, mid):
    """Forces and the per-atom pair set through the pruned inner list at steps
    between prunes and between outer rebuilds: every in-cutoff pair must still
    be in the list (the prune and rebuild rules are exact)."""
    eng = G.engine_for_workload(mid)
    eng.set_tuning(skin=0.2, prune_skin=0.03)
    s = mid.systems[0]
    rc = mid.params["cutoff"]
    seen_prunes = set()
    for k in range(4):
        eng.step(7, dt=0.001, gamma=1.0, seed=40 + k)
        st = eng.stats()
        seen_prunes.add(st["n_prunes"])
        c, per_atom = eng.count_pairs(per_atom=True)
        X = eng.positions()
        for r in (0, 3):
            a, b = eng.offsets[r], eng.offsets[r + 1]
            lo = O.neighbor_counts(s, rc - 1e-5, pos=X[a:b])
            hi = O.neighbor_counts(s, rc + 1e-5, pos=X[a:b])
            got = per_atom[a:b]
            assert np.all((got >= lo) & (got <= hi)), k
        check_replicas(eng, mid, etol_mode="components", dabs=1e-3)
    st = eng.stats()
    assert st["n_prunes"] > st["n_rebuilds"] >= 1
    assert len(seen_prunes) > 1
    eng.close()


def test_determinism_and_graph_path(G, mid):
    eng = G.engine_for_workload(mid)
    F1, E1, D1 = eng.compute()
    F2, E2, D2 = eng.compute()
    assert np.array_equal(F1, F2) and np.array_equal(E1, E2) and np.array_equal(D1, D2)
    eng.step(30, dt=0.0005, gamma=5.0, seed=11)
    xa, va = eng.positions(), eng.velocities()
    eng.close()
    # same start, graph-captured loop: identical trajectory
    eng2 = G.engine_for_workload(mid)
    eng2.set_tuning(graph_steps=10)
    eng2.step(30, dt=0.0005, gamma=5.0, seed=11)
    assert np.array_equal(eng2.positions(), xa)
    assert np.array_equal(eng2.velocities(), va)
    eng2.close()


def test_bonds_across_the_periodic_wrap_fp32(G):
    """Waters whose atoms sit on both sides of the box edge in the stored
    (wrapped) positions: a bond vector formed as a box-sized difference and
    then shifted would carry a rounding of ulp(L) ~ 5e-7 nm, which the stiff
    O-H bonds (3e5 kJ/mol/nm^2) turn into up to ~0.07 kJ/mol/nm. The FP32
    forces on those atoms match the oracle within 0.02 kJ/mol/nm (the FP32
    pair arithmetic leaves a few 1e-3) and 1e-5 relative RMS."""
    s = S.water_box(31, 5.0)
    X = np.array(s.pos, dtype=np.float64)
    L = np.asarray(s.box, dtype=np.float64)
    # move the box contents by half a box and wrap: molecules straddle every face
    X = np.mod(X + 0.5 * L, L).astype(np.float32).astype(np.float64)
    b = np.asarray(s.bonds).reshape(-1, 2)
    d = X[b[:, 1]] - X[b[:, 0]]
    split = np.unique(b[(np.abs(d) > 0.5 * L).any(1)])
    assert len(split) >= 20
    s.pos = X
    sch = S.schedule_k12()
    w = S.Workload("wrap", [s], np.zeros(1, np.int32), [sch], np.zeros(1, np.int32),
                   np.zeros(1, np.int32), S.params_for(0.9, 3.47))
    eng = G.engine_for_workload(w)
    F, _, _ = eng.compute()
    Xg = eng.positions()
    Fr, _, _ = oracle_state(s, w.params, sch.state(0), Xg)
    err = np.linalg.norm(F[split] - Fr[split], axis=1)
    assert err.max() < 0.02, (err.max(), split[np.argmax(err)])
    assert rel_rms(F[split], Fr[split]) < 1e-5
    eng.close()


def test_checkpoint_resume_bit_identical(G, mid):
    eng = G.engine_for_workload(mid)
    eng.step(20, dt=0.0005, gamma=5.0, seed=4)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ckpt.bin")
        eng.save_checkpoint(path)
        eng.step(25, dt=0.0005, gamma=5.0, seed=5)
        xa, va = eng.positions(), eng.velocities()
        eng.close()
        eng2 = G.engine_for_workload(mid)
        eng2.load_checkpoint(path)
        eng2.step(25, dt=0.0005, gamma=5.0, seed=5)
        assert np.array_equal(eng2.positions(), xa)
        assert np.array_equal(eng2.velocities(), va)
        eng2.close()


# ----------------------------------------------------------------------- integrator

def test_baoab_one_step_matches_oracle(G):
    w = S.water_box(21, 2.2)
    sch = S.schedule_k12()
    W = S.Workload("water", [w], np.zeros(1, np.int32), [sch], np.zeros(1, np.int32),
                   np.zeros(1, np.int32), S.params_for(0.9, 3.47))
    eng = G.engine_for_workload(W)
    x0, v0 = eng.positions(), eng.velocities()
    dt, gamma, seed = 0.001, 1.0, 12345
    eng.step(1, dt=dt, gamma=gamma, seed=seed)
    x1, v1 = eng.positions(), eng.velocities()
    xo, vo, _ = O.baoab_step(w, W.params, sch.state(0), x0, v0, dt, gamma, seed, step=0, replica=0)
    d = x1 - xo
    d -= w.box * np.round(d / w.box)
    assert np.abs(d).max() <= 2e-6
    assert rel_rms(v1, vo) <= 1e-5
    eng.close()


def test_langevin_temperature(G):
    """A long run with the thermostat keeps the kinetic temperature near T."""
    w = S.water_box(22, 2.5)
    sch = S.schedule_k12()
    W = S.Workload("water", [w], np.zeros(1, np.int32), [sch], np.zeros(1, np.int32),
                   np.zeros(1, np.int32), S.params_for(0.9, 3.47))
    eng = G.engine_for_workload(W)
    eng.step(2000, dt=0.001, gamma=5.0, seed=3)
    temps = []
    for _ in range(10):
        eng.step(100, dt=0.001, gamma=5.0, seed=3)
        v = eng.velocities()
        temps.append((w.mass[:, None] * v * v).sum() / (3 * w.n * S.BOLTZMANN_KJ))
    assert abs(np.mean(temps) - 300.0) < 15.0, temps
    eng.close()


# ----------------------------------------------------------------------- error paths

def test_error_statuses(G):
    import paper_2603_22274_gb300 as GG
    w = S.workload_tiny()
    s = w.systems[0]
    with pytest.raises(GG.AbfeError) as e:
        GG.Engine([s], [0], dict(w.params, cutoff=1.0))
    assert e.value.status == 2
    bad = s.copy()
    bad.pos = bad.pos.copy()
    bad.pos[3, 1] = np.nan
    with pytest.raises(GG.AbfeError) as e:
        GG.Engine([bad], [0], w.params)
    assert e.value.status == 4
    bad = s.copy()
    bad.excl = np.array([[0, 99999]], np.int32)
    with pytest.raises(GG.AbfeError) as e:
        GG.Engine([bad], [0], w.params)
    assert e.value.status == 1
    eng = GG.Engine([s], [0], w.params)
    with pytest.raises(GG.AbfeError) as e:
        eng.compute()
    assert e.value.status == 8
    eng.set_schedule(0, [0.0], [1.0], [1.0])
    eng.set_states([0], [0])
    x = eng.positions()
    x[5, 0] = np.inf
    with pytest.raises(GG.AbfeError) as e:
        eng.set_positions(x)
    assert e.value.status == 4
    F, E, D = eng.compute()   # context still usable
    assert np.isfinite(F).all()
    eng.close()


# ----------------------------------------------------------------------- full-size complex leg

@pytest.fixture(scope="module")
def big():
    return S.workload_complex60k(n_replicas=4)


def test_complex60k_sampled_parity(G, big):
    """The 60,000-atom complex window at four states: forces on sampled atoms,
    total energy (all pairs), dU/dlambda and every u_kn entry's lambda part."""
    w = big
    w.state_of_replica = np.array([0, 10, 25, 41], np.int32)
    eng = G.engine_for_workload(w)
    F, E, D = eng.compute()
    X = eng.positions()
    s = w.systems[0]
    sch = w.schedules[0]
    rng = np.random.default_rng(0)
    lig = np.where(s.is_ligand)[0]
    rows = np.unique(np.r_[rng.choice(s.n, 192, replace=False), lig[:16], s.boresch.anchors])
    for r in range(eng.R):
        lam = sch.state(int(w.state_of_replica[r]))
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Xr = X[a:b]
        Fo = O.force_rows(s, w.params, lam[1], lam[2], rows, pos=Xr)
        Fo += O.bonds(s, pos=Xr)[1][rows]
        Fo += O.boresch(s, lam[0], pos=Xr)[1][rows]
        Fo += O.torsion_state(s, w.params, lam[2], pos=Xr)[1][rows]
        assert rel_rms(F[a:b][rows], Fo) <= 1e-5
        if r in (0, 3):
            _, Er, Dr = oracle_state(s, w.params, lam, Xr)
            assert abs(E[r, E_TOTAL] - Er.sum()) <= 1e-6 * abs(Er.sum())
            assert np.all(np.abs(D[r] - Dr) <= 1e-5 * np.abs(Dr) + 1e-4)
    U, dU, _ = eng.eval_ukn()
    for r in (0, 2):
        a, b = eng.offsets[r], eng.offsets[r + 1]
        ref = O.ukn_lambda_part(s, w.params, sch, pos=X[a:b])
        assert np.abs(dU[r, :sch.K] - ref).max() <= 1e-3
    eng.close()


def test_large_context_sampled_parity(G):
    """32 windows of a 41,000-atom complex leg in one context (1.4 M atom
    slots, past the size at which round-one's Coulomb force table could be
    zeroed by a late fill): forces on sampled atoms, total energy, dU/dlambda
    and every u_kn entry's lambda part of the first and last window against
    the oracle."""
    wb = S.workload_batch(n_ligands=1, complex_range=(40000, 42000))
    cpx = wb.systems[0]
    sch = S.schedule_k42()
    R = 32
    st = (np.arange(R, dtype=np.int32) * 5) % sch.K
    w = S.Workload("c32", [cpx], np.zeros(R, np.int32), [sch], np.zeros(R, np.int32), st,
                   wb.params)
    eng = G.engine_for_workload(w)
    assert eng.stats()["slots"] > 1_200_000
    F, E, D = eng.compute()
    U, dU, _ = eng.eval_ukn()
    X = eng.positions()
    rng = np.random.default_rng(3)
    lig = np.where(cpx.is_ligand)[0]
    rows = np.unique(np.r_[rng.choice(cpx.n, 160, replace=False), lig[:12]])
    for r in (0, R - 1):
        lam = sch.state(int(st[r]))
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Xr = X[a:b]
        Fo = (O.force_rows(cpx, w.params, lam[1], lam[2], rows, pos=Xr)
              + O.bonds(cpx, pos=Xr)[1][rows] + O.boresch(cpx, lam[0], pos=Xr)[1][rows]
              + O.torsion_state(cpx, w.params, lam[2], pos=Xr)[1][rows])
        assert rel_rms(F[a:b][rows], Fo) <= 1e-5, (r, rel_rms(F[a:b][rows], Fo))
        _, Er, Dr = oracle_state(cpx, w.params, lam, Xr)
        # the synthetic start's total cancels components of larger magnitude:
        # energy tolerance relative to the sum of the components' magnitudes
        assert abs(E[r, E_TOTAL] - Er.sum()) <= 1e-6 * np.abs(Er).sum()
        assert np.all(np.abs(D[r] - Dr) <= 1e-5 * np.abs(Dr) + 1e-3)
        ref = O.ukn_lambda_part(cpx, w.params, sch, pos=Xr)
        assert np.abs(dU[r, :sch.K] - ref).max() <= 1e-3
    eng.close()


def test_alchemical_waters_parity(G):
    """A ligand with net charge +1 in its solvent leg (a counterion keeps the
    physical state neutral) with two alchemical waters taking up the lost
    charge: forces, energies, dU/dlambda and every u_kn entry against the
    oracle along the charge and vdW stages, FP32 and FP64, before and after
    MD; after device exchanges (which move lambda_q and so the waters'
    charges) the results equal those of a context given the exchanged states."""
    s = S.charged_leg(S.solvent_leg(6, n_lig=40, box=3.0, n_atoms=2800), +1.0)
    assert len(s.alch_water) == 2
    sch = S.schedule_solvent_k30()
    st = np.array([0, 3, 6, 9, 15, 29], np.int32)
    P = S.params_for(1.0, 3.12)
    w = S.Workload("aw", [s], np.zeros(len(st), np.int32), [sch], np.zeros(len(st), np.int32), st, P)
    e64 = G.engine_for_workload(w, precision=1)
    check_replicas(e64, w, ftol=1e-6, etol=1e-9, etol_mode="components", dtol=1e-9, dabs=1e-7)
    check_ukn(e64, w, tol=1e-6)
    e64.close()
    eng = G.engine_for_workload(w)
    check_replicas(eng, w, etol_mode="components", dabs=1e-3)
    check_ukn(eng, w)
    eng.step(15, dt=0.0005, gamma=5.0, seed=9)
    check_replicas(eng, w, etol_mode="components", dabs=1e-3)
    check_ukn(eng, w)
    eng.close()
    # device exchanges between neighbouring charge-stage states change lambda_q:
    # the waters' charges follow
    st = np.arange(2, 8, dtype=np.int32)
    w = S.Workload("aw", [s], np.zeros(len(st), np.int32), [sch], np.zeros(len(st), np.int32), st, P)
    eng = G.engine_for_workload(w)
    eng.step(10, dt=0.0005, gamma=5.0, seed=9)
    for t in range(8):
        eng.replica_exchange(seed=21)
        if not np.array_equal(eng.replica_states(), st):
            break
    new = eng.replica_states()
    assert not np.array_equal(new, st)
    X = eng.positions()
    eng.build_list()
    F1, E1, D1 = eng.compute()
    w2 = S.Workload("aw2", [s], w.system_of_replica, [sch], w.schedule_of_replica, new, P)
    eng2 = G.engine_for_workload(w2)
    eng2.set_positions(X)
    F2, E2, D2 = eng2.compute()
    assert np.array_equal(F1, F2) and np.array_equal(E1, E2) and np.array_equal(D1, D2)
    check_replicas(eng2, w2, etol_mode="components", dabs=1e-3)
    eng.close()
    eng2.close()


def test_alchemical_waters_with_pme_not_implemented(G):
    s = S.charged_leg(S.solvent_leg(6, n_lig=40, box=3.0, n_atoms=2800), +1.0)
    P = dict(S.params_for(1.0, 3.12), pme_order=4, pme_spacing=0.12)
    with pytest.raises(G.AbfeError) as e:
        G.Engine([s], [0], P)
    assert e.value.status == 7
