"""Pins of the FP64 oracle against facts fixed outside it: closed forms,
limits that reduce to textbook values, endpoint reductions, finite
differences, translation invariance, brute force and published test vectors.
None of these calls the CUDA path."""
import math

import numpy as np
import pytest

import abfe_synth as S
import oracle as O
from conftest import golden

KE = S.COULOMB_K


def _closed(name):
    for line in open(golden("closed_forms.txt")):
        if line.startswith(name + " "):
            return float(line.split()[1])
    raise KeyError(name)


def mk(pos, q, sig, eps, lig, box=5.0, excl=()):
    n = len(pos)
    return S.System("t", np.full(3, float(box)), np.asarray(pos, float), np.zeros((n, 3)),
                    np.ones(n), np.asarray(q, float), np.asarray(sig, float),
                    np.asarray(eps, float), np.asarray(lig, np.uint8),
                    np.asarray(excl, np.int32).reshape(-1, 2), np.zeros((0, 2), np.int32),
                    np.zeros(0), np.zeros(0))


def par(rc=1.2, beta=3.0, mode=0, alpha=0.5):
    return dict(cutoff=rc, ewald_beta=beta, sc_alpha=alpha, sc_p=1.0, coulomb_k=KE,
                kT=S.BOLTZMANN_KJ * 300, ligand_mode=mode)


# ---------------------------------------------------------------- random numbers

def test_philox_known_answers():
    for line in open(golden("philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_gauss3_moments():
    z = O.gauss3(200000, 42, 7, 3).ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    # fourth moment of a standard normal is 3
    assert abs((z ** 4).mean() - 3.0) < 0.05
    # different step -> independent stream
    z2 = O.gauss3(1000, 42, 8, 3).ravel()
    assert abs(np.corrcoef(z[:3000], z2)[0, 1]) < 0.1


# ---------------------------------------------------------------- softcore LJ

def test_softcore_at_r0_closed_form():
    eps = 0.7
    r = 1e-4  # r^6 = 1e-24 is negligible against alpha (1-lambda) sigma^6
    s = mk([[1, 1, 1], [1 + r, 1, 1]], [0, 0], [0.3, 0.3], [eps, eps], [1, 0])
    e = O.nonbonded(s, par(), 1.0, 0.5)["energy"]["ligenv_lj"]
    assert e == pytest.approx(_closed("softcore_r0_alpha0.5_lambda0.5_over_eps") * eps, rel=1e-9)


@pytest.mark.parametrize("lig", [[0, 0], [1, 0], [1, 1]])
def test_lj_minimum_and_mixing(lig):
    s1, s2, e1, e2 = 0.28, 0.36, 0.4, 0.9
    sig, eps = 0.5 * (s1 + s2), math.sqrt(e1 * e2)
    rmin = _closed("lj_rmin_over_sigma") * sig
    s = mk([[1, 1, 1], [1 + rmin, 1, 1]], [0, 0], [s1, s2], [e1, e2], lig)
    r = O.nonbonded(s, par(), 1.0, 1.0)
    assert r["E"].sum() == pytest.approx(_closed("lj_umin_over_eps") * eps, rel=1e-12)
    assert np.abs(r["F"]).max() < 1e-9


def test_softcore_lambda_zero_and_one():
    pos = [[1, 1, 1], [1.25, 1.1, 1.05]]
    s_l = mk(pos, [0.3, -0.4], [0.3, 0.34], [0.5, 0.6], [1, 0])
    s_e = mk(pos, [0.3, -0.4], [0.3, 0.34], [0.5, 0.6], [0, 0])
    assert O.nonbonded(s_l, par(), 0.0, 0.0)["E"].sum() == 0.0
    a = O.nonbonded(s_l, par(), 1.0, 1.0)
    b = O.nonbonded(s_e, par(), 1.0, 1.0)
    assert a["E"].sum() == pytest.approx(b["E"].sum(), rel=1e-13)
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-12)


# ---------------------------------------------------------------- Coulomb

@pytest.mark.parametrize("x,name", [(1.0, "erfc_1"), (2.0, "erfc_2")])
def test_real_space_coulomb_textbook_erfc(x, name):
    beta, r = 3.0, x / 3.0
    s = mk([[1, 1, 1], [1, 1 + r, 1]], [0.5, -0.8], [0, 0], [0, 0], [0, 0])
    e = O.nonbonded(s, par(beta=beta), 1.0, 1.0)["energy"]["env_c"]
    assert e == pytest.approx(KE * 0.5 * -0.8 * _closed(name) / r, rel=1e-12)


def test_beta_zero_limit_is_cut_coulomb():
    w = S.water_box(5, 1.9)
    P = par(rc=0.9, beta=1e-9)
    o = O.nonbonded(w, P, 1.0, 1.0, forces=False)
    p = O.pairs_brute(w, 0.9)
    d = w.pos[p[:, 1]] - w.pos[p[:, 0]]
    d -= w.box * np.round(d / w.box)
    r = np.linalg.norm(d, axis=1)
    cut = np.sum(KE * w.charge[p[:, 0]] * w.charge[p[:, 1]] / r)
    assert o["energy"]["env_c"] == pytest.approx(cut, rel=1e-8)


def test_charge_scaling_linear_and_quadratic():
    pos = [[1, 1, 1], [1.3, 1, 1], [1, 1.35, 1.1]]
    s = mk(pos, [0.5, -0.3, 0.2], [0, 0, 0], [0, 0, 0], [1, 1, 0])
    one = O.nonbonded(s, par(), 1.0, 1.0)["energy"]
    half = O.nonbonded(s, par(), 0.5, 1.0)["energy"]
    assert half["ligenv_c"] == pytest.approx(0.5 * one["ligenv_c"], rel=1e-13)
    assert half["liglig_c"] == pytest.approx(0.25 * one["liglig_c"], rel=1e-13)
    dec = O.nonbonded(s, par(mode=1), 0.5, 1.0)["energy"]
    assert dec["liglig_c"] == pytest.approx(one["liglig_c"], rel=1e-13)


# ---------------------------------------------------------------- whole-system endpoints

@pytest.fixture(scope="module")
def tiny():
    w = S.workload_tiny()
    return w.systems[0], w.params


def test_endpoint_coupled_equals_plain(tiny):
    s, P = tiny
    plain = s.copy()
    plain.is_ligand[:] = 0
    a = O.nonbonded(s, P, 1.0, 1.0)
    b = O.nonbonded(plain, P, 1.0, 1.0)
    assert a["E"].sum() == pytest.approx(b["E"].sum(), rel=1e-12)
    np.testing.assert_allclose(a["F"], b["F"], rtol=1e-10, atol=1e-8)


def test_endpoint_annihilated_is_zero_coupling(tiny):
    s, P = tiny
    a = O.nonbonded(s, P, 0.0, 0.0)
    e = a["energy"]
    for k in ("ligenv_lj", "liglig_lj", "ligenv_c", "liglig_c"):
        assert e[k] == 0.0
    lig = s.is_ligand.astype(bool)
    assert np.abs(a["F"][lig]).max() == 0.0
    # environment alone gives the same environment forces
    env = np.where(~lig)[0]
    sub = S.System("env", s.box, s.pos[env], s.vel[env], s.mass[env], s.charge[env],
                   s.sigma[env], s.epsilon[env], s.is_ligand[env],
                   s.excl[(s.excl < len(env)).all(1)], np.zeros((0, 2), np.int32),
                   np.zeros(0), np.zeros(0))
    b = O.nonbonded(sub, P, 1.0, 1.0)
    np.testing.assert_allclose(a["F"][env], b["F"], rtol=1e-12, atol=1e-9)


def test_decouple_keeps_ligand_internal(tiny):
    s, P = tiny
    Pd = dict(P, ligand_mode=1)
    a = O.nonbonded(s, Pd, 0.0, 0.0)["energy"]
    lig = np.where(s.is_ligand.astype(bool))[0]
    sub = S.System("lig", s.box, s.pos[lig], s.vel[lig], s.mass[lig], s.charge[lig],
                   s.sigma[lig], s.epsilon[lig], np.zeros(len(lig), np.uint8),
                   s.excl[(s.excl >= lig[0]).all(1)] - lig[0], np.zeros((0, 2), np.int32),
                   np.zeros(0), np.zeros(0))
    b = O.nonbonded(sub, P, 1.0, 1.0)["energy"]
    assert a["liglig_lj"] == pytest.approx(b["env_lj"], rel=1e-12)
    assert a["liglig_c"] == pytest.approx(b["env_c"], rel=1e-12)
    assert a["ligenv_lj"] == 0.0 and a["ligenv_c"] == 0.0


# ---------------------------------------------------------------- derivatives

def _safe_atoms(s, rc, h, k=12, seed=0):
    """Atoms with no partner within 3h of the cutoff sphere (finite differences
    must not cross the hard cutoff)."""
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.box * np.round(d / s.box)
    r = np.linalg.norm(d, axis=2)
    bad = (np.abs(r - rc) < 3 * h).any(1)
    cand = np.where(~bad)[0]
    rng = np.random.default_rng(seed)
    lig = [i for i in cand if s.is_ligand[i]][:4]
    env = list(rng.choice([i for i in cand if not s.is_ligand[i]], k - len(lig), replace=False))
    return lig + env


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("lam", [(0.0, 0.6, 0.4), (0.0, 1.0, 0.85)])
def test_forces_are_minus_gradient(tiny, lam, mode):
    s, P = tiny
    P = dict(P, ligand_mode=mode)
    h = 1e-6
    F = O.nonbonded(s, P, lam[1], lam[2])["F"]
    for i in _safe_atoms(s, P["cutoff"], h):
        for k in range(3):
            xp, xm = s.pos.copy(), s.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            ep = O.nonbonded(s, P, lam[1], lam[2], forces=False, pos=xp)["E"].sum()
            em = O.nonbonded(s, P, lam[1], lam[2], forces=False, pos=xm)["E"].sum()
            fd = -(ep - em) / (2 * h)
            assert F[i, k] == pytest.approx(fd, rel=2e-5, abs=2e-3 * max(1.0, abs(F[i]).max() * 1e-3))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("lam", [(0.6, 0.4), (1.0, 1.0), (0.0, 0.0), (0.25, 0.999)])
def test_force_rows_equal_full_pass_rows(tiny, lam, mode):
    """force_rows (the per-row reference of the sampled force checks at 60k and
    100k atoms) is a separate loop from nonbonded's pair loop: every row must
    equal the full pass's row up to summation order, in both ligand modes, and
    be minus the gradient of the total energy on rows far from the cutoff."""
    s, P = tiny
    P = dict(P, ligand_mode=mode)
    rows = np.arange(s.n)
    Fr = O.force_rows(s, P, lam[0], lam[1], rows)
    Ff = O.nonbonded(s, P, lam[0], lam[1])["F"]
    scale = np.abs(Ff).max()
    assert np.abs(Fr - Ff).max() <= 1e-12 * scale
    # a subset in shuffled order, with a repeated row
    sub = np.array([s.n - 1, 3, 600, 3, 650, 0])
    np.testing.assert_array_equal(O.force_rows(s, P, lam[0], lam[1], sub), Fr[sub])
    h = 1e-6
    for i in _safe_atoms(s, P["cutoff"], h, k=4, seed=3):
        for k in range(3):
            xp, xm = s.pos.copy(), s.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            ep = O.nonbonded(s, P, lam[0], lam[1], forces=False, pos=xp)["E"].sum()
            em = O.nonbonded(s, P, lam[0], lam[1], forces=False, pos=xm)["E"].sum()
            assert Fr[i, k] == pytest.approx(-(ep - em) / (2 * h), rel=2e-5,
                                             abs=2e-3 * max(1.0, abs(Fr[i]).max() * 1e-3))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("lq,lv", [(0.7, 0.3), (1.0, 1.0), (0.2, 0.999)])
def test_dudlambda_finite_difference(tiny, lq, lv, mode):
    s, P = tiny
    P = dict(P, ligand_mode=mode)
    h = 1e-6
    r = O.nonbonded(s, P, lq, lv, forces=False)
    U = lambda a, b: O.nonbonded(s, P, a, b, forces=False)["E"].sum()
    if lv + h <= 1.0:
        fd_v = (U(lq, lv + h) - U(lq, lv - h)) / (2 * h)
    else:  # second-order one-sided difference at the lambda = 1 end
        fd_v = (3 * U(lq, lv) - 4 * U(lq, lv - h) + U(lq, lv - 2 * h)) / (2 * h)
    fd_q = (U(lq + h, lv) - U(lq - h, lv)) / (2 * h)
    assert r["dudl_v"] == pytest.approx(fd_v, rel=1e-5, abs=1e-3)
    assert r["dudl_q"] == pytest.approx(fd_q, rel=1e-6, abs=1e-6)


def test_translation_invariance(tiny):
    s, P = tiny
    F = O.nonbonded(s, P, 0.5, 0.5)["F"]
    assert np.abs(F.sum(0)).max() < 1e-7 * np.abs(F).max()
    c = S.workload_loop().systems[0]
    # Boresch and bonds: net force zero
    _, Fb, _ = O.boresch(c, 0.7)
    assert np.abs(Fb.sum(0)).max() < 1e-9
    _, Fbd = O.bonds(c)
    assert np.abs(Fbd.sum(0)).max() < 1e-6
    # energy invariant under a rigid periodic shift
    sh = np.mod(s.pos + np.array([0.37, -0.21, 0.55]), s.box)
    e0 = O.nonbonded(s, P, 0.5, 0.5, forces=False)["E"].sum()
    e1 = O.nonbonded(s, P, 0.5, 0.5, forces=False, pos=sh)["E"].sum()
    assert e1 == pytest.approx(e0, rel=1e-11)


# ---------------------------------------------------------------- neighbour pairs

@pytest.mark.parametrize("box,rc", [(1.86, 0.9), (2.9, 1.0), (4.1, 1.2)])
def test_cell_list_matches_brute_force(box, rc):
    w = S.water_box(11, box)
    a = O.pairs_brute(w, rc)
    b = O.pairs_cell(w, rc)
    assert a.shape == b.shape
    assert (a == b).all()
    c = O.neighbor_counts(w, rc)
    assert c.sum() == 2 * len(a)


def test_pair_counts_match_energy_pass(tiny):
    s, P = tiny
    r = O.nonbonded(s, P, 0.5, 0.5, forces=False)
    p = O.pairs_brute(s, P["cutoff"])
    lig = s.is_ligand.astype(bool)
    n_lig = int((lig[p[:, 0]] | lig[p[:, 1]]).sum())
    assert r["npairs_lig"] == n_lig and r["npairs_env"] == len(p) - n_lig


# ---------------------------------------------------------------- Boresch restraint

def _boresch_sys(th0=(1.5, 1.4), ph0=(0.3, 1.2, -2.0), kr=4184.0, kth=41.84, kph=41.84):
    # P1 origin-ish, L1 0.6 nm along x, L2 +y of L1, L3 +z of L2,
    # P2 +y of P1, P3 -z of P2  (in a large box, away from the edges)
    o = np.array([2.0, 2.0, 2.0])
    pos = o + np.array([[0.0, 0.0, 0.0],     # P1
                        [0.0, 0.3, 0.0],     # P2
                        [0.0, 0.3, -0.3],    # P3
                        [0.6, 0.0, 0.0],     # L1
                        [0.6, 0.3, 0.0],     # L2
                        [0.6, 0.3, 0.3]])    # L3
    s = mk(pos, [0] * 6, [0] * 6, [0] * 6, [0, 0, 0, 1, 1, 1], box=6.0)
    s.boresch = S.Boresch(np.arange(6, dtype=np.int32), 0.5, np.array(th0), np.array(ph0),
                          kr, kth, kph)
    return s


def test_boresch_hand_geometry():
    s = _boresch_sys()
    U, F, g = O.boresch(s, 1.0)
    # r = 0.6; both angles are right angles; P2-P1-L1-L2 is cis (0).
    # P1-L1-L2-L3: looking along L1->L2 (+y), the first bond (-x) turns right-handed
    # by +90 deg onto the last (+z). L1-P1-P2-P3: along +y, +x turns by +90 deg onto -z.
    np.testing.assert_allclose(g, [0.6, np.pi / 2, np.pi / 2, 0.0, np.pi / 2, np.pi / 2],
                               atol=1e-12)
    b = s.boresch
    want = (0.5 * b.k_r * (0.6 - b.r0) ** 2
            + 0.5 * b.k_theta * ((np.pi / 2 - b.theta0[0]) ** 2 + (np.pi / 2 - b.theta0[1]) ** 2)
            + b.k_phi * ((1 - np.cos(0.0 - b.phi0[0])) + (1 - np.cos(np.pi / 2 - b.phi0[1]))
                         + (1 - np.cos(np.pi / 2 - b.phi0[2]))))
    assert U == pytest.approx(want, rel=1e-12)


def test_boresch_lambda_zero_and_scaling():
    s = _boresch_sys()
    U0, F0, _ = O.boresch(s, 0.0)
    assert np.abs(F0).max() == 0.0
    U1, F1, _ = O.boresch(s, 1.0)
    U3, F3, _ = O.boresch(s, 0.3)
    assert U0 == U1 == U3   # U_B is the unscaled restraint energy (= dU/dlambda_r)
    np.testing.assert_allclose(F3, 0.3 * F1, rtol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_boresch_finite_difference(seed):
    s = _boresch_sys()
    rng = np.random.default_rng(seed)
    s.pos = s.pos + rng.normal(0, 0.05, s.pos.shape)
    _, F, _ = O.boresch(s, 1.0)
    h = 1e-6
    for i in range(6):
        for k in range(3):
            xp, xm = s.pos.copy(), s.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(O.boresch(s, 1.0, pos=xp, forces=False)[0]
                   - O.boresch(s, 1.0, pos=xm, forces=False)[0]) / (2 * h)
            assert F[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-5)


def test_boresch_periodic_image():
    s = _boresch_sys()
    U, _, g = O.boresch(s, 1.0)
    sh = s.pos.copy()
    sh[3:] += np.array([6.0, 0.0, -6.0])  # move the ligand by whole box vectors
    U2, _, g2 = O.boresch(s, 1.0, pos=sh)
    assert U2 == pytest.approx(U, rel=1e-12)
    np.testing.assert_allclose(g2, g, atol=1e-12)


def test_bonds_finite_difference():
    w = S.water_box(3, 1.9)
    _, F = O.bonds(w)
    h = 1e-6
    for i in (0, 1, 2, 30, 31):
        for k in range(3):
            xp, xm = w.pos.copy(), w.pos.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(O.bonds(w, xp, False)[0] - O.bonds(w, xm, False)[0]) / (2 * h)
            assert F[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-4)


# ---------------------------------------------------------------- reduced potentials

def test_ukn_lambda_part_matches_full_difference(tiny):
    s, P = tiny
    sch = S.schedule_k12()
    full = O.ukn(s, P, sch, with_bonds=False) * P["kT"]
    part = O.ukn_lambda_part(s, P, sch)
    env = O.nonbonded(s, P, 1.0, 1.0, forces=False)
    e_env = env["energy"]["env_lj"] + env["energy"]["env_c"]
    np.testing.assert_allclose(full, part + e_env, rtol=1e-12)


def test_ukn_endpoint_states(tiny):
    s, P = tiny
    sch = S.schedule_k12()
    u = O.ukn(s, P, sch, with_bonds=False)
    plain = s.copy()
    plain.is_ligand[:] = 0
    u0 = O.nonbonded(plain, P, 1, 1, forces=False)["E"].sum() / P["kT"]
    assert u[0] == pytest.approx(u0, rel=1e-12)          # state 0 is fully coupled
    e = O.nonbonded(s, P, 0, 0, forces=False)
    assert u[-1] == pytest.approx(e["E"][:2].sum() / P["kT"], rel=1e-12)  # fully annihilated


# ---------------------------------------------------------------- integrator

def _small_md_system():
    w = S.water_box(21, 2.0)
    P = dict(cutoff=0.9, ewald_beta=3.47, sc_alpha=0.5, sc_p=1.0, coulomb_k=KE,
             kT=S.BOLTZMANN_KJ * 300, ligand_mode=0)
    return w, P


def test_baoab_gamma_zero_is_velocity_verlet():
    w, P = _small_md_system()
    lam = (0.0, 1.0, 1.0)
    dt = 0.001
    x0, v0 = w.pos.copy(), w.vel.copy()
    F0 = O.total_forces(w, P, lam, pos=x0)[0]
    x1, v1, _ = O.baoab_step(w, P, lam, x0, v0, dt, 0.0, seed=1, step=0, F=F0)
    m = w.mass[:, None]
    xv = x0 + dt * v0 + 0.5 * dt * dt * F0 / m
    F1 = O.total_forces(w, P, lam, pos=xv)[0]
    vv = v0 + 0.5 * dt * (F0 + F1) / m
    np.testing.assert_allclose(x1, xv, rtol=0, atol=1e-13)
    np.testing.assert_allclose(v1, vv, rtol=1e-10, atol=1e-9)


def test_baoab_o_step_variance():
    w, P = _small_md_system()
    lam = (0.0, 1.0, 1.0)
    zero = np.zeros_like(w.pos)
    # F = 0 and gamma dt -> infinity: v' = sqrt(kT/m) xi exactly
    x1, v1, _ = O.baoab_step(w, P, lam, w.pos, zero, 1e-12, 1e14, seed=9, step=3, F=zero)
    z = v1 / np.sqrt(P["kT"] / w.mass[:, None])
    assert abs(z.var() - 1.0) < 0.05
    assert abs(z.mean()) < 0.05


# ------------------------------------------------------------------ replica exchange

def test_exchange_downhill_always_accepted_and_permutation():
    from oracle.exchange import attempt, exchange_groups
    rng = np.random.default_rng(3)
    R = 6
    groups = exchange_groups([0] * R, [0] * R)
    states = np.array([3, 0, 5, 1, 4, 2])
    # u_k(x_r) = (k - c_r)^2 with replica r's well at c_r = its own state: every
    # swap is uphill; with c_r at the swapped states every swap is downhill
    u_up = np.array([[(k - states[r]) ** 2 * 5.0 for k in range(R)] for r in range(R)])
    s1, acc = attempt(u_up, states, groups, seed=1, t=0)
    assert sorted(s1) == list(range(R))
    # uphill by 10 kT per swap: essentially never accepted
    assert acc == 0 and np.array_equal(s1, states)
    swapped = states.copy()
    order = sorted(range(R), key=lambda r: states[r])
    for m in (0, 2, 4):
        i, j = order[m], order[m + 1]
        swapped[i], swapped[j] = states[j], states[i]
    u_down = np.array([[(k - swapped[r]) ** 2 * 5.0 for k in range(R)] for r in range(R)])
    s2, acc2 = attempt(u_down, states, groups, seed=1, t=0)
    assert acc2 == 3 and np.array_equal(s2, swapped)
    # odd attempt pairs positions (1,2), (3,4): position 5 has no partner
    s3, acc3 = attempt(u_down, states, groups, seed=1, t=1)
    assert sorted(s3) == list(range(R)) and acc3 <= 2
    del rng


def test_exchange_stationary_ratio_two_replicas():
    """Detailed balance: for two replicas with fixed coordinates the chain of
    attempts visits the swapped assignment with odds exp(-D) (Metropolis)."""
    from oracle.exchange import attempt
    groups = [[0, 1]]
    D = 0.7
    # u[r][k]: assignment A = (0 -> state 0, 1 -> state 1) energy 0, B energy D
    u = np.array([[0.0, 0.5 * D], [0.5 * D, 0.0]])
    st = np.array([0, 1])
    n_b = 0
    n = 6000
    for t in range(0, 2 * n, 2):            # even attempts carry the pair
        st, _ = attempt(u, st, groups, seed=77, t=t)
        n_b += int(st[0] == 1)
    p_b = n_b / n
    expect = math.exp(-D) / (1 + math.exp(-D))
    assert abs(p_b - expect) < 4 * math.sqrt(expect * (1 - expect) / n) + 0.01

