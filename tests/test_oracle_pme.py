"""Pins of the reciprocal-space Ewald references (Madelung constant, beta
invariance, finite differences, SPME -> Ewald sum as the grid refines, the
excluded-pair correction's sign)."""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle.pme import (ewald_reciprocal, exclusion_correction, self_energy, spme)

KE = 138.935458


def real_space(pos, q, box, beta, rc):
    """Plain real-space Ewald sum (minimum image, r < rc), numpy, for the pins."""
    E = 0.0
    for i in range(len(q)):
        d = pos[i + 1:] - pos[i]
        d -= box * np.round(d / box)
        r = np.sqrt((d ** 2).sum(1))
        m = r < rc
        E += KE * float((q[i] * q[i + 1:][m] * erfc(beta * r[m]) / r[m]).sum())
    return E


def rocksalt(cells, a):
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    na = base
    cl = base + np.array([0.5, 0, 0])
    pos, q = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                off = np.array([i, j, k])
                pos += list((na + off) * a) + list((cl + off) * a)
                q += [1.0] * 4 + [-1.0] * 4
    return np.array(pos), np.array(q), np.full(3, cells * a)


def test_madelung_rocksalt():
    """Total Ewald energy of rock salt = -M k_e q^2 / r0 per ion pair,
    M = 1.747565 (NaCl)."""
    a = 0.5
    pos, q, box = rocksalt(4, a)
    beta, rc = 3.6, 0.99
    E = (real_space(pos, q, box, beta, rc) + ewald_reciprocal(pos, q, box, beta, 12, KE, False)[0]
         + self_energy(q, beta, KE))
    per_pair = E / (len(q) / 2)
    expect = -1.747565 * KE / (a / 2)
    assert per_pair == pytest.approx(expect, rel=2e-6)


def _random_neutral(n, L, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, (n, 3))
    q = rng.normal(0, 0.5, n)
    q -= q.mean()
    return pos, q, np.full(3, L)


def test_total_energy_independent_of_beta():
    pos, q, box = _random_neutral(40, 3.0, 1)
    tot = []
    for beta in (2.6, 3.0, 3.4):
        tot.append(real_space(pos, q, box, beta, 1.45)
                   + ewald_reciprocal(pos, q, box, beta, 14, KE, False)[0]
                   + self_energy(q, beta, KE))
    assert max(tot) - min(tot) < 1e-6 * max(abs(t) for t in tot) + 1e-9


def test_reciprocal_forces_by_differences():
    pos, q, box = _random_neutral(12, 2.0, 2)
    beta, kmax = 3.0, 8
    E, F = ewald_reciprocal(pos, q, box, beta, kmax, KE)
    h = 1e-5
    for j, a in [(0, 0), (3, 1), (7, 2)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[j, a] += h
        p2[j, a] -= h
        fd = -(ewald_reciprocal(p1, q, box, beta, kmax, KE, False)[0]
               - ewald_reciprocal(p2, q, box, beta, kmax, KE, False)[0]) / (2 * h)
        assert F[j, a] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    assert np.abs(F.sum(0)).max() < 1e-8 * np.abs(F).max()


def test_spme_converges_to_ewald_sum():
    """SPME approaches the Ewald sum as the grid refines, at the rate of its
    B-spline order (error ~ h^p)."""
    pos, q, box = _random_neutral(30, 2.4, 3)
    beta = 3.1
    Ee, Fe = ewald_reciprocal(pos, q, box, beta, 12, KE)

    def err(K, p):
        Es, Fs = spme(pos, q, box, beta, (K, K, K), p, KE)
        return abs(Es - Ee) / abs(Ee), math.sqrt(((Fs - Fe) ** 2).sum() / (Fe ** 2).sum())

    e16, e32 = err(16, 4), err(32, 4)
    assert e32[0] < 2e-4 and e32[1] < 2e-3
    assert e32[1] < e16[1] / 8                 # ~2^-4 per halving at order 4
    s32 = err(32, 6)
    assert s32[0] < 5e-6 and s32[1] < 5e-5     # order 6 at the same spacing


def test_spme_forces_by_differences():
    pos, q, box = _random_neutral(10, 2.0, 4)
    E, F = spme(pos, q, box, 3.0, (20, 20, 20), 4, KE)
    h = 1e-5
    for j, a in [(0, 0), (5, 2)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[j, a] += h
        p2[j, a] -= h
        fd = -(spme(p1, q, box, 3.0, (20, 20, 20), 4, KE, False)[0]
               - spme(p2, q, box, 3.0, (20, 20, 20), 4, KE, False)[0]) / (2 * h)
        assert F[j, a] == pytest.approx(fd, rel=1e-5, abs=1e-5)


def test_excluded_pair_cancels_reciprocal_and_self():
    """An excluded +q/-q pair far from everything: its reciprocal and self
    energies are cancelled by the correction (what remains is the pair's
    dipole interacting with its periodic images)."""
    box = np.full(3, 6.0)
    pos = np.array([[3.0, 3.0, 3.0], [3.1, 3.0, 3.0]])
    q = np.array([0.8, -0.8])
    beta = 3.0
    Er = ewald_reciprocal(pos, q, box, beta, 16, KE, False)[0]
    Es = self_energy(q, beta, KE)
    Ex = exclusion_correction(pos, q, box, [[0, 1]], beta, KE, False)[0]
    scale = KE * 0.64 / 0.1
    assert abs(Er + Es + Ex) < 1e-3 * scale
    assert Ex > 0                      # removing an attractive pair raises the energy


def test_exclusion_correction_forces_by_differences():
    rng = np.random.default_rng(0)
    pos = rng.uniform(0, 2, (6, 3))
    q = rng.normal(0, 0.5, 6)
    box = np.full(3, 2.0)
    ex = [[0, 1], [2, 3], [1, 4]]
    E, F = exclusion_correction(pos, q, box, ex, 3.1, KE)
    h = 1e-6
    for j, a in [(0, 0), (1, 1), (4, 2), (3, 0)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[j, a] += h
        p2[j, a] -= h
        fd = -(exclusion_correction(p1, q, box, ex, 3.1, KE, False)[0]
               - exclusion_correction(p2, q, box, ex, 3.1, KE, False)[0]) / (2 * h)
        assert F[j, a] == pytest.approx(fd, rel=1e-7, abs=1e-7)
