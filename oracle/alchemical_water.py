"""Reference alchemical waters (TEST INFRASTRUCTURE).

The paper keeps every simulation box neutral along the alchemical path: a
charged ligand's lost fraction of charge is taken up by designated "alchemical
waters", each offsetting a fractional ligand charge between -0.4 and 0.6 e,
with the number of such waters fixed across all windows ("Double annihilation
protocol"). Reading taken: with ligand net charge Q_L and n_w alchemical
waters, the oxygen of water w carries q_w(lambda_q) = q0_w + (1 - lambda_q)
dq_w, sum_w dq_w = Q_L (so the total charge lambda_q Q_L + Q_env + (1 -
lambda_q) Q_L does not depend on lambda_q), n_w the smallest count with
Q_L / n_w in [-0.4, 0.6] and dq_w = Q_L / n_w. Only the Coulomb charges change;
Lennard-Jones terms and bonds of those waters are untouched.

Functions here give the state's charges and the parts of the energy and of
dU/dlambda_q that involve the alchemical waters, by plain loops over the few
alchemical oxygens and all atoms (minimum image, hard cutoff, exclusions,
real-space Ewald erfc(beta r)/r), in FP64.
"""
from __future__ import annotations

import math

import numpy as np


def has_waters(s) -> bool:
    return len(getattr(s, "alch_water", ())) > 0


def charges_at(s, lam_q):
    """The per-atom charges that are not lambda-scaled ligand charges at
    lambda_q: the alchemical oxygens carry q0 + (1 - lambda_q) dq."""
    q = np.array(s.charge, dtype=np.float64)
    if has_waters(s):
        idx = np.asarray(s.alch_water, dtype=np.int64)
        q[idx] += (1.0 - float(lam_q)) * np.asarray(s.alch_water_dq, dtype=np.float64)
    return q


def system_at(s, lam_q):
    """A shallow copy of s whose charge array holds charges_at(s, lam_q)."""
    import copy
    t = copy.copy(s)
    t.charge = charges_at(s, lam_q)
    return t


def _excluded_sets(s):
    ex = {}
    for i, j in np.asarray(s.excl, dtype=np.int64).reshape(-1, 2):
        ex.setdefault(int(i), set()).add(int(j))
        ex.setdefault(int(j), set()).add(int(i))
    return ex


def _erfc_over_r(P, r):
    return np.array([math.erfc(P["ewald_beta"] * x) / x for x in r])


def potentials(s, P, lam_q, pos=None):
    """For every alchemical oxygen a: phi_a = sum over atoms j != a within the
    cutoff, not excluded, of k_e q_j(lambda) erfc(beta r)/r, with q_j(lambda)
    the state's charges (ligand charges times lambda_q, alchemical oxygens at
    lambda_q). Returns phi (FP64, kJ/mol/e)."""
    x = np.asarray(s.pos if pos is None else pos, dtype=np.float64)
    box = np.asarray(s.box, dtype=np.float64)
    q = charges_at(s, lam_q)
    lig = np.asarray(s.is_ligand, dtype=bool)
    q = np.where(lig, float(lam_q) * q, q)
    ex = _excluded_sets(s)
    rc = P["cutoff"]
    out = []
    for a in np.asarray(s.alch_water, dtype=np.int64):
        d = x - x[a]
        d -= box * np.round(d / box)
        r = np.sqrt((d * d).sum(1))
        sel = (r < rc)
        sel[a] = False
        for j in ex.get(int(a), ()):
            sel[j] = False
        j = np.where(sel)[0]
        out.append(P["coulomb_k"] * float(np.sum(q[j] * _erfc_over_r(P, r[j]))))
    return np.array(out)


def dudlq_waters(s, P, lam_q, pos=None):
    """The alchemical waters' part of dU/dlambda_q at lambda_q: each oxygen's
    charge changes by -dq_a per unit lambda_q, so the part is -sum_a dq_a phi_a
    (phi_a includes the other alchemical oxygens; each pair of them is counted
    from both ends, as the product rule requires)."""
    if not has_waters(s):
        return 0.0
    return -float(np.sum(np.asarray(s.alch_water_dq, dtype=np.float64) *
                         potentials(s, P, lam_q, pos)))


def water_pair_energy(s, P, lam_q, pos=None):
    """Coulomb energy of every pair with at least one alchemical oxygen and no
    ligand atom, at lambda_q (each pair once)."""
    if not has_waters(s):
        return 0.0
    x = np.asarray(s.pos if pos is None else pos, dtype=np.float64)
    box = np.asarray(s.box, dtype=np.float64)
    q = charges_at(s, lam_q)
    lig = np.asarray(s.is_ligand, dtype=bool)
    aw = np.asarray(s.alch_water, dtype=np.int64)
    is_aw = np.zeros(len(q), bool)
    is_aw[aw] = True
    ex = _excluded_sets(s)
    rc = P["cutoff"]
    e = 0.0
    for a in aw:
        d = x - x[a]
        d -= box * np.round(d / box)
        r = np.sqrt((d * d).sum(1))
        sel = (r < rc) & ~lig
        sel[a] = False
        sel &= ~(is_aw & (np.arange(len(q)) < a))      # alchemical pairs once
        for j in ex.get(int(a), ()):
            sel[j] = False
        j = np.where(sel)[0]
        e += P["coulomb_k"] * q[a] * float(np.sum(q[j] * _erfc_over_r(P, r[j])))
    return e


def count_for(q_net, lo=-0.4, hi=0.6):
    """The smallest number of alchemical waters n with q_net / n in [lo, hi]."""
    if abs(q_net) < 1e-12:
        return 0
    n = 1
    while not (lo - 1e-12 <= q_net / n <= hi + 1e-12):
        n += 1
    return n
