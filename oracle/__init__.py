"""FP64 CPU oracle for the alchemical nonbonded path (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA path.

The arithmetic lives in ``abfe_oracle.c`` (plain C, double precision, all
pairs with the minimum image); this module compiles it with gcc, loads it with
ctypes and adds the few steps that are plain numpy (the BAOAB step, the reduced
potential row). Each function names the part of the paper it restates:

* softcore LJ, mixing, pair lambda, charge scaling: "Double annihilation protocol";
* real-space Ewald at a hard cutoff: "Additional methodological details";
* Boresch restraint: "Restraints";
* periodic torsions of rotatable ligand bonds scaled by lambda_v (torsion.py)
  and alchemical waters that keep the box neutral (alchemical_water.py):
  "Double annihilation protocol";
* reduced potentials u_kn fed to MBAR: "Simulation protocol";
* BAOAB Langevin splitting (Leimkuhler & Matthews 2013) standing in for the
  paper's LangevinMiddle integrator of "Simulation protocol".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import alchemical_water as _aw
from .torsion import torsions as _torsions

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "abfe_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liborc.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Sys(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", C.c_void_p), ("box", C.c_void_p),
                ("charge", C.c_void_p), ("sigma", C.c_void_p), ("epsilon", C.c_void_p),
                ("is_lig", C.c_void_p), ("ex_off", C.c_void_p), ("ex_idx", C.c_void_p)]


class _Par(C.Structure):
    _fields_ = [("cutoff", C.c_double), ("beta", C.c_double), ("alpha", C.c_double),
                ("p", C.c_double), ("ke", C.c_double), ("mode", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        L.orc_nonbonded.argtypes = [P, P, C.c_double, C.c_double, C.c_int, P, P, P, P]
        L.orc_force_rows.argtypes = [P, P, C.c_double, C.c_double, C.c_int, P, P]
        L.orc_neighbor_counts.argtypes = [P, C.c_double, P]
        L.orc_pairs_brute.argtypes = [P, C.c_double, C.c_int64, P]
        L.orc_pairs_brute.restype = C.c_int64
        L.orc_pairs_cell.argtypes = [P, C.c_double, C.c_int64, P]
        L.orc_pairs_cell.restype = C.c_int64
        L.orc_boresch.argtypes = [P, P, P, C.c_double, P, P, C.c_double, C.c_double, C.c_double,
                                  C.c_double, P, P, P]
        L.orc_bonds.argtypes = [P, P, C.c_int, P, P, P, P, P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_gauss3.argtypes = [C.c_int, C.c_uint64, C.c_uint64, C.c_uint32, P]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleSystem:
    """Contiguous FP64 copies of a system plus its exclusion CSR."""

    def __init__(self, s, pos=None):
        self.s = s
        self.n = s.n
        self.pos = np.ascontiguousarray(s.pos if pos is None else pos, dtype=np.float64)
        self.box = np.ascontiguousarray(s.box, dtype=np.float64)
        self.q = np.ascontiguousarray(s.charge, dtype=np.float64)
        self.sig = np.ascontiguousarray(s.sigma, dtype=np.float64)
        self.eps = np.ascontiguousarray(s.epsilon, dtype=np.float64)
        self.lig = np.ascontiguousarray(s.is_ligand, dtype=np.uint8)
        ex = np.asarray(s.excl, dtype=np.int64).reshape(-1, 2)
        both = np.concatenate([ex, ex[:, ::-1]]) if len(ex) else np.zeros((0, 2), np.int64)
        order = np.lexsort((both[:, 1], both[:, 0]))
        both = both[order]
        cnt = np.bincount(both[:, 0], minlength=self.n) if len(both) else np.zeros(self.n, int)
        self.ex_off = np.zeros(self.n + 1, np.int32)
        self.ex_off[1:] = np.cumsum(cnt)
        self.ex_idx = np.ascontiguousarray(both[:, 1], dtype=np.int32)
        self._c = _Sys(self.n, self.pos.ctypes.data, self.box.ctypes.data, self.q.ctypes.data,
                       self.sig.ctypes.data, self.eps.ctypes.data, self.lig.ctypes.data,
                       self.ex_off.ctypes.data, self.ex_idx.ctypes.data)

    def ref(self):
        return C.byref(self._c)


def _par(P):
    return _Par(P["cutoff"], P["ewald_beta"], P["sc_alpha"], P["sc_p"], P["coulomb_k"],
                int(P.get("ligand_mode", 0)))


ENERGY_NAMES = ("env_lj", "env_c", "ligenv_lj", "liglig_lj", "ligenv_c", "liglig_c")


def nonbonded(s, P, lam_q, lam_v, ligand_only=False, forces=True, pos=None):
    """Nonbonded energies/forces/derivatives at (lam_q, lam_v), all pairs. A
    system with alchemical waters is evaluated with their charges at lam_q, and
    their part of dU/dlambda_q is added (a prepared OracleSystem is taken as
    it is)."""
    if not isinstance(s, OracleSystem) and _aw.has_waters(s):
        r = nonbonded(OracleSystem(_aw.system_at(s, lam_q), pos), P, lam_q, lam_v, ligand_only,
                      forces)
        r["dudl_q"] += _aw.dudlq_waters(s, P, lam_q, pos)
        return r
    o = s if isinstance(s, OracleSystem) else OracleSystem(s, pos)
    F = np.zeros((o.n, 3)) if (forces and not ligand_only) else None
    E = np.zeros(6)
    d = np.zeros(2)
    npairs = np.zeros(2, np.int64)
    par = _par(P)
    rc = lib().orc_nonbonded(o.ref(), C.byref(par), float(lam_q), float(lam_v),
                             int(bool(ligand_only)), _p(F) if F is not None else None,
                             _p(E), _p(d), _p(npairs))
    if rc != 0:
        raise MemoryError("orc_nonbonded failed")
    return dict(F=F, E=E, energy=dict(zip(ENERGY_NAMES, E)), dudl_v=d[0], dudl_q=d[1],
                npairs_env=int(npairs[0]), npairs_lig=int(npairs[1]))


def force_rows(s, P, lam_q, lam_v, rows, pos=None):
    if not isinstance(s, OracleSystem) and _aw.has_waters(s):
        s = _aw.system_at(s, lam_q)
    o = s if isinstance(s, OracleSystem) else OracleSystem(s, pos)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    F = np.zeros((len(rows), 3))
    par = _par(P)
    lib().orc_force_rows(o.ref(), C.byref(par), float(lam_q), float(lam_v), len(rows),
                         _p(rows), _p(F))
    return F


def neighbor_counts(s, rc, pos=None):
    o = s if isinstance(s, OracleSystem) else OracleSystem(s, pos)
    c = np.zeros(o.n, np.int32)
    lib().orc_neighbor_counts(o.ref(), float(rc), _p(c))
    return c


def _pairs(fn, s, rc):
    o = s if isinstance(s, OracleSystem) else OracleSystem(s)
    cap = 1 << 16
    while True:
        out = np.zeros((cap, 2), np.int32)
        m = fn(o.ref(), float(rc), cap, _p(out))
        if m < 0:
            raise MemoryError
        if m <= cap:
            return out[:m]
        cap = int(m)


def pairs_brute(s, rc):
    return _pairs(lib().orc_pairs_brute, s, rc)


def pairs_cell(s, rc):
    p = _pairs(lib().orc_pairs_cell, s, rc)
    return p[np.lexsort((p[:, 1], p[:, 0]))]


def boresch(s, lam_r, pos=None, forces=True):
    """Boresch restraint: returns (U_B unscaled, forces of lam_r*U_B, geometry)."""
    b = s.boresch
    pos = np.ascontiguousarray(s.pos if pos is None else pos, dtype=np.float64)
    box = np.ascontiguousarray(s.box, dtype=np.float64)
    anc = np.ascontiguousarray(b.anchors, dtype=np.int32)
    th0 = np.ascontiguousarray(b.theta0, dtype=np.float64)
    ph0 = np.ascontiguousarray(b.phi0, dtype=np.float64)
    F = np.zeros_like(pos) if forces else None
    U = np.zeros(1)
    geom = np.zeros(6)
    lib().orc_boresch(_p(pos), _p(box), _p(anc), float(b.r0), _p(th0), _p(ph0), float(b.k_r),
                      float(b.k_theta), float(b.k_phi), float(lam_r),
                      _p(F) if F is not None else None, _p(U), _p(geom))
    return float(U[0]), F, geom


def bonds(s, pos=None, forces=True):
    pos = np.ascontiguousarray(s.pos if pos is None else pos, dtype=np.float64)
    box = np.ascontiguousarray(s.box, dtype=np.float64)
    idx = np.ascontiguousarray(s.bonds, dtype=np.int32)
    r0 = np.ascontiguousarray(s.bond_r0, dtype=np.float64)
    kb = np.ascontiguousarray(s.bond_k, dtype=np.float64)
    F = np.zeros_like(pos) if forces else None
    U = np.zeros(1)
    lib().orc_bonds(_p(pos), _p(box), len(idx), _p(idx), _p(r0), _p(kb),
                    _p(F) if F is not None else None, _p(U))
    return float(U[0]), F


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def gauss3(n, seed, step, replica):
    out = np.zeros((n, 3))
    lib().orc_gauss3(int(n), int(seed), int(step), int(replica), _p(out))
    return out


def num_threads():
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------- whole-state helpers

def torsion_state(s, P, lam_v, pos=None, forces=True):
    """Rotatable-bond torsions at lambda_v: (energy of the state, forces or
    None, dU/dlambda_v); see torsion.py."""
    mode = int(P.get("ligand_mode", 0))
    U, F, d = _torsions(s, lam_v, pos=pos, forces=forces, ligand_mode=mode)
    return (lam_v * U if mode == 0 else U), F, d


def state_energy(s, P, lam, pos=None, with_bonds=True):
    """Total potential U(x; lambda) = nonbonded + lambda_r U_B + torsions at
    lambda_v + bonded terms, with the parts and the three partial derivatives
    (restraint, coul, vdw)."""
    lam_r, lam_q, lam_v = lam
    nb = nonbonded(s, P, lam_q, lam_v, forces=False, pos=pos)
    UB = boresch(s, lam_r, pos=pos, forces=False)[0] if s.boresch is not None else 0.0
    Ub = bonds(s, pos=pos, forces=False)[0] if with_bonds else 0.0
    Ut, _, dt = torsion_state(s, P, lam_v, pos=pos, forces=False)
    U = float(nb["E"].sum()) + lam_r * UB + Ub + Ut
    return dict(U=U, nb=nb, U_B=UB, U_bond=Ub, U_tors=Ut,
                dudl=np.array([UB, nb["dudl_q"], nb["dudl_v"] + dt]))


def total_forces(s, P, lam, pos=None, with_bonds=True):
    lam_r, lam_q, lam_v = lam
    nb = nonbonded(s, P, lam_q, lam_v, forces=True, pos=pos)
    F = nb["F"].copy()
    if s.boresch is not None:
        F += boresch(s, lam_r, pos=pos)[1]
    if with_bonds:
        F += bonds(s, pos=pos)[1]
    F += torsion_state(s, P, lam_v, pos=pos)[1]
    return F, nb


def ukn(s, P, sched, pos=None, with_bonds=True):
    """Reduced potentials u_k = U(x; lambda_k) / kT at every state k of the
    schedule (all pairs evaluated at each state)."""
    return np.array([state_energy(s, P, sched.state(k), pos, with_bonds)["U"] / P["kT"]
                     for k in range(sched.K)])


def ukn_lambda_part(s, P, sched, pos=None):
    """The lambda-dependent part of u_k, U_k - U_env, in kJ/mol: every pair with
    a ligand atom at state k plus lambda_r,k U_B plus the rotatable-bond torsions
    at lambda_v,k (annihilation; with decoupling they are lambda independent and
    left out, like the ligand's own pairs are not). The remaining pairs and the
    bonded terms are the same at every state. With alchemical waters the part
    also holds the change of their Coulomb pairs from lambda_q = 1, and the
    ligand pairs see their charges at the state."""
    water = _aw.has_waters(s)
    o = OracleSystem(s, pos)
    UB = boresch(s, 1.0, pos=pos, forces=False)[0] if s.boresch is not None else 0.0
    UT = _torsions(s, 1.0, pos=pos, forces=False)[0] if int(P.get("ligand_mode", 0)) == 0 else 0.0
    w1 = _aw.water_pair_energy(s, P, 1.0, pos) if water else 0.0
    out = np.zeros(sched.K)
    for k in range(sched.K):
        lr, lq, lv = sched.state(k)
        ok = OracleSystem(_aw.system_at(s, lq), pos) if water else o
        nb = nonbonded(ok, P, lq, lv, ligand_only=True, forces=False)
        out[k] = float(nb["E"].sum()) + lr * UB + lv * UT
        if water:
            out[k] += _aw.water_pair_energy(s, P, lq, pos) - w1
    return out


def baoab_step(s, P, lam, x, v, dt, gamma, seed, step, replica=0, F=None):
    """One BAOAB step: B (half kick), A (half drift), O (exact Ornstein-Uhlenbeck
    with c1 = exp(-gamma dt)), A, new forces, B. Returns (x, v, F_new)."""
    m = np.asarray(s.mass, dtype=np.float64)[:, None]
    kT = P["kT"]
    if F is None:
        F = total_forces(s, P, lam, pos=x)[0]
    v = v + 0.5 * dt * F / m
    x = x + 0.5 * dt * v
    c1 = np.exp(-gamma * dt)
    xi = gauss3(s.n, seed, step, replica)
    v = c1 * v + np.sqrt((1.0 - c1 * c1) * kT / m) * xi
    x = x + 0.5 * dt * v
    F2 = total_forces(s, P, lam, pos=x)[0]
    v = v + 0.5 * dt * F2 / m
    return x, v, F2
