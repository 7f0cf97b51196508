"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *draws* inputs: atom coordinates, force-field parameters,
topology (exclusions, bonds), Boresch anchor choices and lambda schedules.
It contains none of the method's arithmetic (no energies, forces, softcore,
Ewald or restraint terms), so it cannot make the oracle and the CUDA path
agree by construction.

The systems stand in for the paper's complex (protein-ligand) and solvent
(ligand-water) legs, whose structures and parameters are not available:

* water-like solvent: rigid-geometry 3-site molecules (O -0.834 e, H +0.417 e,
  O-only Lennard-Jones sigma 0.315 nm, epsilon 0.636 kJ/mol) on a jittered
  lattice at about 33.4 molecules per nm^3 (about 100 atoms per nm^3);
* protein-like core: a dense sphere (about 110 atoms per nm^3) of 14 random
  atom types held together by an elastic network of harmonic bonds;
* ligand: a seeded self-avoiding chain with random charges (made neutral),
  sigma in U[0.25, 0.40] nm and epsilon in U[0.2, 1.0] kJ/mol.

Every coordinate, box length and parameter is rounded to a value that is
exactly representable in IEEE binary32, so that an FP32 device copy and an
FP64 host copy describe the same system.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
from scipy.spatial import cKDTree

from .schedule import (  # noqa: F401  (re-exported)
    LambdaSchedule,
    paper_complex_schedule,
    paper_solvent_schedule,
    schedule_k12,
    schedule_k24,
    schedule_k42,
    schedule_solvent_k30,
)

# Physical constants passed as *inputs* to both the oracle and the CUDA path.
BOLTZMANN_KJ = 0.00831446261815324   # kJ mol^-1 K^-1
COULOMB_K = 138.935458               # kJ mol^-1 nm e^-2

# 3-site water geometry (nm, degrees) and its model parameters.
WATER_ROH = 0.09572
WATER_HOH_DEG = 104.52
WATER_Q_O, WATER_Q_H = -0.834, 0.417
WATER_SIG_O, WATER_EPS_O = 0.315, 0.636
MASS_O, MASS_H, MASS_C = 15.999, 1.008, 12.011

# Harmonic terms that keep the synthetic molecules together during MD.
K_WATER_OH = 3.0e5      # kJ mol^-1 nm^-2
K_WATER_HH = 2.0e5
K_CORE = 2.0e4
K_LIGAND = 2.0e5
K_LIGAND_13 = 2.0e5     # ligand 1-3 pairs (holds the bond angles)


def f32(a):
    """Round to the nearest binary32 value, kept as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Boresch:
    """Anchor atoms and reference geometry of a Boresch restraint.

    anchors: original atom indices (P1, P2, P3, L1, L2, L3).
    theta0:  reference angles (P1-L1-L2, L1-P1-P2), radians.
    phi0:    reference dihedrals (P2-P1-L1-L2, P1-L1-L2-L3, L1-P1-P2-P3), radians.
    """
    anchors: np.ndarray
    r0: float
    theta0: np.ndarray
    phi0: np.ndarray
    k_r: float
    k_theta: float
    k_phi: float


@dataclass
class System:
    name: str
    box: np.ndarray                 # (3,) orthorhombic box lengths, nm
    pos: np.ndarray                 # (n,3) nm, in [0, box)
    vel: np.ndarray                 # (n,3) nm/ps
    mass: np.ndarray                # (n,) amu
    charge: np.ndarray              # (n,) e
    sigma: np.ndarray               # (n,) nm
    epsilon: np.ndarray             # (n,) kJ/mol
    is_ligand: np.ndarray           # (n,) uint8
    excl: np.ndarray                # (m,2) int32, i<j, unique
    bonds: np.ndarray               # (b,2) int32
    bond_r0: np.ndarray             # (b,) nm
    bond_k: np.ndarray              # (b,) kJ/mol/nm^2
    boresch: Optional[Boresch] = None
    info: dict = field(default_factory=dict)
    # periodic torsions of rotatable ligand bonds: atoms (a, b, c, d) about b-c,
    # force constant k (kJ/mol), periodicity n, phase phi0 (rad)
    torsions: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.int32))
    torsion_k: np.ndarray = field(default_factory=lambda: np.zeros(0))
    torsion_n: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    torsion_phi0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    # alchemical waters: oxygen indices and the charge each takes up when the
    # ligand's charges are off (their charge is q0 + (1 - lambda_q) dq)
    alch_water: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    alch_water_dq: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_ligand(self) -> int:
        return int(self.is_ligand.sum())

    def copy(self) -> "System":
        import copy as _c
        return _c.deepcopy(self)

    def save(self, path: str) -> None:
        d = {k: getattr(self, k) for k in ("box", "pos", "vel", "mass", "charge", "sigma",
                                           "epsilon", "is_ligand", "excl", "bonds",
                                           "bond_r0", "bond_k")}
        d["name"] = np.array(self.name)
        if self.boresch is not None:
            b = self.boresch
            d["b_anchors"] = b.anchors
            d["b_vals"] = np.array([b.r0, *b.theta0, *b.phi0, b.k_r, b.k_theta, b.k_phi])
        np.savez_compressed(path, **d)

    @staticmethod
    def load(path: str) -> "System":
        z = np.load(path)
        bor = None
        if "b_anchors" in z:
            v = z["b_vals"]
            bor = Boresch(z["b_anchors"].astype(np.int32), float(v[0]), v[1:3].copy(),
                          v[3:6].copy(), float(v[6]), float(v[7]), float(v[8]))
        return System(str(z["name"]), z["box"], z["pos"], z["vel"], z["mass"], z["charge"],
                      z["sigma"], z["epsilon"], z["is_ligand"], z["excl"], z["bonds"],
                      z["bond_r0"], z["bond_k"], bor)


# ----------------------------------------------------------------------------- helpers

def _rand_rot(rng, n):
    """n uniformly random rotation matrices (from random unit quaternions)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def _water_template():
    h = np.deg2rad(WATER_HOH_DEG) / 2
    return np.array([[0.0, 0.0, 0.0],
                     [WATER_ROH * np.sin(h), WATER_ROH * np.cos(h), 0.0],
                     [-WATER_ROH * np.sin(h), WATER_ROH * np.cos(h), 0.0]])


def _waters_at(rng, sites):
    """Three atoms per site: O at the site, two H in a random orientation."""
    rot = _rand_rot(rng, len(sites))
    t = _water_template()
    return sites[:, None, :] + np.einsum("nij,aj->nai", rot, t)


def _lattice(box, n_side, offset=0.5):
    g = [(np.arange(n_side[d]) + offset) * (box[d] / n_side[d]) for d in range(3)]
    return np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)


def _unit(v):
    return v / np.linalg.norm(v)


def _random_unit(rng):
    return _unit(rng.normal(size=3))


def _grow_chain(rng, n, start, step_lo, step_hi, max_turn_deg, avoid_tree, box,
                clearance, self_min, tries=400, first_dir=None):
    """Self-avoiding chain of n atoms; returns (n,3) or None.

    Consecutive atoms are step_lo..step_hi apart; each new bond turns by at most
    max_turn_deg from the previous one; every atom stays `clearance` away from the
    points in `avoid_tree` (periodic) and `self_min` away from chain atoms three or
    more bonds back.
    """
    pts = [np.asarray(start, float)]
    d_prev = _unit(first_dir) if first_dir is not None else _random_unit(rng)
    cos_max = np.cos(np.deg2rad(max_turn_deg))
    while len(pts) < n:
        ok = False
        for _ in range(tries):
            d = _random_unit(rng)
            if len(pts) > 1 and np.dot(d, d_prev) < cos_max:
                continue
            if len(pts) == 1 and first_dir is not None and np.dot(d, d_prev) < cos_max:
                continue
            p = pts[-1] + rng.uniform(step_lo, step_hi) * d
            if avoid_tree is not None:
                if avoid_tree.query_ball_point(np.mod(p, box), clearance, return_length=True) > 0:
                    continue
            if len(pts) >= 3:
                far = np.asarray(pts[:-2])
                if np.min(np.linalg.norm(far - p, axis=1)) < self_min:
                    continue
            pts.append(p)
            d_prev = d
            ok = True
            break
        if not ok:
            return None
    return np.asarray(pts)


def _chain_angle_bonds(xyz, offset):
    """Harmonic 1-3 bonds (Urey-Bradley form) at the chain's own 1-3 distances:
    they hold each bond angle near its starting value. An angle that starts at
    <= 135 degrees (the only ones a torsion spans, see ligand_torsions) is
    >= 52 kJ/mol away from 180 degrees, where a torsion's gradient diverges.
    The pairs are already excluded (1-3)."""
    j = np.arange(len(xyz) - 2)
    r0 = np.linalg.norm(xyz[2:] - xyz[:-2], axis=1)
    return (np.stack([j, j + 2], 1) + offset).astype(np.int32), r0


def _chain_topology(n_lig, offset):
    """1-2 bonds along the chain; exclusions are 1-2 and 1-3 pairs."""
    i = np.arange(n_lig - 1)
    bonds = np.stack([i, i + 1], 1) + offset
    j = np.arange(n_lig - 2)
    ex = np.concatenate([bonds, np.stack([j, j + 2], 1) + offset])
    return bonds.astype(np.int32), ex.astype(np.int32)


def ligand_torsions(ligand, offset, p_rotatable=0.5):
    """Periodic torsions of the chain's rotatable bonds: each internal bond
    (j, j+1) with neighbours on both sides and both bond angles (at j and j+1)
    at most 135 degrees is rotatable with probability p_rotatable and then
    carries one term on the quadruple (j-1, j, j+1, j+2) with k in U[1, 8]
    kJ/mol, n in {1, 2, 3} and phi0 in {0, pi}. (The chain's 1-3 bonds keep
    those angles away from 180 degrees, where the torsion's gradient diverges.)
    The draws come from a generator seeded by the ligand's own coordinates, so
    the rest of the system's random stream is unchanged and both legs of a
    ligand get the same terms. Returns (idx [m][4], k, n, phi0)."""
    xyz = np.asarray(ligand["xyz"], dtype=np.float64)
    n_lig = len(xyz)
    rng = np.random.default_rng(int(np.abs(xyz).sum() * 1.0e6) % (2 ** 32))
    b1 = xyz[:-2] - xyz[1:-1]
    b2 = xyz[2:] - xyz[1:-1]
    cos_a = (b1 * b2).sum(1) / (np.linalg.norm(b1, axis=1) * np.linalg.norm(b2, axis=1))
    bent = np.r_[False, cos_a >= np.cos(np.deg2rad(135.0)), False]   # per atom
    j = np.arange(1, n_lig - 2)
    pick = rng.uniform(size=len(j)) < p_rotatable
    rot = j[pick & bent[j] & bent[j + 1]]
    idx = (np.stack([rot - 1, rot, rot + 1, rot + 2], 1) + offset).astype(np.int32)
    k = f32(rng.uniform(1.0, 8.0, len(rot)))
    n = rng.integers(1, 4, len(rot)).astype(np.int32)
    phi0 = f32(np.where(rng.uniform(size=len(rot)) < 0.5, 0.0, np.pi))
    return idx.reshape(-1, 4), k, n, phi0


def _water_topology(n_water, offset):
    base = offset + 3 * np.arange(n_water)
    bonds = np.concatenate([np.stack([base, base + 1], 1), np.stack([base, base + 2], 1),
                            np.stack([base + 1, base + 2], 1)])
    r0 = np.concatenate([np.full(n_water, WATER_ROH), np.full(n_water, WATER_ROH),
                         np.full(n_water, 2 * WATER_ROH * np.sin(np.deg2rad(WATER_HOH_DEG) / 2))])
    k = np.concatenate([np.full(2 * n_water, K_WATER_OH), np.full(n_water, K_WATER_HH)])
    return bonds.astype(np.int32), r0, k


def _ligand_params(rng, n_lig, q_sd=0.3, strong=0):
    q = rng.normal(0.0, q_sd, n_lig)
    q -= q.mean()
    if strong:
        # `strong` atoms carry alternating +-2 e; the rest are re-neutralised.
        idx = rng.choice(n_lig, size=strong, replace=False)
        q[idx] = np.where(np.arange(strong) % 2 == 0, 2.0, -2.0)
        rest = np.setdiff1d(np.arange(n_lig), idx)
        q[rest] -= q.sum() / len(rest)
    sig = rng.uniform(0.25, 0.40, n_lig)
    eps = rng.uniform(0.2, 1.0, n_lig)
    return q, sig, eps


def _maxwell(rng, mass, kT):
    v = rng.normal(size=(len(mass), 3)) * np.sqrt(kT / mass)[:, None]
    v -= (mass[:, None] * v).sum(0) / mass.sum()
    return v


def _unique_pairs(p):
    p = np.sort(np.asarray(p, dtype=np.int64), axis=1)
    p = np.unique(p, axis=0)
    return p.astype(np.int32)


def _assemble(name, box, parts, excl, bonds, bond_r0, bond_k, boresch, rng, T, info):
    pos = np.concatenate([p["pos"] for p in parts])
    box = f32(box)
    pos = f32(np.mod(pos, box))
    pos = np.where(pos >= box, 0.0, pos)
    mass = np.concatenate([p["mass"] for p in parts])
    sys = System(
        name=name, box=box, pos=pos,
        vel=f32(_maxwell(rng, mass, BOLTZMANN_KJ * T)),
        mass=f32(mass),
        charge=f32(np.concatenate([p["q"] for p in parts])),
        sigma=f32(np.concatenate([p["sig"] for p in parts])),
        epsilon=f32(np.concatenate([p["eps"] for p in parts])),
        is_ligand=np.concatenate([p["lig"] for p in parts]).astype(np.uint8),
        excl=_unique_pairs(excl),
        bonds=np.asarray(bonds, np.int32).reshape(-1, 2),
        bond_r0=f32(bond_r0), bond_k=f32(bond_k), boresch=boresch, info=info)
    return sys


# Small repulsive core on water hydrogens for MD workloads. With O-only LJ a
# flexible hydrogen feels no repulsion from any negatively charged atom and can
# collapse onto it at elevated temperature; single-frame workloads keep O-only LJ.
H_LJ_MD = (0.1, 0.1)   # sigma nm, epsilon kJ/mol


def _water_part(xyz, h_lj=(0.0, 0.0)):
    nw = xyz.shape[0]
    return dict(pos=xyz.reshape(-1, 3),
                mass=np.tile([MASS_O, MASS_H, MASS_H], nw),
                q=np.tile([WATER_Q_O, WATER_Q_H, WATER_Q_H], nw),
                sig=np.tile([WATER_SIG_O, h_lj[0], h_lj[0]], nw),
                eps=np.tile([WATER_EPS_O, h_lj[1], h_lj[1]], nw),
                lig=np.zeros(3 * nw, np.uint8))


# ----------------------------------------------------------------------------- systems

def tiny(seed: int = 1235) -> System:
    """Tiny oracle case: 216 waters on a 6^3 lattice in a 1.86 nm box plus a
    24-atom chain solute at the centre (672 atoms, one frame).

    The chain is grown with 0.10-0.15 nm steps between the waters; seeds are
    drawn until every solute atom is at least 0.15 nm from every water atom.
    """
    box = f32(np.full(3, 1.86))
    for attempt in range(200):
        rng = np.random.default_rng(seed * 1000 + attempt)
        sites = _lattice(box, (6, 6, 6)) + rng.uniform(-0.01, 0.01, (216, 3))
        wat = _waters_at(rng, sites)
        tree = cKDTree(np.mod(wat.reshape(-1, 3), box), boxsize=box)
        chain = _grow_chain(rng, 24, box / 2 + rng.uniform(-0.05, 0.05, 3), 0.10, 0.15, 75.0,
                            tree, box, 0.15, 0.20, tries=600)
        if chain is not None:
            break
    else:  # pragma: no cover
        raise RuntimeError("tiny(): no clash-free chain found")
    dmin = float(tree.query(np.mod(chain, box))[0].min())
    q, sig, eps = _ligand_params(rng, 24)
    lig = dict(pos=chain, mass=np.full(24, MASS_C), q=q, sig=sig, eps=eps,
               lig=np.ones(24, np.uint8))
    wb, wr0, wk = _water_topology(216, 0)
    lb, lex = _chain_topology(24, 648)
    lr0 = np.linalg.norm(chain[1:] - chain[:-1], axis=1)
    return _assemble("tiny-672", box, [_water_part(wat), lig],
                     np.concatenate([wb, lex]), np.concatenate([wb, lb]),
                     np.concatenate([wr0, lr0]),
                     np.concatenate([wk, np.full(23, K_LIGAND)]),
                     None, rng, 300.0, dict(min_solute_water=dmin, seed=seed))


def make_ligand(rng, n_lig, q_sd=0.3, strong=0, tries=200):
    """A ligand-like chain in vacuum: 0.15 nm bonds, bond angles >= 110 degrees,
    atoms three or more bonds apart kept >= 0.30 nm apart."""
    for _ in range(tries):
        c = _grow_chain(rng, n_lig, np.zeros(3), 0.15, 0.15, 70.0, None, None, 0.0, 0.30)
        if c is not None:
            break
    else:  # pragma: no cover
        raise RuntimeError("make_ligand(): growth failed")
    c -= c[0]
    q, sig, eps = _ligand_params(rng, n_lig, q_sd, strong)
    return dict(xyz=c, q=q, sig=sig, eps=eps)


def _fill_water(rng, box, solute_xyz, n_target_atoms, clear_o=0.28, clear_h=0.20):
    """Waters on a jittered lattice, removing those that clash with the solute,
    then dropping random waters until the atom count is reached."""
    solute_xyz = np.mod(solute_xyz, box)
    tree = cKDTree(solute_xyz, boxsize=box) if len(solute_xyz) else None
    need = (n_target_atoms - len(solute_xyz))
    if need % 3:
        raise ValueError("target atom count minus solute must be a multiple of 3")
    need //= 3
    spacing = (1.0 / 33.4) ** (1 / 3)
    n_side = np.maximum(1, np.round(box / spacing).astype(int))
    for grow in range(12):
        ns = n_side + grow
        sites = _lattice(box, ns)
        sites = sites + rng.uniform(-0.02, 0.02, sites.shape)
        wat = _waters_at(rng, sites)
        if tree is not None:
            o_ok = tree.query_ball_point(np.mod(wat[:, 0], box), clear_o, return_length=True) == 0
            h_ok = np.ones(len(wat), bool)
            for a in (1, 2):
                h_ok &= tree.query_ball_point(np.mod(wat[:, a], box), clear_h,
                                              return_length=True) == 0
            wat = wat[o_ok & h_ok]
        if len(wat) >= need:
            keep = np.sort(rng.choice(len(wat), size=need, replace=False))
            return wat[keep]
    raise RuntimeError("could not place enough waters")


def complex_leg(seed: int, n_atoms: int = 60000, box: Optional[float] = None,
                core_diameter: float = 4.5, n_types: int = 14, n_lig: int = 60,
                ligand: Optional[dict] = None, k_r: float = 4184.0, k_ang: float = 41.84,
                r0: float = 0.6, strong_ligand_charges: int = 0, T: float = 300.0,
                core_density: float = 110.0, h_lj=H_LJ_MD) -> System:
    """Protein-ligand leg: dense core sphere + ligand at its surface + water.

    The core is a jittered cubic lattice (about `core_density` atoms/nm^3) inside
    a sphere; core atoms closer than 0.32 nm are bonded (elastic network) and
    those bonded pairs are the core's exclusions. The ligand chain starts 0.4 nm
    outside the core surface; Boresch anchors are L1..L3 = ligand atoms 0..2,
    P1 = the core atom whose distance to L1 is closest to r0, P2 and P3 = core
    atoms about 0.3 nm further into the core; reference angles and dihedrals
    are drawn (U[80,100] degrees and U[-180,180] degrees).
    """
    rng = np.random.default_rng(seed)
    if box is None:
        box = (n_atoms / 100.0) ** (1 / 3)
    box = f32(np.full(3, box))
    centre = box / 2
    # --- core
    a = (1.0 / core_density) ** (1 / 3)
    R = core_diameter / 2
    m = int(np.ceil(R / a)) + 1
    g = np.arange(-m, m + 1) * a
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    grid = grid[np.linalg.norm(grid, axis=1) <= R]
    core = centre + grid + rng.uniform(-0.01, 0.01, grid.shape)
    n_core = len(core)
    # core types: sigma in [0.25, 0.39] nm and charges within +-0.8 e, the
    # ligand's ranges. Smaller, more charged atoms let a water H (sigma 0.1 nm)
    # fall into a -500..-900 kJ/mol well at ~0.1 nm; the heat that releases
    # blew windows up in long MD runs.
    t_sig = 0.25 + (rng.uniform(0.20, 0.39, n_types) - 0.20) * (0.14 / 0.19)
    t_eps = rng.uniform(0.1, 1.0, n_types)
    t_mass = rng.choice([12.011, 14.007, 15.999, 32.06], n_types)
    ctype = rng.integers(0, n_types, n_core)
    cq = np.clip(rng.normal(0.0, 0.4, n_core), -0.8, 0.8)
    cq -= cq.mean()
    # --- ligand
    if ligand is None:
        ligand = make_ligand(rng, n_lig, strong=strong_ligand_charges)
    n_lig = len(ligand["q"])
    ctree = cKDTree(core)
    placed = None
    for _ in range(2000):
        u = _random_unit(rng)
        start = centre + u * (R + 0.4)
        rot = _rand_rot(rng, 1)[0]
        xyz = ligand["xyz"] @ rot.T
        # bias the chain to point away from the core
        if np.dot(xyz[-1] - xyz[0], u) < 0:
            xyz = -xyz
        xyz = xyz + start
        if ctree.query(xyz)[0].min() >= 0.30:
            placed = xyz
            break
    if placed is None:  # pragma: no cover
        raise RuntimeError("complex_leg(): could not place ligand")
    # --- total count: core + ligand + 3*waters == n_atoms (drop core atoms if needed)
    extra = (3 - (n_atoms - n_core - n_lig) % 3) % 3
    if extra:
        far = np.argsort(np.linalg.norm(core - centre, axis=1))[::-1][:extra]
        keep = np.setdiff1d(np.arange(n_core), far)
        core, ctype, cq = core[keep], ctype[keep], cq[keep]
        cq -= cq.mean()
        n_core = len(core)
    wat = _fill_water(rng, box, np.concatenate([core, placed]), n_atoms)
    nw = len(wat)
    # --- topology
    ctree = cKDTree(core)
    cb = np.array(sorted(ctree.query_pairs(0.32)), dtype=np.int64).reshape(-1, 2)
    cb_r0 = np.linalg.norm(core[cb[:, 0]] - core[cb[:, 1]], axis=1)
    off_lig = n_core
    off_w = n_core + n_lig
    lb, lex = _chain_topology(n_lig, off_lig)
    lr0 = np.linalg.norm(placed[1:] - placed[:-1], axis=1)
    ab, ar0 = _chain_angle_bonds(placed, off_lig)
    wb, wr0, wk = _water_topology(nw, off_w)
    # --- Boresch anchors
    L1 = placed[0]
    dist = np.linalg.norm(core - L1, axis=1)
    p1 = int(np.argmin(np.abs(dist - r0)))
    inward = _unit(centre - core[p1])
    p2 = int(np.argmin(np.linalg.norm(core - (core[p1] + 0.3 * inward), axis=1)))
    side = _unit(np.cross(inward, _random_unit(rng)))
    p3 = int(np.argmin(np.linalg.norm(core - (core[p2] + 0.3 * side), axis=1)))
    if len({p1, p2, p3}) < 3:  # pragma: no cover
        raise RuntimeError("degenerate protein anchors")
    bor = Boresch(np.array([p1, p2, p3, off_lig, off_lig + 1, off_lig + 2], np.int32),
                  float(f32(r0)), f32(np.deg2rad(rng.uniform(80, 100, 2))),
                  f32(np.deg2rad(rng.uniform(-180, 180, 3))),
                  float(f32(k_r)), float(f32(k_ang)), float(f32(k_ang)))
    parts = [dict(pos=core, mass=t_mass[ctype], q=cq, sig=t_sig[ctype], eps=t_eps[ctype],
                  lig=np.zeros(n_core, np.uint8)),
             dict(pos=placed, mass=np.full(n_lig, MASS_C), q=ligand["q"], sig=ligand["sig"],
                  eps=ligand["eps"], lig=np.ones(n_lig, np.uint8)),
             _water_part(wat, h_lj)]
    excl = np.concatenate([cb, lex, wb])
    bonds = np.concatenate([cb, lb, ab, wb])
    r0s = np.concatenate([cb_r0, lr0, ar0, wr0])
    ks = np.concatenate([np.full(len(cb), K_CORE), np.full(len(lb), K_LIGAND),
                         np.full(len(ab), K_LIGAND_13), wk])
    sys = _assemble(f"complex-{n_atoms}", box, parts, excl, bonds, r0s, ks, bor, rng, T,
                    dict(seed=seed, n_core=n_core, n_lig=n_lig, n_water=nw))
    sys.torsions, sys.torsion_k, sys.torsion_n, sys.torsion_phi0 = ligand_torsions(ligand, off_lig)
    return sys


def solvent_leg(seed: int, ligand: Optional[dict] = None, n_lig: int = 60, box: float = 3.5,
                n_atoms: Optional[int] = None, T: float = 300.0, h_lj=H_LJ_MD) -> System:
    """Ligand-solvent leg: the ligand at the box centre surrounded by water."""
    rng = np.random.default_rng(seed)
    box = f32(np.full(3, box))
    if ligand is None:
        ligand = make_ligand(rng, n_lig)
    n_lig = len(ligand["q"])
    xyz = ligand["xyz"] - ligand["xyz"].mean(0) + box / 2
    if n_atoms is None:
        n_atoms = int(round(box[0] ** 3 * 105.0))
    n_atoms -= (n_atoms - n_lig) % 3
    wat = _fill_water(rng, box, xyz, n_atoms)
    nw = len(wat)
    lb, lex = _chain_topology(n_lig, 0)
    lr0 = np.linalg.norm(xyz[1:] - xyz[:-1], axis=1)
    ab, ar0 = _chain_angle_bonds(xyz, 0)
    wb, wr0, wk = _water_topology(nw, n_lig)
    parts = [dict(pos=xyz, mass=np.full(n_lig, MASS_C), q=ligand["q"], sig=ligand["sig"],
                  eps=ligand["eps"], lig=np.ones(n_lig, np.uint8)), _water_part(wat, h_lj)]
    sys = _assemble(f"solvent-{n_atoms}", box, parts, np.concatenate([lex, wb]),
                    np.concatenate([lb, ab, wb]), np.concatenate([lr0, ar0, wr0]),
                    np.concatenate([np.full(len(lb), K_LIGAND), np.full(len(ab), K_LIGAND_13),
                                    wk]), None, rng, T,
                    dict(seed=seed, n_lig=n_lig, n_water=nw))
    sys.torsions, sys.torsion_k, sys.torsion_n, sys.torsion_phi0 = ligand_torsions(ligand, 0)
    return sys


def charged_leg(s: System, q_net: float, lo: float = -0.4, hi: float = 0.6) -> System:
    """A copy of a ligand leg whose ligand carries net charge q_net, kept neutral
    in the physical state by a counterion, with alchemical waters for the
    alchemical path.

    The ligand's charges are shifted evenly so that they sum to q_net; the water
    farthest from the ligand's centroid becomes the counterion (its oxygen
    carries -q_net with sigma 0.44 nm, epsilon 0.42 kJ/mol; its hydrogens no
    charge); the n waters next-farthest become alchemical waters, n the smallest
    count with q_net / n in [lo, hi], each taking up dq = q_net / n."""
    t = s.copy()
    lig = np.where(t.is_ligand.astype(bool))[0]
    t.charge = t.charge.copy()
    t.charge[lig] += (q_net - t.charge[lig].sum()) / len(lig)
    n = 0
    if abs(q_net) > 1e-12:
        n = 1
        while not (lo - 1e-12 <= q_net / n <= hi + 1e-12):
            n += 1
    cen = t.pos[lig].mean(0)
    oxy = np.where((t.is_ligand == 0) & (np.abs(t.charge - WATER_Q_O) < 1e-6))[0]
    d = t.pos[oxy] - cen
    d -= t.box * np.round(d / t.box)
    far = oxy[np.argsort(-np.linalg.norm(d, axis=1))]
    ion = far[0]
    t.charge[ion] = -q_net
    t.charge[ion + 1] = 0.0
    t.charge[ion + 2] = 0.0
    t.sigma = t.sigma.copy()
    t.epsilon = t.epsilon.copy()
    t.sigma[ion], t.epsilon[ion] = 0.44, 0.42
    t.charge, t.sigma, t.epsilon = f32(t.charge), f32(t.sigma), f32(t.epsilon)
    t.alch_water = np.sort(far[1:1 + n]).astype(np.int32)
    t.alch_water_dq = f32(np.full(n, q_net / n if n else 0.0))
    t.name = s.name + f"-q{q_net:+g}"
    return t


def water_box(seed: int, box: float, n_atoms: Optional[int] = None, T: float = 300.0,
              h_lj=H_LJ_MD) -> System:
    """Pure water-like solvent (used by the list-builder and integrator tests)."""
    rng = np.random.default_rng(seed)
    box = f32(np.full(3, box))
    if n_atoms is None:
        n_atoms = 3 * int(round(box[0] ** 3 * 33.4))
    wat = _fill_water(rng, box, np.zeros((0, 3)), n_atoms)
    wb, wr0, wk = _water_topology(len(wat), 0)
    return _assemble(f"water-{n_atoms}", box, [_water_part(wat, h_lj)], wb, wb, wr0, wk, None, rng,
                     T, dict(seed=seed))


# ----------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    """A set of distinct systems and the replicas (lambda windows) that use them."""
    name: str
    systems: list
    system_of_replica: np.ndarray     # (R,) int32
    schedules: list                   # LambdaSchedule per schedule id
    schedule_of_replica: np.ndarray   # (R,) int32
    state_of_replica: np.ndarray      # (R,) int32
    params: dict

    @property
    def n_replicas(self) -> int:
        return int(len(self.system_of_replica))

    @property
    def total_atoms(self) -> int:
        return int(sum(self.systems[s].n for s in self.system_of_replica))


BASE_SEED = 1234


def params_for(cutoff, beta, T=300.0, skin=0.1, ligand_mode=0):
    return dict(cutoff=cutoff, ewald_beta=beta, sc_alpha=0.5, sc_p=1.0, coulomb_k=COULOMB_K,
                kT=BOLTZMANN_KJ * T, skin=skin, ligand_mode=ligand_mode, T=T)


def workload_tiny() -> Workload:
    """One frame of the 672-atom tiny system at all 12 states (cutoff 0.9 nm, beta 3.47)."""
    s = tiny(BASE_SEED + 1)
    sch = schedule_k12()
    K = sch.K
    return Workload("tiny-672-K12", [s], np.zeros(K, np.int32), [sch], np.zeros(K, np.int32),
                    np.arange(K, dtype=np.int32), params_for(0.9, 3.47, skin=0.0))


def workload_complex60k(n_replicas: int = 1) -> Workload:
    """The 60,000-atom complex-leg window (8.5 nm box, 60-atom ligand, K=42)."""
    s = complex_leg(BASE_SEED + 2, n_atoms=60000, box=8.5, n_lig=60)
    sch = schedule_k42()
    st = np.arange(n_replicas, dtype=np.int32) % sch.K
    return Workload("complex-60k-K42", [s], np.zeros(n_replicas, np.int32), [sch],
                    np.zeros(n_replicas, np.int32), st, params_for(1.0, 3.12))


def workload_batch(n_ligands: int = 16, complex_range=(40000, 80000), solvent_box=3.5,
                   solvent_atoms: int = 4500) -> Workload:
    """16 ligands x (complex leg, 42 windows + solvent leg, 30 windows) = 1,152 replicas."""
    rng = np.random.default_rng(BASE_SEED + 3)
    systems, sys_of, sch_of, st_of = [], [], [], []
    s42, s30 = schedule_k42(), schedule_solvent_k30()
    for li in range(n_ligands):
        n_lig = int(rng.integers(30, 91))
        lig = make_ligand(np.random.default_rng(BASE_SEED + 3 + 1000 * (li + 1)), n_lig)
        n_c = int(rng.integers(complex_range[0], complex_range[1] + 1))
        systems.append(complex_leg(BASE_SEED + 3 + 1000 * (li + 1) + 1, n_atoms=n_c,
                                   ligand=lig))
        systems.append(solvent_leg(BASE_SEED + 3 + 1000 * (li + 1) + 2, ligand=lig,
                                   box=solvent_box, n_atoms=solvent_atoms))
        ci, si = len(systems) - 2, len(systems) - 1
        sys_of += [ci] * s42.K + [si] * s30.K
        sch_of += [0] * s42.K + [1] * s30.K
        st_of += list(range(s42.K)) + list(range(s30.K))
    return Workload(f"batch-{len(sys_of)}", systems, np.array(sys_of, np.int32), [s42, s30],
                    np.array(sch_of, np.int32), np.array(st_of, np.int32),
                    params_for(1.0, 3.12))


def workload_loop() -> Workload:
    """24 replicas of a 25k-atom complex-shaped system (20-atom ligand, cutoff 0.9 nm, K=24)."""
    s = complex_leg(BASE_SEED + 4, n_atoms=25000, core_diameter=3.5, n_lig=20)
    sch = schedule_k24()
    return Workload("loop-25k-x24-K24", [s], np.zeros(24, np.int32), [sch],
                    np.zeros(24, np.int32), np.arange(24, dtype=np.int32),
                    params_for(0.9, 3.47))


def workload_precision() -> Workload:
    """100,000 atoms in a 10 nm box, 90-atom ligand with four +-2 e atoms,
    cutoff 1.2 nm, beta 2.6, K=42."""
    s = complex_leg(BASE_SEED + 5, n_atoms=100000, box=10.0, n_lig=90, strong_ligand_charges=4)
    sch = schedule_k42()
    return Workload("precision-100k-K42", [s], np.zeros(1, np.int32), [sch],
                    np.zeros(1, np.int32), np.zeros(1, np.int32), params_for(1.2, 2.6))
