"""Alchemical lambda schedules (inputs to both the oracle and the CUDA path).

A schedule is K states, each a triple (lambda_r, lambda_q, lambda_v):

* lambda_r scales the Boresch restraint (0 = off, 1 = fully on);
* lambda_q scales the ligand partial charges (1 = physical, 0 = none);
* lambda_v is the softcore vdW coupling of ligand pairs (1 = physical).

The path runs from the physical bound state to the decoupled one in three
stages that share their end points (paper, appendix "Additional methodological
details", and the window counts of section "Simulation protocol"):
restraint on (lambda_r 0 -> 1), then charges off (lambda_q 1 -> 0), then vdW
off (lambda_v 1 -> 0). The paper prints each list in ascending order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# The paper's universal schedules, as printed (ascending).
PAPER_CHARGE = [0.00, 0.05, 0.10, 0.15, 0.20, 0.25, 0.30, 0.35, 0.40, 0.44, 0.48, 0.52, 0.56,
                0.60, 0.64, 0.68, 0.72, 0.76, 0.80, 0.82, 0.84, 0.86, 0.88, 0.90, 0.92, 0.94,
                0.96, 0.98, 1.00]
PAPER_VDW = [0.000, 0.040, 0.080, 0.115, 0.150, 0.180, 0.210, 0.240, 0.270, 0.300, 0.330, 0.360,
             0.390, 0.420, 0.450, 0.480, 0.510, 0.540, 0.568, 0.596, 0.624, 0.650, 0.676, 0.702,
             0.728, 0.752, 0.776, 0.798, 0.820, 0.840, 0.860, 0.878, 0.894, 0.908, 0.921, 0.933,
             0.945, 0.956, 0.966, 0.975, 0.983, 0.990, 0.996, 0.999, 1.000]
PAPER_RESTRAINT = [0.00, 0.01, 0.03, 0.10, 0.30, 0.50, 0.75, 1.00]


@dataclass
class LambdaSchedule:
    name: str
    lam_r: np.ndarray
    lam_q: np.ndarray
    lam_v: np.ndarray

    @property
    def K(self) -> int:
        return int(len(self.lam_r))

    def state(self, k):
        return float(self.lam_r[k]), float(self.lam_q[k]), float(self.lam_v[k])


def staged(name, restraint=None, charge=(), vdw=()):
    """Concatenate the three stages, dropping each later stage's first point.

    `restraint` is lambda_r in path order (0 -> 1) or None for a leg without a
    restraint; `charge` and `vdw` are lambda_q and lambda_v in path order (1 -> 0).
    """
    lr, lq, lv = [], [], []
    r_end = 0.0
    if restraint is not None:
        for x in restraint:
            lr.append(x); lq.append(1.0); lv.append(1.0)
        r_end = float(restraint[-1])
    for n, x in enumerate(charge):
        if n == 0 and lr:
            continue
        lr.append(r_end); lq.append(x); lv.append(1.0)
    for n, x in enumerate(vdw):
        if n == 0 and lr:
            continue
        lr.append(r_end); lq.append(0.0); lv.append(x)
    return LambdaSchedule(name, np.array(lr), np.array(lq), np.array(lv))


def paper_complex_schedule() -> LambdaSchedule:
    """The paper's protein-ligand path: 8 + 28 + 44 = 80 windows."""
    return staged("paper-complex-80", PAPER_RESTRAINT, PAPER_CHARGE[::-1], PAPER_VDW[::-1])


def paper_solvent_schedule() -> LambdaSchedule:
    """The paper's ligand-solvent path (no restraint): 29 + 44 = 73 windows."""
    return staged("paper-solvent-73", None, PAPER_CHARGE[::-1], PAPER_VDW[::-1])


def schedule_k12() -> LambdaSchedule:
    """Charges 1 -> 0 over 5 states, then vdW 1 -> 0 over 7 more (no restraint)."""
    q = [1.0, 0.75, 0.5, 0.25, 0.0]
    v = [1.0] + [j / 7 for j in range(6, -1, -1)]
    return staged("k12", None, q, v)


def schedule_k42() -> LambdaSchedule:
    """Restraint 8 (the paper's values), charges 12, vdW 22."""
    q = [1 - j / 12 for j in range(0, 13)]
    v = [1 - j / 22 for j in range(0, 23)]
    return staged("k42", PAPER_RESTRAINT, q, v)


def schedule_solvent_k30() -> LambdaSchedule:
    """Solvent leg: charges 1 -> 0 over 10 states, then vdW over 20 more."""
    q = [1 - j / 9 for j in range(0, 10)]
    v = [1 - j / 20 for j in range(0, 21)]
    return staged("solvent-k30", None, q, v)


def schedule_k24() -> LambdaSchedule:
    """Restraint {0, .1, .5, 1}, then 8 charge and 12 vdW states."""
    q = [1 - j / 8 for j in range(0, 9)]
    v = [1 - j / 12 for j in range(0, 13)]
    return staged("k24", [0.0, 0.1, 0.5, 1.0], q, v)
