"""Reference replica exchange of lambda states (TEST INFRASTRUCTURE).

The paper runs replica exchange among the windows that one GPU hosts and never
across GPUs ("Simulation protocol"). This restates the neighbour-swap scheme of
Hamiltonian replica exchange: replicas exchange their states (coordinates stay
put); a swap of replica i (state a) and replica j (state b) is accepted with
the Metropolis probability min(1, exp(-D)),
    D = [u_b(x_i) + u_a(x_j)] - [u_a(x_i) + u_b(x_j)],
which keeps the joint distribution prod_r exp(-u_{s(r)}(x_r)) stationary.
Attempt t pairs neighbouring states of every group - the group's states in
ascending order at positions (m, m+1), m = t mod 2, t mod 2 + 2, ... A group is
the replicas sharing a system and a schedule.

Random numbers come from the oracle's own Philox4x32-10 (the C oracle, pinned
to the published known-answer vectors): counter (t lo, t hi, group, m), key
(seed lo, seed hi); U = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53 and the swap is
taken iff D <= 0 or ln U < -D (FP64, the same decision precision as the device).
"""
from __future__ import annotations

import math

import numpy as np

from . import philox4x32_10


def exchange_groups(system_of_replica, schedule_of_replica):
    """Groups in order of first appearance: lists of replica indices."""
    keys, groups = [], []
    for r, k in enumerate(zip(system_of_replica, schedule_of_replica)):
        k = (int(k[0]), int(k[1]))
        if k not in keys:
            keys.append(k)
            groups.append([])
        groups[keys.index(k)].append(r)
    return groups


def uniform53(x0, x1):
    return ((int(x0) >> 5) * 67108864 + (int(x1) >> 6) + 0.5) * 2.0 ** -53


def attempt(ukn, states, groups, seed, t):
    """One attempt. ukn: [R][>=K] reduced potentials u_k(x_r); states: [R].
    Returns (new states, number of accepted swaps)."""
    st = np.array(states, dtype=np.int64).copy()
    acc = 0
    for g, members in enumerate(groups):
        order = sorted(members, key=lambda r: (st[r], r))
        held = [int(st[r]) for r in order]
        if len(set(held)) != len(held):
            raise ValueError("a group holds a state twice")
        m = t & 1
        while m + 1 < len(order):
            ri, rj = order[m], order[m + 1]
            a, b = held[m], held[m + 1]
            d = (ukn[ri][b] + ukn[rj][a]) - (ukn[ri][a] + ukn[rj][b])
            x = philox4x32_10([t & 0xFFFFFFFF, (t >> 32) & 0xFFFFFFFF, g, m],
                              [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
            u = uniform53(x[0], x[1])
            if d <= 0.0 or math.log(u) < -d:
                st[ri], st[rj] = b, a
                acc += 1
            m += 2
    return st, acc
