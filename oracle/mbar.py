"""FP64 reference estimators for the u_kn rows (TEST INFRASTRUCTURE).

The paper estimates each GPU segment's free energy with MBAR and sums the
segments ("Simulation protocol"), using BAR and FEP as diagnostics. Written
from the estimators' definitions:

* MBAR (Shirts & Chodera 2008): dimensionless free energies f_i solve
  f_i = -ln sum_n exp(-u_i(x_n)) / sum_k N_k exp(f_k - u_k(x_n)),
  with f_0 = 0; solved here by plain self-consistent iteration in log space.
* BAR (Bennett 1976): for two states with forward work w_F = u_1 - u_0 on
  samples of state 0 and reverse work w_R = u_0 - u_1 on samples of state 1,
  Delta f solves sum_F 1/(1 + exp(ln(N_F/N_R) + w_F - Delta f))
  = sum_R 1/(1 + exp(ln(N_R/N_F) + w_R + Delta f)); solved by bisection.
"""
from __future__ import annotations

import numpy as np


def _logsumexp(a, axis):
    m = np.max(a, axis=axis, keepdims=True)
    return (m + np.log(np.sum(np.exp(a - m), axis=axis, keepdims=True))).squeeze(axis)


def mbar(u_kn, N_k, tol=1e-12, max_iter=100000):
    """u_kn: (K, N) reduced potentials of every sample at every state; samples
    are ordered by the state they were drawn from (N_k of each). Returns f_k
    (f_0 = 0) and the number of iterations."""
    u = np.asarray(u_kn, dtype=np.float64)
    N_k = np.asarray(N_k, dtype=np.float64)
    K, N = u.shape
    assert N_k.sum() == N
    logN = np.log(np.where(N_k > 0, N_k, 1.0))
    has = N_k > 0
    f = np.zeros(K)
    for it in range(1, max_iter + 1):
        # log denominator of every sample: ln sum_k N_k exp(f_k - u_kn), sampled states only
        ld = _logsumexp((logN + f)[has, None] - u[has], axis=0)
        fn = -_logsumexp(-u - ld[None, :], axis=1)
        fn -= fn[0]
        if np.max(np.abs(fn - f)) < tol:
            return fn, it
        f = fn
    return f, max_iter


def bar(w_F, w_R, tol=1e-13):
    """Delta f (state 1 minus state 0) from forward and reverse reduced works."""
    w_F = np.asarray(w_F, dtype=np.float64)
    w_R = np.asarray(w_R, dtype=np.float64)
    M = np.log(len(w_F) / len(w_R))

    def g(df):
        a = np.sum(1.0 / (1.0 + np.exp(M + w_F - df)))
        b = np.sum(1.0 / (1.0 + np.exp(-M + w_R + df)))
        return a - b

    lo, hi = -1.0, 1.0
    while g(lo) > 0:
        lo *= 2
    while g(hi) < 0:
        hi *= 2
    while hi - lo > tol * max(1.0, abs(lo)):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
