"""Reference reciprocal-space Ewald terms (TEST INFRASTRUCTURE).

The paper's electrostatics are PME with a 1.0 nm real-space cutoff
("Additional methodological details"); the real-space part is in the C oracle.
This module holds the rest of the Ewald energy, in FP64, each function from its
published definition:

* ewald_reciprocal - the plain Ewald k-space sum
      E = k_e / (2 pi V) sum_{m != 0} exp(-pi^2 |m|^2 / beta^2) / |m|^2 |S(m)|^2,
      S(m) = sum_j q_j exp(2 pi i m . r_j),  m = (n1/L1, n2/L2, n3/L3),
  with forces F_j = -dE/dr_j, over all integer |n_a| <= kmax.
* spme - smooth particle-mesh Ewald (Essmann et al. 1995): charges spread with
  cardinal B-splines M_p on a K1 x K2 x K3 grid, Q's discrete Fourier transform
  (numpy's FFT as the library step) times B(m) C(m), where
  C(m) = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2) (C(0) = 0) and
  B(m) = prod_a |b_a(m_a)|^2, |b_a(m)|^-2 = |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K_a)|^2;
  E = (k_e / 2) sum_m B C |F(Q)|^2, the potential on the grid is its derivative
  with respect to Q, and forces follow from the B-spline derivatives.
* self_energy - -k_e beta / sqrt(pi) sum_j q_j^2.
* exclusion_correction - -k_e sum over excluded pairs q_i q_j erf(beta r)/r
  (the reciprocal sum includes every pair; the real-space sum skips excluded
  ones), with its forces.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def _minimg(d, box):
    return d - box * np.round(d / box)


def ewald_reciprocal(pos, q, box, beta, kmax, ke, forces=True):
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    box = np.asarray(box, np.float64)
    V = float(np.prod(box))
    n = np.arange(-kmax, kmax + 1)
    N1, N2, N3 = np.meshgrid(n, n, n, indexing="ij")
    m = np.stack([N1.ravel() / box[0], N2.ravel() / box[1], N3.ravel() / box[2]], 1)
    m = m[np.any(np.stack([N1.ravel(), N2.ravel(), N3.ravel()], 1) != 0, axis=1)]
    m2 = (m ** 2).sum(1)
    g = np.exp(-(math.pi ** 2) * m2 / beta ** 2) / m2
    E = 0.0
    F = np.zeros_like(pos) if forces else None
    for c0 in range(0, len(m), 4096):
        mc, gc = m[c0:c0 + 4096], g[c0:c0 + 4096]
        ph = np.exp(2j * math.pi * (pos @ mc.T))        # (N, M)
        S = (q[:, None] * ph).sum(0)
        E += ke / (2 * math.pi * V) * float((gc * np.abs(S) ** 2).sum())
        if forces:
            # dE/dr_j = -(2 k_e q_j / V) sum_m g m Im(conj(S) e^{i theta_j})
            im = np.imag(np.conj(S)[None, :] * ph)       # (N, M)
            F += (2 * ke / V) * q[:, None] * ((gc[None, :] * im) @ mc)
    return E, F


def bspline(p, u):
    """Cardinal B-spline M_p(u) (support [0, p]) by the recursion
    M_n(u) = u/(n-1) M_{n-1}(u) + (n-u)/(n-1) M_{n-1}(u-1), M_2(u) = 1 - |u-1|."""
    u = np.asarray(u, np.float64)
    if p == 2:
        return np.where((u >= 0) & (u <= 2), 1.0 - np.abs(u - 1.0), 0.0)
    return (u * bspline(p - 1, u) + (p - u) * bspline(p - 1, u - 1.0)) / (p - 1)


def bspline_deriv(p, u):
    """M_p'(u) = M_{p-1}(u) - M_{p-1}(u-1)."""
    return bspline(p - 1, u) - bspline(p - 1, u - 1.0)


def bspline_moduli(p, K):
    """|b(m)|^2 for m = 0..K-1."""
    k = np.arange(p - 1)
    Mk = bspline(p, k + 1.0)
    m = np.arange(K)
    den = (Mk[None, :] * np.exp(2j * math.pi * m[:, None] * k[None, :] / K)).sum(1)
    return 1.0 / np.abs(den) ** 2


def spme(pos, q, box, beta, grid, order, ke, forces=True):
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    box = np.asarray(box, np.float64)
    K = np.asarray(grid, dtype=np.int64)
    p = int(order)
    V = float(np.prod(box))
    N = len(q)
    u = (pos / box) * K                                   # scaled fractional coordinates
    u = u - K * np.floor(u / K)
    Q = np.zeros(tuple(K))
    idx, w, dw = [], [], []
    for a in range(3):
        base = np.floor(u[:, a]).astype(np.int64)
        t = np.arange(p)
        kk = base[:, None] - t[None, :]                   # grid points whose spline covers u
        x = u[:, a][:, None] - kk                         # in [t, t+1)
        idx.append(np.mod(kk, K[a]))
        w.append(bspline(p, x))
        dw.append(bspline_deriv(p, x) * K[a] / box[a])    # d/dr of the weight
    for j in range(N):
        Q[np.ix_(idx[0][j], idx[1][j], idx[2][j])] += q[j] * np.einsum(
            "a,b,c->abc", w[0][j], w[1][j], w[2][j])
    f = [np.fft.fftfreq(int(K[a])) * K[a] / box[a] for a in range(3)]
    M1, M2, M3 = np.meshgrid(f[0], f[1], f[2], indexing="ij")
    m2 = M1 ** 2 + M2 ** 2 + M3 ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.where(m2 > 0, np.exp(-(math.pi ** 2) * m2 / beta ** 2) / (math.pi * V * m2), 0.0)
    B = np.einsum("a,b,c->abc", bspline_moduli(p, int(K[0])), bspline_moduli(p, int(K[1])),
                  bspline_moduli(p, int(K[2])))
    FQ = np.fft.fftn(Q)
    BC = B * C
    E = 0.5 * ke * float((BC * np.abs(FQ) ** 2).sum())
    if not forces:
        return E, None
    phi = ke * np.real(np.fft.ifftn(BC * FQ)) * Q.size    # dE/dQ(k)
    F = np.zeros_like(pos)
    for j in range(N):
        P = phi[np.ix_(idx[0][j], idx[1][j], idx[2][j])]
        F[j, 0] = -q[j] * np.einsum("abc,a,b,c->", P, dw[0][j], w[1][j], w[2][j])
        F[j, 1] = -q[j] * np.einsum("abc,a,b,c->", P, w[0][j], dw[1][j], w[2][j])
        F[j, 2] = -q[j] * np.einsum("abc,a,b,c->", P, w[0][j], w[1][j], dw[2][j])
    return E, F


def self_energy(q, beta, ke):
    q = np.asarray(q, np.float64)
    return -ke * beta / math.sqrt(math.pi) * float((q ** 2).sum())


def exclusion_correction(pos, q, box, excl, beta, ke, forces=True):
    """-k_e sum_{(i,j) excluded} q_i q_j erf(beta r)/r (minimum image) and forces."""
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    F = np.zeros_like(pos)
    E = 0.0
    for i, j in np.asarray(excl, dtype=np.int64).reshape(-1, 2):
        d = _minimg(pos[j] - pos[i], np.asarray(box, np.float64))
        r = float(np.sqrt((d ** 2).sum()))
        e = erf(beta * r)
        E -= ke * q[i] * q[j] * e / r
        if forces:
            # dE/dr = -k_e qq [ (2 beta / sqrt pi) exp(-beta^2 r^2) / r - erf / r^2 ]
            dEdr = -ke * q[i] * q[j] * (2 * beta / math.sqrt(math.pi) * math.exp(-(beta * r) ** 2) / r
                                        - e / r ** 2)
            F[j] -= dEdr * d / r
            F[i] += dEdr * d / r
    return E, F


def scaled_charges(s, lam_q):
    """Charges at a coupling state: ligand charges times lambda_q (Double
    annihilation protocol)."""
    q = np.asarray(s.charge, np.float64).copy()
    lig = np.asarray(s.is_ligand, bool)
    q[lig] *= lam_q
    return q
