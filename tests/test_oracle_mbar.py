"""Pins of the reference estimators: exact free energies of harmonic
oscillators, MBAR = BAR for two states, invariances."""
import numpy as np
import pytest

from oracle.mbar import bar, mbar


def harmonic_samples(ks, n, seed):
    """Samples of 1D oscillators u_k(x) = k x^2 / 2 (in kT units) drawn exactly
    from each state; exact f_k - f_0 = ln(k_k / k_0) / 2."""
    rng = np.random.default_rng(seed)
    xs = np.concatenate([rng.normal(0.0, 1.0 / np.sqrt(k), n) for k in ks])
    u = 0.5 * np.asarray(ks)[:, None] * xs[None, :] ** 2
    return u, np.full(len(ks), n)


def test_mbar_harmonic_exact():
    ks = [1.0, 1.5, 2.2, 3.0, 4.5]
    u, N = harmonic_samples(ks, 20000, 1)
    f, it = mbar(u, N)
    exact = 0.5 * np.log(np.array(ks) / ks[0])
    assert np.abs(f - exact).max() < 0.02      # statistical error ~ 0.005 at this N


def test_mbar_two_states_equals_bar():
    u, N = harmonic_samples([1.0, 2.0], 5000, 2)
    f, _ = mbar(u, N)
    n = N[0]
    w_F = u[1, :n] - u[0, :n]
    w_R = u[0, n:] - u[1, n:]
    assert f[1] == pytest.approx(bar(w_F, w_R), abs=1e-9)


def test_mbar_invariances():
    u, N = harmonic_samples([1.0, 1.7, 2.9], 3000, 3)
    f, _ = mbar(u, N)
    # a per-sample constant (e.g. the lambda-independent energy) cancels
    c = np.random.default_rng(4).normal(0, 50, u.shape[1])
    f2, _ = mbar(u + c[None, :], N)
    np.testing.assert_allclose(f2, f, atol=1e-9)
    # identical states: zero free-energy differences
    f3, _ = mbar(np.vstack([u[0], u[0], u[0]]), N)
    np.testing.assert_allclose(f3, 0.0, atol=1e-12)


def test_bar_exact_for_gaussian_works():
    # shifted harmonic wells with equal curvature: Delta f = 0
    rng = np.random.default_rng(5)
    x0 = rng.normal(0, 1, 20000)
    x1 = rng.normal(1.0, 1, 20000)
    u0 = lambda x: 0.5 * x ** 2
    u1 = lambda x: 0.5 * (x - 1.0) ** 2
    df = bar(u1(x0) - u0(x0), u0(x1) - u1(x1))
    assert abs(df) < 0.03


def test_mbar_unequal_counts_and_unsampled_state():
    """Unequal N_k exercise the N_k weights; a state with no samples is still
    predicted (its exact value follows from the oscillator partition function)."""
    ks = [1.0, 2.0, 3.5, 5.0]
    counts = [30000, 8000, 0, 15000]
    rng = np.random.default_rng(6)
    xs = np.concatenate([rng.normal(0.0, 1.0 / np.sqrt(k), n) for k, n in zip(ks, counts)])
    u = 0.5 * np.asarray(ks)[:, None] * xs[None, :] ** 2
    f, _ = mbar(u, np.array(counts))
    exact = 0.5 * np.log(np.array(ks) / ks[0])
    assert np.abs(f - exact).max() < 0.03
    # dropping the weights (treating the pooled samples as equal counts) is detectably wrong
    f_bad, _ = mbar(u, np.full(4, u.shape[1] // 4) + np.array([u.shape[1] - 4 * (u.shape[1] // 4), 0, 0, 0]))
    assert np.abs(f_bad - exact).max() > 0.1
