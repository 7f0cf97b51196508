"""MBAR on the device (abfe_mbar / abfe_mbar_device) against the FP64 oracle.

Both sides iterate the same self-consistent equations to max |df| < 1e-12, so
the converged f_k agree to rounding: the test allows 1e-9 kT. Inputs are seeded
samples of harmonic oscillators (exact f known), a wide schedule whose free
energies span hundreds of kT, a state without samples and a two-state case.
"""
import numpy as np
import pytest

from oracle.mbar import mbar as mbar_oracle

pytestmark = pytest.mark.gpu


def _harmonic(ks, counts, seed, shift=0.0):
    rng = np.random.default_rng(seed)
    xs = np.concatenate([rng.normal(0.0, 1.0 / np.sqrt(k), n) for k, n in zip(ks, counts)])
    u = 0.5 * np.asarray(ks)[:, None] * xs[None, :] ** 2 + shift
    return u, np.asarray(counts)


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    return G


CASES = {
    "harmonic-5": ([1.0, 1.5, 2.2, 3.0, 4.5], [4000] * 5, 0.0),
    "unsampled": ([1.0, 2.0, 3.5, 5.0], [3000, 800, 0, 1500], 0.0),
    # stiffness spanning 1e-3 .. 1e5: f_k spans ~9 kT in ln k / 2, with large
    # per-sample constants added (cancel in MBAR)
    "wide-40": (list(np.geomspace(1e-3, 1e5, 40)), [250] * 40, 1234.5),
    "two-state": ([1.0, 2.0], [20000, 17000], 0.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mbar_matches_oracle(G, name):
    ks, counts, shift = CASES[name]
    u, N = _harmonic(ks, counts, seed=100 + list(CASES).index(name), shift=shift)
    f_ref, it_ref = mbar_oracle(u, N, tol=1e-12)
    f, it = G.mbar(u, N, tol=1e-12)
    assert np.abs(f - f_ref).max() < 1e-9, np.abs(f - f_ref).max()
    assert abs(it - it_ref) <= 2
    if name != "wide-40":   # 250 samples per state: statistical error too large there
        exact = 0.5 * np.log(np.asarray(ks) / ks[0])
        assert np.abs(f - exact).max() < 0.1


def test_mbar_device_tensor_and_large_span(G):
    import torch
    # states far apart: free energies spanning ~500 kT (shifted oscillators with
    # offsets), exercising the log-space sums
    ks = np.linspace(1.0, 3.0, 12)
    u, N = _harmonic(ks, [3000] * 12, seed=7)
    offs = np.linspace(0.0, 480.0, 12)
    u = u + offs[:, None]
    f_ref, _ = mbar_oracle(u, N, tol=1e-12)
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    f, it = G.mbar(ut, N, tol=1e-12)
    assert np.abs(f - f_ref).max() < 1e-9
    assert f[-1] > 400


def test_mbar_errors(G):
    u, N = _harmonic([1.0, 2.0], [10, 10], seed=1)
    with pytest.raises(G.AbfeError):
        G.mbar(u, np.array([10, 9]))            # counts do not sum to N
    bad = u.copy()
    bad[1, 3] = np.nan
    with pytest.raises(G.AbfeError):
        G.mbar(bad, N)
    f, it = G.mbar(u, N, tol=1e-300, max_iter=3)  # not converged: reports max_iter
    assert it == 3
