"""The autotuners (abfe_autotune, abfe_autotune_cadence) on a 6,000-atom complex
window at six states: the chosen tuning is one of the candidates, a second
context with the same key reads it back from the cache file without a new
sweep, the cadence tuner leaves the trajectory where it found it, and the
tuned contexts still match the FP64 oracle (forces, energies, dU/dlambda,
u_kn) within the tolerances of the parity tests."""
import json

import numpy as np
import pytest

import abfe_synth as S
from test_gpu_parity import check_replicas, check_ukn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    return G


@pytest.fixture(scope="module")
def mid():
    c = S.complex_leg(77, n_atoms=6000, core_diameter=2.0, n_lig=30)
    sch = S.schedule_k42()
    st = np.array([0, 5, 9, 20, 31, 41], np.int32)
    return S.Workload("mid-6000", [c], np.zeros(len(st), np.int32), [sch],
                      np.zeros(len(st), np.int32), st, S.params_for(1.0, 3.12))


KNOBS = ("group", "max_entries", "block_threads", "prune_skin")


def _valid(t):
    assert t["group"] in (1, 2, 4)
    assert t["max_entries"] in (16, 32, 64, 128, 512)
    assert t["block_threads"] in (128, 256)


def test_autotune_choice_cache_hit_and_parity(G, mid, tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    eng = G.engine_for_workload(mid)
    t1 = eng.autotune(cache, reps=1)
    _valid(t1)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["group"] == t1["group"] and rec["max_entries"] == t1["max_entries"]
    check_replicas(eng, mid, etol_mode="components")
    check_ukn(eng, mid)
    eng.close()
    # same key: the cached choice, no second sweep (no new cache line)
    eng2 = G.engine_for_workload(mid)
    t2 = eng2.autotune(cache, reps=1)
    assert {k: t2[k] for k in KNOBS if k in t2} == {k: t1[k] for k in KNOBS if k in t1}
    assert len(open(cache).read().splitlines()) == 1
    check_replicas(eng2, mid, etol_mode="components")
    eng2.close()


def test_autotune_cadence_keeps_state_and_parity(G, mid):
    eng = G.engine_for_workload(mid)
    eng.step(10, dt=0.0005, gamma=5.0, seed=2)
    x0, v0 = eng.positions(), eng.velocities()
    t = eng.autotune_cadence(dt=0.0005, gamma=5.0, seed=3, n_steps=8)
    assert 0.1 - 1e-12 <= t["skin"] <= 0.3 + 1e-12
    assert 0.0 < t["prune_skin"] <= min(t["skin"], 0.15) + 1e-12
    # the trial steps run from a saved state that is restored afterwards
    assert np.array_equal(eng.positions(), x0)
    assert np.array_equal(eng.velocities(), v0)
    # after MD the ligand-environment Coulomb sum behind dU/dlambda_q is a
    # cancellation of +-100 kJ/mol pair terms evaluated in FP32: its absolute
    # floor is the u_kn tolerance, 1e-3 kJ/mol
    check_replicas(eng, mid, etol_mode="components", dabs=1e-3)
    check_ukn(eng, mid)
    eng.step(10, dt=0.0005, gamma=5.0, seed=4)
    check_replicas(eng, mid, etol_mode="components", dabs=1e-3)
    eng.close()
