"""Replica exchange on the device (abfe_replica_exchange) against the oracle's
neighbour-swap exchange.

Decision parity is exact: both sides get the same reduced potentials (seeded
random rows, or the oracle's own u_kn of the replicas' coordinates), draw the
same Philox uniforms and decide in FP64, so the state of every replica after
every attempt must be identical. Device-evaluated rows are checked the same
way (the oracle's exchange decides on the rows the device evaluated), by
properties (a permutation of each group's states), and by forces after an
exchange that equal those of a context set to the new states directly.
"""
import os
import tempfile

import numpy as np
import pytest

import abfe_synth as S
import oracle as O
from oracle.exchange import attempt, exchange_groups

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    O.build()
    return G


def _two_groups(seed=3):
    """12 windows of a tiny complex (schedule K=12) and 6 windows of a water box
    on another schedule: two exchange groups, states shuffled."""
    a = S.tiny(S.BASE_SEED + 1)
    b = S.water_box(21, 2.2)
    s12 = S.schedule_k12()
    s6 = S.LambdaSchedule("charge-6", np.zeros(6), np.linspace(1.0, 0.0, 6), np.ones(6))
    rng = np.random.default_rng(seed)
    st_a = rng.permutation(12)
    st_b = rng.permutation(6)
    sys_of = np.r_[np.zeros(12, np.int32), np.ones(6, np.int32)]
    sch_of = np.r_[np.zeros(12, np.int32), np.ones(6, np.int32)]
    w = S.Workload("xchg", [a, b], sys_of, [s12, s6], sch_of,
                   np.r_[st_a, st_b].astype(np.int32), S.params_for(0.9, 3.47))
    return w


def test_decisions_match_oracle_on_given_rows(G):
    w = _two_groups()
    eng = G.engine_for_workload(w)
    groups = exchange_groups(w.system_of_replica, w.schedule_of_replica)
    rng = np.random.default_rng(11)
    ld = 12
    states = w.state_of_replica.astype(np.int64)
    total = 0
    for t in range(8):
        u = rng.normal(0.0, 1.5, (w.n_replicas, ld))
        st_gpu, acc_gpu = eng.replica_exchange(seed=2024, ukn=u, ld=ld)
        states, acc_ref = attempt(u, states, groups, seed=2024, t=t)
        assert np.array_equal(st_gpu, states), t
        assert acc_gpu == acc_ref
        total += acc_ref
    assert 0 < total < 8 * 9            # a mix of accepted and rejected swaps
    assert np.array_equal(eng.replica_states(), states)
    s = eng.stats()
    assert s["n_exchange_attempts"] == 8 and s["n_exchange_accepted"] == total
    eng.close()


def test_decisions_match_oracle_on_oracle_ukn(G):
    """Rows from the oracle's FP64 u_kn of jittered copies of one system."""
    a = S.tiny(S.BASE_SEED + 1)
    sch = S.schedule_k12()
    K = sch.K
    rng = np.random.default_rng(5)
    st0 = rng.permutation(K).astype(np.int32)
    w = S.Workload("xchg1", [a], np.zeros(K, np.int32), [sch], np.zeros(K, np.int32), st0,
                   S.params_for(0.9, 3.47, skin=0.0))
    eng = G.engine_for_workload(w)
    X = np.concatenate([a.pos + rng.normal(0, 0.003, a.pos.shape) for _ in range(K)])
    eng.set_positions(X)
    rows = np.array([O.ukn(a, w.params, sch, pos=X[r * a.n:(r + 1) * a.n]) for r in range(K)])
    groups = exchange_groups(w.system_of_replica, w.schedule_of_replica)
    states = st0.astype(np.int64)
    for t in range(4):
        st_gpu, acc = eng.replica_exchange(seed=99, ukn=rows, ld=K)
        states, acc_ref = attempt(rows, states, groups, seed=99, t=t)
        assert np.array_equal(st_gpu, states) and acc == acc_ref
    eng.close()


def test_device_rows_exchange_properties_and_forces(G):
    w = _two_groups(seed=8)
    eng = G.engine_for_workload(w)
    eng.step(20, dt=0.0005, gamma=5.0, seed=3)
    groups = exchange_groups(w.system_of_replica, w.schedule_of_replica)
    states = w.state_of_replica.astype(np.int64)
    total = 0
    for t in range(6):
        st, acc, u = eng.replica_exchange(seed=5, return_ukn=True)
        assert sorted(st[:12]) == list(range(12)) and sorted(st[12:]) == list(range(6))
        # the oracle's exchange, given exactly the rows the device evaluated and
        # decided with, takes the same decisions
        states, acc_ref = attempt(u, states, groups, seed=5, t=t)
        assert np.array_equal(st, states), t
        assert acc == acc_ref
        total += acc
        eng.step(5, dt=0.0005, gamma=5.0, seed=30 + t)
    assert total > 0
    X = eng.positions()
    eng.build_list()          # both contexts then hold lists built at the same coordinates
    F1, E1, D1 = eng.compute()
    # a context given the same coordinates and the exchanged states directly
    w2 = S.Workload(w.name, w.systems, w.system_of_replica, w.schedules, w.schedule_of_replica,
                    st.astype(np.int32), w.params)
    eng2 = G.engine_for_workload(w2)
    eng2.set_positions(X)
    F2, E2, D2 = eng2.compute()
    assert np.array_equal(D1, D2) and np.array_equal(E1, E2) and np.array_equal(F1, F2)
    eng.close()
    eng2.close()


def test_exchange_checkpoint_and_errors(G):
    w = _two_groups(seed=9)
    eng = G.engine_for_workload(w)
    rng = np.random.default_rng(1)
    u = [rng.normal(0.0, 1.0, (w.n_replicas, 12)) for _ in range(4)]
    eng.replica_exchange(seed=7, ukn=u[0], ld=12)
    eng.replica_exchange(seed=7, ukn=u[1], ld=12)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "c.bin")
        eng.save_checkpoint(path)
        a1 = eng.replica_exchange(seed=7, ukn=u[2], ld=12)
        eng2 = G.engine_for_workload(w)
        eng2.load_checkpoint(path)
        a2 = eng2.replica_exchange(seed=7, ukn=u[2], ld=12)
        assert np.array_equal(a1[0], a2[0]) and a1[1] == a2[1]
        eng2.close()
    eng.close()
    # a group holding a state twice cannot exchange
    w3 = S.Workload(w.name, w.systems, w.system_of_replica, w.schedules, w.schedule_of_replica,
                    np.r_[np.zeros(12), np.arange(6)].astype(np.int32), w.params)
    eng3 = G.engine_for_workload(w3)
    with pytest.raises(G.AbfeError):
        eng3.replica_exchange(seed=1)
    eng3.close()


def _run_in_loop(G, w, graph_steps, n_chunks, every=5, seed=77, ckpt=None):
    """Relax 10 steps, then n_chunks x `every` steps with in-loop exchanges;
    returns the engine and, per chunk, (states before, rows after, states
    after, attempt index)."""
    eng = G.engine_for_workload(w)
    eng.step(10, dt=0.0005, gamma=5.0, seed=3)
    eng.set_tuning(graph_steps=graph_steps)
    eng.set_exchange(every, seed=seed)
    log = []
    for k in range(n_chunks):
        before = eng.replica_states()
        t = eng.stats()["n_exchange_attempts"]
        eng.step(every, dt=0.001, gamma=1.0, seed=100 + k)
        after = eng.replica_states()
        U, _, _ = eng.eval_ukn()
        log.append((before, U, after, t))
        if ckpt is not None and k == 1:
            eng.save_checkpoint(ckpt)
    return eng, log


def test_exchange_inside_step_loop_matches_oracle_and_direct(G):
    """Exchanges at the end of every 5th step inside abfe_step: after each
    attempt the states equal the oracle's exchange on the u_kn rows of the
    coordinates that attempt saw; a captured step graph (conditional exchange
    node) and direct launches give the same trajectory, states and counts bit
    for bit; a checkpoint between attempts resumes the same trajectory."""
    w = _two_groups(seed=4)
    groups = exchange_groups(w.system_of_replica, w.schedule_of_replica)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "x.bin")
        e1, log1 = _run_in_loop(G, w, graph_steps=0, n_chunks=4, ckpt=path)
        total = 0
        for before, U, after, t in log1:
            ref, acc = attempt(U, before.astype(np.int64), groups, seed=77, t=t)
            assert np.array_equal(after, ref), t
            total += acc
        assert total > 0
        s1 = e1.stats()
        assert s1["n_exchange_attempts"] == log1[-1][3] + 1
        assert s1["n_exchange_accepted"] == total
        x1, v1, st1 = e1.positions(), e1.velocities(), e1.replica_states()
        e1.close()
        e2, log2 = _run_in_loop(G, w, graph_steps=5, n_chunks=4)
        assert np.array_equal(e2.positions(), x1) and np.array_equal(e2.velocities(), v1)
        assert np.array_equal(e2.replica_states(), st1)
        assert e2.stats()["n_exchange_accepted"] == total
        e2.close()
        # resume from the checkpoint taken after the second chunk
        e3 = G.engine_for_workload(w)
        e3.load_checkpoint(path)
        e3.set_exchange(5, seed=77)
        for k in (2, 3):
            e3.step(5, dt=0.001, gamma=1.0, seed=100 + k)
        assert np.array_equal(e3.positions(), x1) and np.array_equal(e3.velocities(), v1)
        assert np.array_equal(e3.replica_states(), st1)
        e3.close()
