"""Benchmark: lambda-state pair evaluations per second and aggregate ns/day of
batched alchemical windows (one launch per stage for all windows, step loop in
a CUDA graph) against the plain one-window-per-launch path, on synthetic
systems shaped like the paper's complex and solvent legs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload batch|complex60k|loop]
    python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank runs its own
segment of windows (distinct ligands, same size: weak scaling) with no
communication on the data path; only the start/stop barrier and the max of the
timings cross ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("λ-state pair evals/s & batched-window ns/day (vs plain) at oracle tolerance, "
          "1 GB300")
# FP32 operations per in-cutoff environment pair in the force kernel (FMA = 2),
# counted from pair_env in csrc/pair_kernels.cu (force path, no energy): 43 FP32
# instructions = 61 flops, plus 3 MUFU operations (rsqrt, ex2, rcp) not counted.
FLOPS_PER_PAIR = 61
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: batch 500, complex60k 1000, loop 20000, tiny 100)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--equilibrate", type=int, default=1500,
                    help="steps at gamma = 10/ps after the relaxation, before tuning and timing "
                         "(1,500 bring the synthetic starts to their steady kinetic temperature)")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--exchange-every", type=int, default=10,
                    help="after the timed region: time the same steps with an in-loop replica "
                         "exchange attempt every N steps (0 = skip)")
    ap.add_argument("--export-every", type=int, default=None,
                    help="steps between u_kn/dU/dlambda exports inside the timed region "
                         "(default: loop 250, others 0 = no export)")
    ap.add_argument("--study", default=None, choices=["precision", "mbar"],
                    help="run the 100k-atom precision study or the MBAR study instead of the "
                         "throughput bench")
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "complex60k", "loop", "tiny"])
    ap.add_argument("--dt", type=float, default=0.001)
    ap.add_argument("--gamma", type=float, default=1.0)
    ap.add_argument("--graph-steps", type=int, default=500)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune-cache", default=None)
    ap.add_argument("--pme", default=None,
                    help="ORDER:SPACING_NM: add reciprocal-space Ewald (smooth PME) to every window")
    ap.add_argument("--tuning", default=None,
                    help="G:MAX_ENTRIES:BLOCK[:SKIN[:PRUNE_SKIN]] applied after (or "
                         "instead of) the autotuner")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = {"batch": 500, "complex60k": 1000, "loop": 20000, "tiny": 100}.get(a.workload, 100)
    if a.export_every is None:
        a.export_every = 250 if a.workload == "loop" else 0
    return a


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_workload(name, rank):
    import abfe_synth as S
    if name == "batch":
        # each rank: its own 16 ligands (seed offset), same sizes distribution
        if rank:
            S.BASE_SEED = 1234 + 100000 * rank
        return S.workload_batch()
    if name == "complex60k":
        return S.workload_complex60k(n_replicas=1)
    if name == "loop":
        return S.workload_loop()
    return S.workload_tiny()


def workload_desc(w, name):
    atoms = int(sum(w.systems[s].n for s in w.system_of_replica))
    if name == "batch":
        d = (f"batch: {w.n_replicas} windows = 16 ligands x (complex leg 40k-80k atoms, 42 "
             f"windows + solvent leg 3.5 nm box ~4.5k atoms, 30 windows), {atoms} atoms")
    else:
        d = f"{w.name}: {w.n_replicas} windows, {atoms} atoms"
    return d, atoms


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.p = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self, dev=0):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            t = [x.strip() for x in line.split(",")]
            if len(t) < 9 or not t[0].isdigit() or int(t[0]) != dev:
                continue
            try:
                sm.append(float(t[1]))
                mx.append(float(t[2]))
            except ValueError:
                continue
            for n, v in zip(names, t[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(w, budget_s=12.0):
    """The FP64 oracle, as it stands, on the host cores: forces and energies of
    solvent-leg windows of the workload (all pairs), until the budget is spent."""
    import oracle as O
    idx = [r for r in range(w.n_replicas) if w.systems[w.system_of_replica[r]].n <= 6000]
    if not idx:
        idx = [0]
    pairs, t0, n_done = 0, time.perf_counter(), 0
    while True:
        r = idx[n_done % len(idx)]
        s = w.systems[w.system_of_replica[r]]
        lam = w.schedules[w.schedule_of_replica[r]].state(int(w.state_of_replica[r]))
        o = O.nonbonded(s, w.params, lam[1], lam[2])
        pairs += o["npairs_env"] + o["npairs_lig"]
        n_done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    s0 = w.systems[w.system_of_replica[idx[0]]]
    return {"value": pairs / el, "unit": "pair-evals/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n_done} all-pairs FP64 force+energy evaluations of {s0.n}-atom windows "
                      f"({pairs} in-cutoff pairs, {el:.1f} s)"}


def run_reference(args):
    """--impl reference: the oracle as the reference arm (rank 0 only)."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    w = make_workload(args.workload, 0)
    desc, atoms = workload_desc(w, args.workload)
    import oracle as O
    idx = [r for r in range(w.n_replicas) if w.systems[w.system_of_replica[r]].n <= 6000] or [0]

    def one(k):
        r = idx[k % len(idx)]
        s = w.systems[w.system_of_replica[r]]
        lam = w.schedules[w.schedule_of_replica[r]].state(int(w.state_of_replica[r]))
        o = O.nonbonded(s, w.params, lam[1], lam[2])
        return o["npairs_env"] + o["npairs_lig"], s.n

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    pairs = 0
    n_at = 0
    for k in range(args.steps):
        p, n_at = one(k)
        pairs += p
    el = time.perf_counter() - t0
    v = pairs / el
    sample = (f"each step: one all-pairs FP64 force+energy evaluation of one {n_at}-atom window "
              f"of the workload")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pair-evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc},
        "cpu_baseline": {"kind": "oracle", "cores": O.num_threads(), "sample": sample, "value": v,
                         "unit": "pair-evals/s"},
        "e2e": {"value": v, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def ns_per_day(n_windows, steps, dt_ps, seconds):
    return n_windows * steps * dt_ps * 1e-3 / seconds * 86400.0


def plain_path(w, args, stream):
    """Each distinct system as its own one-window context, kernels launched
    directly (no graph, no batching); time per step, summed over all windows."""
    import torch

    import paper_2603_22274_gb300 as G
    import abfe_synth as S
    t_sys = {}
    for sid, s in enumerate(w.systems):
        reps = np.where(w.system_of_replica == sid)[0]
        if len(reps) == 0:
            continue
        r = int(reps[0])
        one = S.Workload("one", [s], np.zeros(1, np.int32), [w.schedules[w.schedule_of_replica[r]]],
                         np.zeros(1, np.int32), np.array([w.state_of_replica[r]], np.int32), w.params)
        e = G.engine_for_workload(one, stream=stream)
        e.set_tuning(graph_steps=0)
        e.step(20, dt=0.0005, gamma=20.0, seed=99)
        e.step(5, dt=args.dt, gamma=args.gamma, seed=98)
        n = 20
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e.step(n, dt=args.dt, gamma=args.gamma, seed=97)
        b.record(stream)
        b.synchronize()
        t_sys[sid] = a.elapsed_time(b) / 1000.0 / n
        e.close()
    per_step = sum(t_sys[int(w.system_of_replica[r])] for r in range(w.n_replicas))
    return per_step, t_sys


def precision_study(args):
    """100,000-atom complex-shaped system (90-atom ligand with four +-2 e atoms,
    cutoff 1.2 nm, beta 2.6, K = 42): frames saved from the engine's own MD are
    evaluated by the FP32 path, the all-FP64 GPU path and the FP64 oracle."""
    import torch

    import oracle as O
    import paper_2603_22274_gb300 as G
    import abfe_synth as S
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    w = S.workload_precision()
    s, P, sch = w.systems[0], w.params, w.schedules[0]
    e32 = G.engine_for_workload(w, stream=stream, precision=0)
    e64 = G.engine_for_workload(w, stream=stream, precision=1)
    e32.step(200, dt=0.0005, gamma=20.0, seed=5)        # relax the synthetic start
    rng = np.random.default_rng(0)
    rows = np.unique(np.r_[rng.choice(s.n, 256, replace=False), np.where(s.is_ligand)[0]])
    err = {t: {"ukn": [], "force": [], "energy": []} for t in ("32", "64")}
    t_gpu = {"32": 0.0, "64": 0.0}
    to = 0.0
    pairs = 0
    full_every = max(1, args.frames // 4)
    lam = sch.state(0)
    for fr in range(args.frames):
        e32.step(50, dt=0.001, gamma=1.0, seed=100 + fr)
        X = e32.positions()
        e64.set_positions(X)
        got = {}
        for eng, tag in ((e32, "32"), (e64, "64")):
            torch.cuda.synchronize()
            t = time.perf_counter()
            F, E, D = eng.compute()
            U, dU, Dd = eng.eval_ukn(sch.K)
            torch.cuda.synchronize()
            t_gpu[tag] += time.perf_counter() - t
            got[tag] = (F[rows], E[0, G.ENERGY_NAMES.index("total")], dU[0, :sch.K])
        t = time.perf_counter()
        ref_du = O.ukn_lambda_part(s, P, sch, pos=X)
        Fo = (O.force_rows(s, P, lam[1], lam[2], rows, pos=X) + O.bonds(s, pos=X)[1][rows]
              + O.boresch(s, lam[0], pos=X)[1][rows]
              + O.torsion_state(s, P, lam[2], pos=X)[1][rows])
        full = None
        if fr % full_every == 0:
            nb = O.nonbonded(s, P, lam[1], lam[2], forces=False, pos=X)
            full = (nb["E"].sum() + O.bonds(s, pos=X, forces=False)[0]
                    + lam[0] * O.boresch(s, lam[0], pos=X, forces=False)[0]
                    + O.torsion_state(s, P, lam[2], pos=X, forces=False)[0])
            pairs += nb["npairs_env"] + nb["npairs_lig"]
        to += time.perf_counter() - t
        for tag in ("32", "64"):
            Fg, Eg, dUg = got[tag]
            err[tag]["ukn"].append(float(np.abs(dUg - ref_du).max()))
            err[tag]["force"].append(float(np.sqrt(((Fg - Fo) ** 2).sum() / (Fo ** 2).sum())))
            if full is not None:
                err[tag]["energy"].append(float(abs(Eg - full) / abs(full)))
    c = e32.count_pairs()
    n_pairs = float(c.sum())
    out = {"study": "precision", "workload": "precision-100k-K42: 100,000 atoms, 10 nm box, 90-atom "
           "ligand (four +-2 e atoms), cutoff 1.2 nm, beta 2.6 nm^-1, K=42",
           "frames": args.frames, "data": "synthetic, frames from the engine's own MD (50 steps apart)"}
    for tag in ("32", "64"):
        out["fp" + tag] = {"ukn_lambda_part_max_abs_err_kJmol": max(err[tag]["ukn"]),
                           "force_rel_rms_err_max": max(err[tag]["force"]),
                           "total_energy_rel_err_max": max(err[tag]["energy"]),
                           "pair_evals_per_s": n_pairs * args.frames / t_gpu[tag],
                           "what": "abfe_compute + abfe_eval_ukn per frame, host clock"}
    out["oracle"] = {"pair_evals_per_s_full_evaluations": pairs / max(to, 1e-9),
                     "cores": O.num_threads(), "seconds": to}
    out["tolerances"] = {"ukn_kJmol": 1e-3, "force_rel_rms": 1e-5, "energy_rel": 1e-6}
    print(json.dumps(out))
    e32.close()
    e64.close()


# DRAM bytes (read + write) of one k_env_rows launch from an ncu capture, with
# the in-cutoff pairs of that launch: valid only for the kernel sources it was
# taken on (hash); the timed launches' traffic is scaled by their pair count
# (the traffic is the row words and the j atoms: it grows with the pairs). The
# command and the figures are in the named profile summary.
ENV_DRAM = {
    "batch": {"bytes": 11133695744 + 948676096, "pairs": 8236086179.0, "sha": "3dacd9c4d6d72193",
              "source": "profiles/k_env_rows_batch1152_dram.md"},
}


def measured_hbm_gbs():
    """The measured copy bandwidth of this GPU pool (GB/s) and where it came from;
    6,800 GB/s (an earlier GB300 measurement) when no measurement file exists."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback"


def _kernel_sha():
    import hashlib
    h = hashlib.sha256()
    base = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2603_22274_gb300", "csrc")
    for f in ("pair_kernels.cu", "abfe_internal.cuh", "erfc_coeffs.h"):
        with open(os.path.join(base, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def apply_tuning(eng, spec):
    t = spec.split(":")
    kw = dict(group=int(t[0]), max_entries=int(t[1]), block_threads=int(t[2]))
    if len(t) > 3:
        kw["skin"] = float(t[3])
    if len(t) > 4:
        kw["prune_skin"] = float(t[4])
    eng.set_tuning(**kw)


def env_traffic(workload, pairs_per_launch):
    e = ENV_DRAM.get(workload)
    if not e or e["sha"] != _kernel_sha():
        return None, None
    return e["bytes"] * pairs_per_launch / e["pairs"], e["source"]


def mbar_study(args):
    """MBAR over one 80-window segment (the paper's protein-ligand window count):
    u_kn of 80 states x 2,000 samples each, resident in HBM (102 MB, FP64),
    solved to max |df| < 1e-10 by abfe_mbar_device; the oracle's numpy MBAR is
    timed per iteration on a bounded number of iterations of the same matrix.
    Synthetic: 1-D harmonic states whose stiffness grows by a factor 1.25 per
    window (neighbour overlap comparable to an alchemical schedule)."""
    import torch

    import paper_2603_22274_gb300 as G
    from oracle.mbar import mbar as mbar_oracle
    torch.cuda.set_device(0)
    K, per = 80, 2000
    ks = 1.25 ** np.arange(K)
    rng = np.random.default_rng(42)
    xs = np.concatenate([rng.normal(0.0, 1.0 / np.sqrt(k), per) for k in ks])
    u = 0.5 * ks[:, None] * xs[None, :] ** 2
    N_k = np.full(K, per)
    N = K * per
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    f, it = G.mbar(ut, N_k, tol=1e-10)                       # warm-up (graph build, allocator)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    torch.cuda.synchronize()
    th = time.perf_counter()
    ev0.record(stream)
    for _ in range(reps):
        f, it = G.mbar(ut, N_k, tol=1e-10)
    ev1.record(stream)
    ev1.synchronize()
    host_s = (time.perf_counter() - th) / reps
    dev_s = ev0.elapsed_time(ev1) / 1000.0 / reps
    # end to end from host memory (copy of u_kn inside)
    th = time.perf_counter()
    f_h, it_h = G.mbar(u, N_k, tol=1e-10)
    e2e_s = time.perf_counter() - th
    # oracle: iterations of the same equations, timed on a bounded count
    n_or = 20
    t = time.perf_counter()
    f_o, it_o = mbar_oracle(u, N_k, tol=1e-300, max_iter=n_or)
    or_s_iter = (time.perf_counter() - t) / n_or
    exact = 0.5 * np.log(ks / ks[0])
    per_iter = dev_s / max(it, 1)
    elems = K * N
    out = {"study": "mbar", "workload": f"MBAR segment: K={K} states x {per} samples (N={N}), FP64 u_kn in HBM",
           "data": "synthetic harmonic-state u_kn (stiffness x1.25 per window), seed 42",
           "iterations": it, "device_s": dev_s, "host_s": host_s, "e2e_s_from_host": e2e_s,
           "us_per_iteration": per_iter * 1e6,
           "iterations_per_s": it / dev_s,
           "u_kn_elements_per_s": elems * it / dev_s,
           "max_abs_df_vs_exact_kT": float(np.abs(f - exact).max()),
           "host_vs_device_input_identical": bool(np.array_equal(f, f_h)),
           "roofline": {"bound": "alu", "achieved": 4 * elems / per_iter / 1e12,
                        "peak": 1.25, "unit": "TFLOP/s (FP64)",
                        "frac": 4 * elems / per_iter / 1e12 / 1.25,
                        "note": "algorithmic FP64 flops = two K x N FMA passes per iteration "
                                "(arrangement B); peak = nominal GB300 FP64 rate (no measured "
                                "FP64 peak available); HBM: two reads of the 8-byte K x N matrix "
                                "per iteration give %.0f GB/s of %.1f %s" %
                                ((2 * 8 * elems / per_iter / 1e9,) + measured_hbm_gbs())},
           "cpu_baseline": {"value": elems / or_s_iter, "unit": "u_kn elements/s per iteration",
                            "kind": "oracle", "cores": 1,
                            "sample": f"{n_or} iterations of numpy MBAR on the same matrix"},
           "gpu_vs_oracle_per_iteration": or_s_iter / per_iter}
    print(json.dumps(out))


# Algorithmic HBM bytes per atom slot of the integrator (k_integrate, one BAOAB
# pass): read position, velocity, the three 64-bit force accumulators, the
# prune and build references and the original index (16 + 16 + 24 + 16 + 16 +
# 4); write position, velocity and the cleared accumulators (16 + 16 + 24).
# Padding slots read their original index only.
INTEGRATE_BYTES_ATOM = 148
INTEGRATE_BYTES_PAD = 4
# Algorithmic HBM bytes per atom slot of one outer rebuild (k_rb_prepare ... k_rb_gather:
# copy aside 36 + write column and permutation 8, column fill 12, per-column sort 24,
# gather and cluster boxes 92 + 104 written) and of one prune's position pass
# (k_prune_prep: read position and original index, write the prune reference, 36).
REBUILD_BYTES_ATOM = 276
PRUNE_PREP_BYTES_ATOM = 36


def kinetic_temperature(eng, w):
    """Kinetic temperature of all atoms of all windows (no constraints), K."""
    vel = eng.velocities()
    mass = np.concatenate([np.asarray(w.systems[sy].mass, np.float64) for sy in w.system_of_replica])
    return float((mass[:, None] * vel ** 2).sum() / (3 * len(mass) * 0.00831446261815324))


def parity_of_timed_batch(eng, w, rng_seed=7):
    """Oracle error norms of windows of the timed workload at the positions the
    timed steps left (outside the timed region): one solvent-leg window in full
    (every atom's force, total energy, dU/dlambda, every u_kn entry's lambda
    part) and one complex-leg window (forces on sampled atoms, full total
    energy, dU/dlambda, every u_kn entry's lambda part), both at intermediate
    lambda states."""
    import oracle as O
    F, E, D = eng.compute()
    U, dU, _ = eng.eval_ukn(max(s.K for s in w.schedules))
    X = eng.positions()
    n_of = np.array([w.systems[w.system_of_replica[r]].n for r in range(w.n_replicas)])
    sol = [r for r in range(w.n_replicas) if n_of[r] < 10000]
    cpx = [r for r in range(w.n_replicas) if n_of[r] >= 10000]
    picks = []
    if sol:
        picks.append(("solvent", sol[len(sol) // 2], None))
    if cpx:
        picks.append(("complex", cpx[len(cpx) // 2], 256))
    out = {"tolerances": {"force_rel_rms": 1e-5, "energy_rel": 1e-6, "ukn_lambda_part_kJmol": 1e-3,
                          "dudl_abs_kJmol": 1e-3},
           "windows": []}
    rng = np.random.default_rng(rng_seed)
    t0 = time.perf_counter()
    for kind, r, n_rows in picks:
        s = w.systems[w.system_of_replica[r]]
        sch = w.schedules[w.schedule_of_replica[r]]
        lam = sch.state(int(eng.replica_states()[r]))
        a, b = eng.offsets[r], eng.offsets[r + 1]
        Xr = X[a:b]
        nb = O.nonbonded(s, w.params, lam[1], lam[2], forces=n_rows is None, pos=Xr)
        ub, fb = O.bonds(s, pos=Xr)
        ut, ft, dt = O.torsion_state(s, w.params, lam[2], pos=Xr)
        fb = fb + ft
        UB, FB = 0.0, np.zeros_like(fb)
        if s.boresch is not None:
            UB, FB, _ = O.boresch(s, lam[0], pos=Xr)
        e_ref = float(nb["E"].sum() + ub + lam[0] * UB + ut)
        if n_rows is None:
            rows = np.arange(s.n)
            Fo = nb["F"] + fb + FB
        else:
            lig = np.where(s.is_ligand)[0]
            rows = np.unique(np.r_[rng.choice(s.n, n_rows, replace=False), lig[:16]])
            Fo = O.force_rows(s, w.params, lam[1], lam[2], rows, pos=Xr) + fb[rows] + FB[rows]
        Fg = F[a:b][rows]
        d_ref = np.array([UB, nb["dudl_q"], nb["dudl_v"] + dt])
        du_ref = O.ukn_lambda_part(s, w.params, sch, pos=Xr)
        out["windows"].append({
            "leg": kind, "replica": int(r), "atoms": int(s.n), "state": [float(v) for v in lam],
            "force_rows": int(len(rows)),
            "force_rel_rms": float(np.sqrt(((Fg - Fo) ** 2).sum() / (Fo ** 2).sum())),
            "energy_rel": float(abs(E[r, -1] - e_ref) / abs(e_ref)),
            "dudl_max_abs_kJmol": float(np.abs(D[r] - d_ref).max()),
            "ukn_lambda_part_max_abs_kJmol": float(np.abs(dU[r, :sch.K] - du_ref).max()),
            "ukn_entries": int(sch.K)})
    tol = out["tolerances"]
    out["within_tolerance"] = bool(all(
        v["force_rel_rms"] <= tol["force_rel_rms"] and v["energy_rel"] <= tol["energy_rel"]
        and v["ukn_lambda_part_max_abs_kJmol"] <= tol["ukn_lambda_part_kJmol"]
        and v["dudl_max_abs_kJmol"] <= tol["dudl_abs_kJmol"] for v in out["windows"]))
    out["oracle_s"] = time.perf_counter() - t0
    del F, X
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.study == "precision":
        precision_study(args)
        return
    if args.study == "mbar":
        mbar_study(args)
        return
    ws, rank, local = dist_setup()
    import torch

    import paper_2603_22274_gb300 as G
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    t_setup = time.perf_counter()
    w = make_workload(args.workload, rank)
    if args.pme:
        po, sp = args.pme.split(":")
        w.params = dict(w.params, pme_order=int(po), pme_spacing=float(sp))
    desc, atoms = workload_desc(w, args.workload)
    if args.pme:
        desc += f", smooth PME order {po}, grid spacing <= {sp} nm"
    eng = G.engine_for_workload(w, stream=stream)
    if args.tuning:
        apply_tuning(eng, args.tuning)
    # relax the synthetic start (strong friction, short step), then bring the
    # kinetic temperature to T with a stronger thermostat at the production step
    eng.step(100, dt=0.0005, gamma=20.0, seed=1000 + rank)
    eng.step(args.equilibrate, dt=args.dt, gamma=10.0, seed=1100 + rank)
    if not args.no_autotune:
        eng.autotune(args.tune_cache, reps=3)
        eng.autotune_cadence(dt=args.dt, gamma=args.gamma, seed=500 + rank, n_steps=48)
    if args.tuning:
        apply_tuning(eng, args.tuning)
    tune = eng.tuning()
    # the timed steps are whole replays of one captured graph of gs steps; the
    # graph is captured (with its profiling event nodes) during the warm-up
    # --graph-steps 0: direct launches (no graph), e.g. for per-kernel profilers
    gs = max(1, min(args.graph_steps, args.steps)) if args.graph_steps > 0 else 0
    if gs:
        args.steps = gs * int(math.ceil(args.steps / gs))
    eng.set_tuning(graph_steps=gs)
    c0 = eng.count_pairs()
    eng.step(1, dt=args.dt, gamma=args.gamma, seed=1999 + rank)   # forces valid again
    eng.set_profiling((gs or args.steps) + 8)
    # the graph is captured (with its profiling event nodes) by its first replay,
    # which runs before the warm-up; the warm-up is exactly W steps
    n_capture = gs
    if gs:
        eng.step(gs, dt=args.dt, gamma=args.gamma, seed=1998 + rank)
    n_warm = max(args.warmup, 1)
    eng.step(n_warm, dt=args.dt, gamma=args.gamma, seed=2000 + rank)
    st0 = eng.stats()
    t_kin0 = kinetic_temperature(eng, w)
    setup_s = time.perf_counter() - t_setup

    clocks = ClockSampler(os.path.join(tempfile.gettempdir(), f"abfe_clocks_{rank}.csv"))
    clocks.start()
    time.sleep(0.5)
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    th0 = time.perf_counter()
    ev0.record(stream)
    n_exports = 0
    if args.export_every > 0:
        kmax0 = max(s.K for s in w.schedules)
        for k0 in range(0, args.steps, args.export_every):
            eng.step(min(args.export_every, args.steps - k0), dt=args.dt, gamma=args.gamma,
                     seed=3000 + rank + k0)
            eng.eval_ukn(kmax0)          # u_kn rows and dU/dlambda to host every export
            n_exports += 1
    else:
        eng.step(args.steps, dt=args.dt, gamma=args.gamma, seed=3000 + rank)
    ev1.record(stream)
    ev1.synchronize()
    host_el = time.perf_counter() - th0
    barrier(ws)
    el = ev0.elapsed_time(ev1) / 1000.0
    clk = clocks.stop(local)
    prof = eng.profile()
    st1 = eng.stats()
    c1 = eng.count_pairs()
    st_c = eng.stats()
    lane_groups = st_c["env_lane_groups"]
    # host-forced outer builds and prunes, timed with CUDA events around their
    # launches (outside the timed region)
    pb0 = eng.profile()
    for _ in range(3):
        eng.build_list()
    pb1 = eng.profile()
    st_b = eng.stats()
    n_b = max(pb1["build_launches"] - pb0["build_launches"], 1)
    n_p = max(pb1["prune_launches"] - pb0["prune_launches"], 1)
    build_ms = (pb1["build_ms"] - pb0["build_ms"]) / n_b
    prune_ms = (pb1["prune_ms"] - pb0["prune_ms"]) / n_p
    # kinetic temperature after the timed steps (all atoms, no constraints)
    t_kin = kinetic_temperature(eng, w)
    pairs_step = 0.5 * (c0.sum() + c1.sum())
    env_pairs_step = 0.5 * (c0[:, 0].sum() + c1[:, 0].sum())
    lig_pairs = 0.5 * (c0[:, 1].sum() + c1[:, 1].sum())
    # u_kn: every ligand pair is evaluated at each distinct lambda_v of its schedule
    kv = float(np.mean([len(set(np.round(w.schedules[w.schedule_of_replica[r]].lam_v, 12)))
                        for r in range(w.n_replicas)]))
    el_max = allmax(ws, el)
    pairs_all = allsum(ws, pairs_step * args.steps + n_exports * lig_pairs * kv)
    windows_all = allsum(ws, w.n_replicas)
    value = pairs_all / el_max
    nsd = ns_per_day(windows_all, args.steps, args.dt, el_max)
    rebuilds = st1["n_rebuilds"] - st0["n_rebuilds"]
    prunes = st1["n_prunes"] - st0["n_prunes"]
    win_rebuilds = st1["n_window_rebuilds"] - st0["n_window_rebuilds"]
    win_prunes = st1["n_window_prunes"] - st0["n_window_prunes"]
    slots = st1["slots"]
    int_bytes = atoms * INTEGRATE_BYTES_ATOM + (slots - atoms) * INTEGRATE_BYTES_PAD
    int_ms = prof["integrate_ms"] / max(prof["integrate_launches"], 1)
    hbm_peak, hbm_src = measured_hbm_gbs()
    # outer build: the rebuild kernels' per-atom traffic plus the builder's list
    # writes (8 B per entry, 40 B per masked entry, 32 B per work item) and reads
    # of the cluster boxes (40 B per cluster) and positions (16 B per atom)
    b_bytes = (atoms * (REBUILD_BYTES_ATOM + 16) + 40 * st_b["clusters"] + 8 * st_b["n_entries"]
               + 40 * st_b["n_xentries"] + 32 * (st_b["n_items_env"] + st_b["n_items_lig"]))
    # prune: the position pass plus reads of the outer list and the j rows written
    p_bytes = (slots * PRUNE_PREP_BYTES_ATOM + 8 * st_b["n_entries"] + 40 * st_b["n_xentries"]
               + 4 * st_b["n_rows"] + 8 * st_b["n_xrows"])
    hbm = {"integrate": {"kernel": "k_integrate", "ms_per_launch": int_ms,
                         "bytes_per_launch": int_bytes,
                         "achieved_gbs": int_bytes / (int_ms * 1e-3) / 1e9,
                         "bytes_per_atom": INTEGRATE_BYTES_ATOM},
           "list_build": {"kernels": "k_rb_* + k_build_list_env/lig (outer list)",
                          "ms_per_build": build_ms, "bytes_per_build": b_bytes,
                          "achieved_gbs": b_bytes / (build_ms * 1e-3) / 1e9,
                          "note": "latency-bound builder: the GB/s is its algorithmic traffic over "
                                  "its time, not a bandwidth limit"},
           "prune": {"kernels": "k_prune_prep + k_prune (inner rows)", "ms_per_prune": prune_ms,
                     "bytes_per_prune": p_bytes,
                     "achieved_gbs": p_bytes / (prune_ms * 1e-3) / 1e9},
           "peak_gbs": hbm_peak, "peak_source": hbm_src}
    for k in ("integrate", "list_build", "prune"):
        hbm[k]["frac"] = hbm[k]["achieved_gbs"] / hbm_peak

    # ---- e2e through the public API with host outputs: K steps + the u_kn / dU/dlambda export
    kmax = max(s.K for s in w.schedules)
    e2e_steps = gs * max(1, min(args.steps, 500) // gs) if gs else min(args.steps, 500)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    eng.step(e2e_steps, dt=args.dt, gamma=args.gamma, seed=4000 + rank)
    U, dU, D = eng.eval_ukn(kmax)
    e2e_el = allmax(ws, time.perf_counter() - t0)
    e2e_units = allsum(ws, pairs_step * e2e_steps + lig_pairs * kv)
    e2e = {"value": e2e_units / e2e_el, "unit": "pair-evals/s",
           "h2d_bytes_per_step": 4 * 32 / e2e_steps,
           "d2h_bytes_per_step": (2 * U.nbytes + D.nbytes + 64) / e2e_steps,
           "what": f"abfe_step({e2e_steps}) + abfe_eval_ukn to host buffers, timed on the host clock"}

    # ---- roofline of the dominant kernel (environment pair kernel)
    env_ms = prof["env_ms"] / max(prof["env_launches"], 1)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    flops_launch = env_pairs_step * FLOPS_PER_PAIR
    achieved = flops_launch / (env_ms * 1e-3) / 1e12
    peak = n_sm * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    clk_mhz = clk["sm_mhz"] if clk else None
    traffic, traffic_src = env_traffic(args.workload, env_pairs_step)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
            "kernel": "k_env (environment cluster-pair force kernel)",
            "flops_per_pair": FLOPS_PER_PAIR, "pairs_per_launch": env_pairs_step,
            "launch_ms": env_ms, "launches_timed": prof["env_launches"],
            "lane_efficiency": float(c1[:, 0].sum()) / max(32.0 * lane_groups, 1.0),
            "peak_note": f"FP32 peak = {n_sm} SMs x 128 lanes x 2 x {SM_MAX_MHZ:.0f} MHz (max clock)"}
    if clk_mhz:
        roof["frac_at_median_clock"] = achieved / (peak * clk_mhz / SM_MAX_MHZ)

    # replica exchange inside the captured step loop: the same steps with an
    # attempt every N steps, against the timed region's time per step
    exch = None
    if args.exchange_every > 0 and gs:
        eng.set_exchange(args.exchange_every, seed=77 + rank)
        st_x0 = eng.stats()
        eng.step(gs, dt=args.dt, gamma=args.gamma, seed=5000 + rank)   # captures the graph
        torch.cuda.synchronize()
        xa = torch.cuda.Event(enable_timing=True)
        xb = torch.cuda.Event(enable_timing=True)
        xa.record(stream)
        eng.step(gs, dt=args.dt, gamma=args.gamma, seed=5001 + rank)
        xb.record(stream)
        xb.synchronize()
        st_x1 = eng.stats()
        eng.set_exchange(0)
        ms_x = xa.elapsed_time(xb) / gs
        n_att = (st_x1["n_exchange_attempts"] - st_x0["n_exchange_attempts"]) / 2.0
        exch = {"every_steps": args.exchange_every, "steps": gs, "attempts_per_graph": n_att,
                "ms_per_step_with_exchange": ms_x, "ms_per_step_without": 1000 * el / args.steps,
                "ms_per_attempt": (ms_x - 1000 * el / args.steps) * gs / max(n_att, 1.0),
                "accepted": st_x1["n_exchange_accepted"] - st_x0["n_exchange_accepted"],
                "what": "abfe_set_exchange: u_kn energy pass, device exchange and new-state forces "
                        "inside a conditional node of the captured step graph"}

    parity = None
    if rank == 0 and not args.no_parity:
        parity = parity_of_timed_batch(eng, w)

    out = None
    if rank == 0:
        plain = None
        if not args.no_plain:
            per_step, t_sys = plain_path(w, args, stream)
            plain_nsd = ns_per_day(w.n_replicas, 1, args.dt, per_step)
            nsd_1 = ns_per_day(w.n_replicas, args.steps, args.dt, el)
            plain = {"ns_per_day": plain_nsd, "batched_ns_per_day": nsd_1,
                     "batched_vs_plain": nsd_1 / plain_nsd,
                     "method": "each distinct system as a one-window context, direct launches, "
                               "per-step time summed over all windows"}
        cpu = None if args.no_cpu else cpu_baseline(w)
        # per step: integrate, step_end, env, lig, bonds, torsions, boresch; per rebuild
        # event: 5 rebuild kernels, the two builders and the item prefix; per prune event:
        # the position pass, the prune and the row-item prefix; per export: the force
        # pass (15) + u_kn, assemble, finalize
        launches = args.steps * 7 + 8 * rebuilds + 3 * prunes + 2 + n_exports * 18
        out = {
            "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": ws,
            "steps": args.steps, "warmup": n_warm, "ms_per_step": 1000 * el_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc, "windows": int(windows_all), "atoms_per_gpu": atoms,
                       "dt_ps": args.dt, "gamma_per_ps": args.gamma, "cutoff_nm": w.params["cutoff"],
                       "skin_nm": w.params["skin"], "tuning": tune, "graph_steps": gs,
                       "graph_capture_steps": n_capture, "equilibration_steps": args.equilibrate,
                       "l2": "inputs larger than L2 (all windows resident in HBM)",
                       "parallelism": f"{ws} GPU(s), window segments per GPU, no data-path collective"},
            "ns_per_day": nsd, "pair_evals_per_step": pairs_step, "rebuilds_timed": rebuilds,
            "prunes_timed": prunes,
            "window_rebuilds_per_step": win_rebuilds / max(args.steps, 1) / w.n_replicas,
            "window_prunes_per_step": win_prunes / max(args.steps, 1) / w.n_replicas, "hbm": hbm, "parity": parity, "exchange": exch,
            "exports_timed": n_exports, "kinetic_temperature_K": t_kin,
            "kinetic_temperature_before_K": t_kin0,
            "plain": plain, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
            "gpu_launches": launches, "clocks": clk, "setup_s": setup_s, "timed_host_s": host_el,
            "device_bytes": int(st1["device_bytes"]),
            "profile_ms_per_launch": {k[:-3]: prof[k] / max(prof[k[:-3] + "_launches"], 1)
                                      for k in ("env_ms", "lig_ms", "integrate_ms")},
            "profile_note": "event times on each kernel's own stream; lig runs on the forked stream "
                            "beside env, so its time includes the time it shares the SMs with env",
        }
        print(json.dumps(out))
    eng.close()


if __name__ == "__main__":
    main()
