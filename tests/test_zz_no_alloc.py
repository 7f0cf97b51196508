"""The allocation-free entry point abfe_ukn_frame_noalloc, for callers that
cannot allocate device memory themselves (for example a plugin inside a host MD
engine whose device memory belongs to the host application). Its inputs and
output are the caller's device buffers; its only scratch is a fixed array
inside the library.

This file is collected last on purpose. The tests call the entry point through
the C ABI twice in a row (the second call reuses the scratch left by the first)
and compare each result with the lambda-dependent u_kn part that the existing
context entry point abfe_eval_ukn returns for the same frame, and with the FP64
oracle's u_kn lambda part directly (both ligand modes, with and without a
restraint, at the largest supported state count), within the u_kn tolerance of
the other tests (1e-3 kJ/mol per entry). A ligand index outside the atom range
must give NaN results, not a memory access. The entry point has no torsion
input, so the systems here carry no rotatable-bond torsions.
"""
import ctypes as C

import numpy as np
import pytest

import abfe_synth as S
import oracle as O

pytestmark = pytest.mark.gpu


def _no_torsions(s):
    s.torsions = np.zeros((0, 4), np.int32)
    s.torsion_k, s.torsion_n, s.torsion_phi0 = np.zeros(0), np.zeros(0, np.int32), np.zeros(0)
    return s


def _frame(G, s, P, sch, X, keep):
    import torch
    B = G._binding
    dev = torch.device("cuda")
    f = B.NoallocFrame()
    f.n_atoms = s.n
    for d in range(3):
        f.box[d] = float(s.box[d])
    lig = np.where(s.is_ligand)[0].astype(np.int32)
    excl = np.full((len(lig), B.NOALLOC_MAX_EXCL), -1, np.int32)
    where = {int(a): i for i, a in enumerate(lig)}
    fill = np.zeros(len(lig), int)
    for i, j in np.asarray(s.excl):
        for a, b in ((i, j), (j, i)):
            if a in where:
                k = where[a]
                excl[k, fill[k]] = b
                fill[k] += 1
    t = dict(pos=torch.tensor(X, dtype=torch.float32, device=dev),
             q=torch.tensor(s.charge, dtype=torch.float32, device=dev),
             sig=torch.tensor(s.sigma, dtype=torch.float32, device=dev),
             eps=torch.tensor(s.epsilon, dtype=torch.float32, device=dev),
             lig=torch.tensor(s.is_ligand, dtype=torch.uint8, device=dev),
             idx=torch.tensor(lig, device=dev),
             excl=torch.tensor(excl, device=dev))
    keep.append(t)
    f.pos, f.charge, f.sigma = t["pos"].data_ptr(), t["q"].data_ptr(), t["sig"].data_ptr()
    f.epsilon, f.is_ligand = t["eps"].data_ptr(), t["lig"].data_ptr()
    f.n_lig, f.lig_idx, f.lig_excl = len(lig), t["idx"].data_ptr(), t["excl"].data_ptr()
    f.K = sch.K
    for k in range(sch.K):
        f.lam_r[k], f.lam_q[k], f.lam_v[k] = sch.state(k)
    f.cutoff, f.ewald_beta = P["cutoff"], P["ewald_beta"]
    f.sc_alpha, f.sc_p, f.coulomb_k = P["sc_alpha"], P["sc_p"], P["coulomb_k"]
    f.ligand_mode = int(P.get("ligand_mode", 0))
    b = s.boresch
    f.has_boresch = 1 if b is not None else 0
    if b is not None:
        for i in range(6):
            f.anchors[i] = int(b.anchors[i])
        f.b_r0 = b.r0
        f.b_theta0[0], f.b_theta0[1] = b.theta0
        f.b_phi0[0], f.b_phi0[1], f.b_phi0[2] = b.phi0
        f.b_kr, f.b_ktheta, f.b_kphi = b.k_r, b.k_theta, b.k_phi
    return f


def test_noalloc_matches_context_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    c = _no_torsions(S.complex_leg(5, n_atoms=4500, core_diameter=1.6, n_lig=24))
    sch = S.schedule_k42()
    P = S.params_for(1.0, 3.12)
    w = S.Workload("one", [c], np.zeros(1, np.int32), [sch], np.zeros(1, np.int32),
                   np.array([7], np.int32), P)
    eng = G.engine_for_workload(w)
    U, dU, _ = eng.eval_ukn()
    X = eng.positions()
    eng.close()
    keep = []
    f = _frame(G, c, P, sch, X, keep)
    out = torch.full((sch.K,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out.fill_(float("nan"))
        st = G.lib().abfe_ukn_frame_noalloc(C.byref(f), C.c_void_p(out.data_ptr()),
                                            C.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - dU[0, :sch.K]).max() <= 1e-3, np.abs(got - dU[0, :sch.K]).max()
    # sizes beyond the stated maxima are rejected before any launch
    f.K = G._binding.NOALLOC_MAX_K + 1
    assert G.lib().abfe_ukn_frame_noalloc(C.byref(f), C.c_void_p(out.data_ptr()), None) == 1


def _run(G, f, K, out):
    import torch
    out.fill_(float("nan"))
    st = G.lib().abfe_ukn_frame_noalloc(C.byref(f), C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()[:K]


def _k128():
    """128 states: restraint on over 8, charges off over 40, vdW off over 80."""
    lr = np.r_[np.linspace(0.0, 1.0, 8), np.ones(120)]
    lq = np.r_[np.ones(8), np.linspace(1.0, 0.0, 41)[1:], np.zeros(80)]
    lv = np.r_[np.ones(48), np.linspace(1.0, 0.0, 81)[1:]]
    return S.LambdaSchedule("k128", lr, lq, lv)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("leg", ["complex", "solvent"])
def test_noalloc_matches_oracle_at_max_states(mode, leg):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    O.build()
    if leg == "complex":
        s = S.complex_leg(5, n_atoms=4500, core_diameter=1.6, n_lig=24)      # with a restraint
    else:
        s = S.solvent_leg(6, n_lig=40, box=3.0, n_atoms=2800)                # no restraint
    s = _no_torsions(s)
    sch = _k128()
    assert sch.K == G._binding.NOALLOC_MAX_K
    P = S.params_for(1.0, 3.12, ligand_mode=mode)
    X = S.f32(np.mod(s.pos, s.box))
    ref = O.ukn_lambda_part(s, P, sch, pos=X)
    if mode == 1:
        # decoupling: the ligand's own pairs do not depend on lambda
        e = O.nonbonded(s, P, 1.0, 1.0, forces=False, pos=X)["energy"]
        ref = ref - e["liglig_lj"] - e["liglig_c"]
    keep = []
    f = _frame(G, s, P, sch, X, keep)
    out = torch.empty(sch.K, dtype=torch.float64, device="cuda")
    for _ in range(2):
        got = _run(G, f, sch.K, out)
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-3, np.abs(got - ref).max()


def test_noalloc_bad_ligand_index_gives_nan_then_recovers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    G.lib()
    s = _no_torsions(S.solvent_leg(6, n_lig=40, box=3.0, n_atoms=2800))
    sch = S.schedule_solvent_k30()
    P = S.params_for(1.0, 3.12)
    X = S.f32(np.mod(s.pos, s.box))
    keep = []
    f = _frame(G, s, P, sch, X, keep)
    out = torch.empty(sch.K, dtype=torch.float64, device="cuda")
    good = _run(G, f, sch.K, out)
    assert np.isfinite(good).all()
    idx = keep[-1]["idx"]
    saved = int(idx[3].item())
    for bad in (s.n, -1):
        idx[3] = bad                       # an atom index outside [0, n)
        got = _run(G, f, sch.K, out)
        assert np.isnan(got).all()
    idx[3] = saved                         # the scratch left by the bad call is overwritten
    np.testing.assert_array_equal(_run(G, f, sch.K, out), good)
