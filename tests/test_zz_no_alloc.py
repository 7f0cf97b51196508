"""The allocation-free entry point abfe_ukn_frame_noalloc, for callers that
cannot allocate device memory themselves (for example a plugin inside a host MD
engine whose device memory belongs to the host application). Its inputs and
output are the caller's device buffers; its only scratch is a fixed array
inside the library.

This file is collected last on purpose. The test calls the entry point through
the C ABI twice in a row (the second call reuses the scratch left by the first)
and compares each result with the lambda-dependent u_kn part that the existing
context entry point abfe_eval_ukn returns for the same frame, within the u_kn
tolerance of the other tests (1e-3 kJ/mol per entry).
"""
import ctypes as C

import numpy as np
import pytest

import abfe_synth as S

pytestmark = pytest.mark.gpu


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
    c = S.complex_leg(5, n_atoms=4500, core_diameter=1.6, n_lig=24)
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
