"""The 100,000-atom precision configuration (10 nm box, 90-atom ligand with four
+-2 e atoms, cutoff 1.2 nm, beta 2.6 nm^-1, K = 42): one frame from the engine's
own MD, FP32 and all-FP64 GPU paths against the FP64 oracle at full size
(every u_kn entry's lambda part, forces of sampled atoms, the total energy)."""
import numpy as np
import pytest

import abfe_synth as S
import oracle as O

pytestmark = pytest.mark.gpu


def test_precision_100k_one_frame():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_22274_gb300 as G
    w = S.workload_precision()
    s, P, sch = w.systems[0], w.params, w.schedules[0]
    e32 = G.engine_for_workload(w, precision=0)
    e32.step(60, dt=0.0005, gamma=20.0, seed=5)
    e32.step(20, dt=0.001, gamma=1.0, seed=6)
    X = e32.positions()
    e64 = G.engine_for_workload(w, precision=1)
    e64.set_positions(X)
    lam = sch.state(0)
    rng = np.random.default_rng(1)
    rows = np.unique(np.r_[rng.choice(s.n, 200, replace=False), np.where(s.is_ligand)[0],
                           s.boresch.anchors])
    ref_du = O.ukn_lambda_part(s, P, sch, pos=X)
    Fo = (O.force_rows(s, P, lam[1], lam[2], rows, pos=X) + O.bonds(s, pos=X)[1][rows]
          + O.boresch(s, lam[0], pos=X)[1][rows] + O.torsion_state(s, P, lam[2], pos=X)[1][rows])
    nb = O.nonbonded(s, P, lam[1], lam[2], forces=False, pos=X)
    Eo = (nb["E"].sum() + O.bonds(s, pos=X, forces=False)[0]
          + lam[0] * O.boresch(s, lam[0], pos=X, forces=False)[0]
          + O.torsion_state(s, P, lam[2], pos=X, forces=False)[0])
    for eng, ftol, utol, etol in ((e32, 1e-5, 1e-3, 1e-6), (e64, 1e-6, 1e-5, 1e-9)):
        F, E, D = eng.compute()
        _, dU, _ = eng.eval_ukn(sch.K)
        assert np.abs(dU[0, :sch.K] - ref_du).max() <= utol
        f = F[rows]
        assert np.sqrt(((f - Fo) ** 2).sum() / (Fo ** 2).sum()) <= ftol
        assert abs(E[0, G.ENERGY_NAMES.index("total")] - Eo) <= etol * abs(Eo)
    e32.close()
    e64.close()
