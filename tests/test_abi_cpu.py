"""Host-side checks that need no GPU: the C-ABI library builds, loads and
exports every entry point declared in include/abfe.h; the Python binding's
structure layouts match the header; lambda schedules reproduce the paper's
window counts."""
import os
import re
import subprocess

import numpy as np
import pytest

import abfe_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "abfe.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(abfe_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_header_symbol():
    import paper_2603_22274_gb300 as G
    G.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", G.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing
    L = G.lib()   # dlopen succeeds without a GPU
    for f in header_functions():
        assert hasattr(L, f)
    assert sorted(G.exported_symbols()) == header_functions()


def test_status_strings_without_gpu():
    import paper_2603_22274_gb300 as G
    L = G.lib()
    assert L.abfe_status_string(0) == b"ok"
    assert L.abfe_status_string(3) == b"neighbour list overflow"
    assert L.abfe_num_replicas(None) == 0
    assert L.abfe_last_error(None) is not None


def test_struct_layouts_match_header():
    """Compile a tiny C program against abfe.h and compare sizes/offsets with
    the ctypes structures of the binding."""
    import ctypes as C
    import tempfile
    from paper_2603_22274_gb300 import _binding as B
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "abfe.h"
int main(void){
  printf("%zu %zu %zu %zu %zu\n", sizeof(abfe_system_desc), sizeof(abfe_params),
         sizeof(abfe_tuning), sizeof(abfe_stats), sizeof(abfe_profile));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(abfe_system_desc, n_excl), offsetof(abfe_system_desc, anchors),
         offsetof(abfe_system_desc, b_kphi), offsetof(abfe_params, precision),
         offsetof(abfe_system_desc, n_torsions), offsetof(abfe_system_desc, torsion_phi0));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        a, b = subprocess.check_output([exe], text=True).strip().splitlines()
    sizes = list(map(int, a.split()))
    offs = list(map(int, b.split()))
    assert sizes == [C.sizeof(B.SystemDesc), C.sizeof(B.Params), C.sizeof(B.Tuning),
                     C.sizeof(B.Stats), C.sizeof(B.Profile)]
    assert offs == [B.SystemDesc.n_excl.offset, B.SystemDesc.anchors.offset,
                    B.SystemDesc.b_kphi.offset, B.Params.precision.offset,
                    B.SystemDesc.n_torsions.offset, B.SystemDesc.torsion_phi0.offset]


def test_paper_schedules_window_counts():
    c = S.paper_complex_schedule()
    s = S.paper_solvent_schedule()
    assert c.K == 80 and s.K == 73
    # path: restraint on, then charges off, then vdW off, shared end points
    assert c.lam_r[0] == 0 and c.lam_r[7] == 1 and np.all(c.lam_r[7:] == 1)
    assert np.all(np.diff(c.lam_q) <= 0) and np.all(np.diff(c.lam_v) <= 0)
    assert c.lam_q[-1] == 0 and c.lam_v[-1] == 0 and s.lam_r.max() == 0
    assert sorted(set(np.round(c.lam_r, 6))) == [0.0, 0.01, 0.03, 0.1, 0.3, 0.5, 0.75, 1.0]
    for f, K in [(S.schedule_k12, 12), (S.schedule_k42, 42), (S.schedule_solvent_k30, 30),
                 (S.schedule_k24, 24)]:
        assert f().K == K


def test_generator_shapes():
    t = S.tiny(1235)
    assert t.n == 672 and t.n_ligand == 24 and t.info["min_solute_water"] >= 0.15
    assert abs(t.charge[t.is_ligand == 1].sum()) < 1e-6
    # every stored value is exactly representable in binary32
    for a in (t.pos, t.charge, t.sigma, t.epsilon, t.box):
        assert np.array_equal(a, a.astype(np.float32).astype(np.float64))
    c = S.complex_leg(9, n_atoms=9000, core_diameter=2.2, n_lig=20)
    assert c.n == 9000 and c.n_ligand == 20 and c.boresch is not None
    assert len(set(c.boresch.anchors.tolist())) == 6
