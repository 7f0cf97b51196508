"""GB300-native alchemical nonbonded engine for absolute binding free energy
lambda windows: Beutler-softcore LJ + real-space Ewald Coulomb over a cluster
neighbour list, a Boresch restraint and BAOAB Langevin dynamics, batched over
all windows of many ligands in one launch per stage, emitting forces, dU/dlambda
and the MBAR reduced-potential row u_kn.

The compute path is the C-ABI library libabfe.so (include/abfe.h, CUDA for
sm_103a); this package only loads it and marshals arguments.
"""
from ._binding import (  # noqa: F401
    DUDL_NAMES,
    ENERGY_NAMES,
    N_DUDL,
    N_ENERGY,
    AbfeError,
    boresch_correction,
    Engine,
    engine_for_workload,
    exported_symbols,
    lib,
    mbar,
    use_torch_allocator,
)
from .build import LIB as LIB_PATH  # noqa: F401
from .build import build  # noqa: F401
