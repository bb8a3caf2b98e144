"""GB300 (sm_103a) implementation of the per-time-step path of the decoupled phase-field
scheme for two immiscible dielectric fluids (Yang, Christov & Dong, arXiv 2305.09020).

The compute path lives in the CUDA library built from ``csrc/`` behind the C-ABI of
``include/pf.h``; ``native`` is its thin Python binding.
"""
from . import native  # noqa: F401
from .native import (PF_BCSET_NN, PF_BCSET_P, PF_BCSET_U, PF_BCSET_V, PF_FIELD_E, PF_FIELD_OLD,  # noqa: F401
                     PF_FIELD_P, PF_FIELD_PHI, PF_FIELD_PSI, PF_FIELD_U, PF_FIELD_V, PF_FP64, PF_MIXED,
                     PfError, Solver, from_workload)
