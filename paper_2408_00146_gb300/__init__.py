"""GB300 (sm_103a) implementation of the fused collide-and-stream time step of
the coupled central-moment lattice Boltzmann system of arXiv 2408.00146
(surfactant-laden bubbles in self-rewetting fluids).

The computation lives in the CUDA library built from ``csrc/`` behind the C
ABI of ``include/lbm.h``; :mod:`.lbm` is its Python binding.
"""
from .lbm import (  # noqa: F401
    LbmError, Sim, load, lbm_create, lbm_derive, lbm_create_ex, lbm_destroy, lbm_get_derived,
    lbm_get_populations, lbm_init, lbm_launch_count, lbm_observe, lbm_step, lbm_step_batch,
    lbm_workspace_bytes,
)
