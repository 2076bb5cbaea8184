"""GB300-native (sm_103a) tensorized RVEA: one generation of reproduction,
evaluation and reference-vector guided selection per call, in hand-written
CUDA behind a small C ABI (include/rvea.h)."""
from .rvea import (DTLZ1_LINEAR, DTLZ2_SPHERE, NEURO_LINEAR, Run, RveaError, gamma,
                   lattice_size, select, step_batch, workspace_bytes)

__all__ = ["Run", "RveaError", "step_batch", "select", "gamma", "workspace_bytes",
           "lattice_size", "DTLZ2_SPHERE", "DTLZ1_LINEAR", "NEURO_LINEAR"]
