"""GB300-native (sm_103a) tensorized RVEA: one generation of reproduction,
evaluation and reference-vector guided selection per call, in hand-written
CUDA behind a small C ABI (include/rvea.h)."""
from .rvea import (DTLZ1_LINEAR, DTLZ2_SPHERE, DTLZ3_SPHERE, DTLZ4_SPHERE, NEURO_LINEAR, REPRO_CSO,
                   REPRO_DE, REPRO_PSO, REPRO_RANDOM, REPRO_SBX_PM, Batch, Run, RveaError, Server,
                   autotune, gamma, get_plan, lattice_for, lattice_size, select, set_plan, step_batch,
                   workspace_bytes)

__all__ = ["Run", "Batch", "Server", "RveaError", "step_batch", "autotune", "get_plan", "set_plan",
           "select", "gamma", "workspace_bytes", "lattice_size", "lattice_for", "DTLZ2_SPHERE", "DTLZ1_LINEAR",
           "NEURO_LINEAR", "DTLZ3_SPHERE", "DTLZ4_SPHERE", "REPRO_SBX_PM", "REPRO_DE", "REPRO_RANDOM",
           "REPRO_CSO", "REPRO_PSO"]
