"""Seeded synthetic workloads for the exact-GP hot path.

This module only *draws inputs*: features X, targets y and test points X'.
It holds none of the method's arithmetic (no kernel, no solve), so both the
CUDA path and the FP64 oracle can take their inputs from here without
sharing any computation.

The real MOB-ML pair-energy features (QM7b-T / GDB-13-T, Sec. 4) are not
available, so the workloads below stand in for them at the paper's sizes
(N = 175,795 and 1,152,157 off-diagonal pairs, 124,973 diagonal pairs,
Tables 1-2): clustered Gaussian-mixture features, Matern-5/2 ARD
hyperparameters and smooth random-Fourier-feature targets.

Random draws use numpy's PCG64 ``default_rng(seed)`` only.
"""
from .workloads import (  # noqa: F401
    Workload,
    CONFIGS,
    make_workload,
    mixture_features,
    rff_targets,
    molecule_request,
)
