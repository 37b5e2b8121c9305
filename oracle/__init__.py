"""FP64 CPU oracle for exact-GP inference by blackbox matrix products.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import, call, link or run
anything in this package.  The product path (the CUDA library and its
binding) never does; it shares no code, header, table or constant with it.

Contents
--------
* ``gp_oracle``   -- plain, slow, obviously correct NumPy/SciPy definitions
                     of every quantity on the path (kernel, K-hat products,
                     pivoted Cholesky, PCG/mBCG, Lanczos quadrature,
                     log marginal likelihood, gradients, prediction).
* ``kmv_oracle.c`` -- the same kernel definition as streamed rows in C with
                     OpenMP (FP64 accumulation), for row samples of problems
                     too large for a dense matrix.
* ``build()`` / ``load_c()`` -- compile and load the C part (gcc, no
                     machine-specific flags).

Every function cites the passage of arXiv 2109.09817 it follows.
"""
from .gp_oracle import *  # noqa: F401,F403
from .cbuild import build, load_c  # noqa: F401
