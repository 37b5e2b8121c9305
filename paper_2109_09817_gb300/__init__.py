"""GB300-native exact Gaussian-process inference by blackbox K-hat products.

The method is BBMM/mBCG as used in arXiv 2109.09817 (MOB-ML pair energies):
K-hat V products formed tile by tile from the features, a pivoted-Cholesky
preconditioner, batched preconditioned CG, Lanczos log-determinants,
hyperparameter gradients and prediction.  All arithmetic runs in libgp
(CUDA, sm_103a) behind the C ABI of include/gp.h; this package is the thin
binding.  Importing it does not load the library; the first Context does,
and fails loudly if libgp.so has not been built.
"""
from ._lib import (GP_FP32_SPLIT_F16, GP_FP32_PLAIN, GP_FP32_SPLIT_TF32,  # noqa: F401
                   GP_TF32, GP_VAR_EXACT, GP_VAR_NONE, GP_PC_SIGMA, GP_PC_RESID,
                   GP_STOP_RECURRENCE, GP_STOP_TRUE, EXPORTS, LIB_PATH)


def __getattr__(name):
    # the torch-facing binding is imported lazily so that `import` alone
    # needs neither torch nor the built library
    import importlib
    if name.startswith("__") or name in ("api", "autograd", "_lib", "build"):
        if name in ("api", "autograd", "build"):
            return importlib.import_module(__name__ + "." + name)
        raise AttributeError(name)
    api = importlib.import_module(__name__ + ".api")
    if hasattr(api, name):
        return getattr(api, name)
    if name == "MarginalLikelihood":
        return importlib.import_module(__name__ + ".autograd").MarginalLikelihood
    raise AttributeError(name)
