"""GB300-native SPFOM: the data-parallel iteration of the sales-based
primal-dual first-order method for choice-based LPs under the generalized
attraction model, as sm_103a CUDA kernels behind the C ABI of include/spfom.h.

``Solver`` is the Python face of that ABI; ``build.build()`` compiles the
library in-tree. Nothing here falls back to a CPU implementation.
"""
from .spfom import (EXPORTS, MLP, InstanceArrays, Solver, SpfomError, VEC_G, VEC_MARGINS, VEC_S, VEC_SUM_G,
                    VEC_SUM_Y, VEC_Y, VEC_YBAR, default_params, lib)

__all__ = ["Solver", "MLP", "SpfomError", "InstanceArrays", "default_params", "lib", "EXPORTS", "VEC_Y", "VEC_YBAR",
           "VEC_SUM_Y", "VEC_SUM_G", "VEC_G", "VEC_S", "VEC_MARGINS"]
