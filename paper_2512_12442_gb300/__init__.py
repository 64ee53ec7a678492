"""GB300 (sm_103a) library for Gaussian-process reconstruction and level-crossing
probability fields, after Li, Michaud, Biswas & Shen, "Efficient Level-Crossing
Probability Calculation for Gaussian Process Modeled Data".

The compute path is libgprlcp.so (CUDA, include/gpr_lcp.h); this package is its
ctypes binding.  Importing the binding does not need a GPU; calling it does.
"""
from .api import *  # noqa: F401,F403
from .api import GPRError, Model, lcp_options, make_grid  # noqa: F401
