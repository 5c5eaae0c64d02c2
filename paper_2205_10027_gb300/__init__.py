"""GB300-native pISTA solver for the graphical lasso.

The compute path lives in the C-ABI library ``libglasso.so`` (hand-written sm_103a CUDA
kernels); ``binding`` marshals arguments to it.  Importing this package does not load the
library: ``paper_2205_10027_gb300.binding`` does, and raises if it is missing.
"""
__version__ = "0.1.0"
