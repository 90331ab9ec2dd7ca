"""GB300-native distribution-function-correction IB-LBM (arXiv 1803.09380).

The compute path is the CUDA library ``libibm.so`` built from ``csrc/`` for
sm_103a and reached through its C ABI (declared in ``include/ibm.h``); the
Python binding in :mod:`.ibm` only marshals arguments.  Importing this package
loads nothing; :func:`ibm.load` loads the library and raises if it is missing.
"""
__all__ = ["ibm", "workloads", "build"]
