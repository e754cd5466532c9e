"""GB300-native H-MLE: Gaussian log-likelihood of a Matern field with the
covariance held as a hierarchical matrix, evaluated by hand-written CUDA
kernels for sm_103a behind a C ABI (``include/hmle.h``).

Submodules (imported lazily so that importing the package never requires
the CUDA library):

* ``paper_2104_07146_gb300.hmle``  -- ctypes binding of ``libhmle.so``.
* ``paper_2104_07146_gb300.build`` -- nvcc build of ``libhmle.so``.
* ``paper_2104_07146_gb300.synth`` -- seeded synthetic inputs.
"""
__all__ = ["hmle", "build", "synth"]
