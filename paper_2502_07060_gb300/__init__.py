"""Batched Berends-Giele recursion for colour-ordered n-gluon tree amplitudes
on GB300 (sm_103a), after arXiv:2502.07060.

* ``paper_2502_07060_gb300.bg``     -- ctypes binding of the C-ABI library
  ``libbg.so`` (bg_plan_create / bg_eval / ...); importing it loads the CUDA
  library and fails loudly when it has not been built.
* ``paper_2502_07060_gb300.inputs`` -- seeded synthetic momenta and
  polarisation states (host side, numpy).
* ``paper_2502_07060_gb300.build``  -- nvcc build of the CUDA library.
"""
