"""Oracle: plain, slow, obviously correct CPU implementation of the method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import anything under this package.  It
shares no code with the CUDA library (``paper_1705_04374_gb300``) and never
imports it.

Modules:
  solver     FP64 C solver (WENO5 / HLLC / low-storage RK3 / CFL / QoIs), via ctypes
  cloud      seeded cloud-geometry sampler (Section 3.1 distributions)
  estimator  MLMC and OF-MLMC estimators, coefficients and sample numbers (Section 2.4)
  mlp        FP64 MLP surrogate forward / backward / Adam
"""
