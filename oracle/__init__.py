"""The oracle: a plain, slow, FP64 CPU implementation of the paper's method.

TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA path.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it; the product package shares no code with it and never imports it.

Modules:
  tensor    -- demag tensor (Newell closed form near, quadrature far; C core)
  micromag  -- H_eff terms, LLG right-hand side, RK4/Euler, energies
  adjoint   -- discrete adjoint (exact gradient of the discrete forward map)
  cnn       -- the 3D conv surrogate's forward/backward and Adam step

Parity unpinned: none; every function is pinned by tests in ``tests/``.
"""
