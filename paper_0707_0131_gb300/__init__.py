"""GB300-native incremental eigCG for lattice-QCD Wilson fermions.

Hot path (CUDA, sm_103a) behind the C ABI of include/eigcg.h:
  Wilson dslash with fused CG updates, eigCG window restart, init-CG deflation,
  basis growth, mixed-precision reliable updates and multi-RHS batching.

  fixtures   seeded synthetic inputs (gauge fields, right-hand sides)
  _lib       ctypes binding with the C names (eig_op_create, eig_eigcg_solve, ...)
  api        Op / Basis convenience classes over the binding
  build      nvcc build of libeigcg.so
"""
