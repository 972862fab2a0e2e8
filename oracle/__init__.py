"""CPU oracle for the elastoplastic hot path (plain numpy/scipy, FP64).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of
`__graft_entry__` and the CPU-baseline leg of `bench.py` may import this
package.  It shares no code with the CUDA path and never calls it.

Modules:
  elements      reference elements and quadrature (Appendix)
  constitutive  return mappings and consistent tangents (Sections 2.2, 2.3, 7.1, 7.2)
  fem           geometry, B, D, K = K_elast + B^T(D_t - D_e)B, F (Sections 6, 7, 9)
  newton        ALG-NEWTON load path and the homogeneous one-point solve (Section 4)

Pins: every function is checked by tests/test_oracle_*.py against closed
forms, invariants, brute force or values printed in the paper.  Parity
unpinned: none of the functions above; the full-size non-homogeneous
workloads (fixed-base Q1 cube, P2 tetrahedral strip) have no printed value,
so only their building blocks are pinned.
"""
