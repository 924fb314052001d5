"""FP64 CPU oracle for DPar2 (arXiv 2203.12798) -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the CUDA
path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import it; the library itself
never does, and the oracle shares no code with the CUDA path.

Contents
  philox.py  Philox4x32-10 counter-based generator (Salmon et al., SC'11) and
             the Box-Muller Gaussian stream derived from it.
  dpar2.py   Algorithm 1 (randomized SVD), Algorithm 2 (PARAFAC2-ALS),
             Algorithm 3 (DPar2: two-stage compression + ALS on the
             compressed slices, written with materialised Y_k and the plain
             MTTKRP definitions), the fitness of Sec. IV-A, the preprocessed
             size of Theorem 2, and the learned-sketch loss and gradient.

Every function is pinned by a ``-m "not gpu"`` test in tests/test_oracle_*.py
to something other than itself (closed forms, exact-recovery cases, brute
force, invariants, published known-answer vectors); see the module docstrings
for the pin of each function.
"""
