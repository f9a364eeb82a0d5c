"""CPU FP64 oracle for MG-MLMC++ trace estimation (Frommer & Nasr Khalil, 2023).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, obviously correct
restatement of the method in numpy/scipy double precision, written from the
paper, and it shares no code with the CUDA library: only the test-suite, the
package's smoke check and the CPU-baseline leg of the benchmark may import it.
The product path never calls it and has no CPU fallback.

Modules
  schwinger   2D Schwinger Wilson-Dirac operator (sparse and dense), gamma5,
              free-field closed forms.
  rng         counter-based Rademacher streams (SplitMix64 finaliser).
  linalg      QR with positive diagonal, CholeskyQR2, exact traces.
  multigrid   aggregation prolongators, SAP smoothing, Galerkin coarse
              operators, the level hierarchy.
  estimators  plain Hutchinson (Algorithm 1), the MG-MLMC level differences,
              MG-MLMC++ (Algorithm 2) with direct solves.
  deflation   exactly deflated Hutchinson (Section 2): smallest singular
              triplets from the Hermitian gamma5 D, subspace iteration.
  nn          the learned gauge-covariant preconditioner (not in the paper):
              forward, backward, the tensor-core number format.
  tune_mass   bare-mass tuning of the benchmark fields (input preparation:
              m0 from the leftmost eigenvalue of D(0)).
"""
