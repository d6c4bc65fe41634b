"""CPU oracle for the ParaDiag-II all-at-once solver (test infrastructure).

This package is the plain, slow, FP64 statement of what the GPU library
computes, written from the paper (Gander, Liu, Wu, Yue, Zhou, "ParaDiag:
Parallel-in-Time Algorithms Based on the Diagonalization Technique",
arXiv:2005.09158).  It is test infrastructure only: the tests, the smoke
check and the CPU-baseline leg of the benchmark import it; the product path
never does, and it shares no code with the CUDA library.

Modules
  operators     K (centred finite differences), the Toeplitz B1/B2 (eq. 2.5b,
                eq. 3.2b), the alpha-circulants C1/C2 (eq. 2.11b, eq. 3.4),
                apply-A (eq. 1.1) and the right-hand side b.
  stepping      O1: exact solution of A u = b by sequential block forward
                substitution in time; the adjoint by backward substitution.
  paradiag      O2: P_alpha^{-1} r by the three steps of eq. 1.3 with the
                Fourier matrix of Lemma 1 written out densely; the stationary
                iteration eq. 5.1; flexible GMRES on A with P_alpha^{-1}.
  dense         O3: dense Kronecker A and P_alpha for tiny sizes.
  closed_forms  O4: Lemma 1 eigenvalues, spatial eigenvalues, the per-mode
                contraction of eq. 5.1, the spectrum of Theorem 3.1.
  control       O5: the heat source inversion functional and its gradient.
  paradiag1     O6: ParaDiag-I with geometric time steps (Section 2.1.1):
                closed-form V, V^{-1}, the column scaling D~, the three steps
                of eq. 2.7, and the exact variable-step solution by stepping.
  hybrid        O7: ParaDiag-I with the hybrid midpoint + backward-Euler
                discretisation (Section 2.1.2): B, the Newton roots of the
                Chebyshev characteristic equation, the closed-form V, the
                three-step solve and the exact solution by a sparse LU.
  windows       O8: windowing -- consecutive windows chained from the last
                time level, each solved exactly.
  control_wave  O9: optimal control of the wave equation (Section 4): the
                saddle-point leap-frog system, the gamma-balanced block
                circulant preconditioner by Theorem 4, flexible GMRES.
  nonlinear     O10: U' + K U + phi(U) = f with a cubic reaction (eq. 1.4): the
                all-at-once residual, the exact solution by stepping with
                Newton per step, the simplified Newton iteration eq. 1.5 with
                the space-time averaged Jacobian K + sigma I.

Every function is pinned by a test in tests/test_oracle_*.py against a
closed form, an invariant, a bound of the paper, a worked example the paper
prints, or brute force.  No function here is parity-unpinned.
"""
