"""Plain, slow FP64 CPU oracle for the block-sparse MPS eigensolver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA path (``paper_2604_16118_gb300``) and never
imports it; the only common dependency is the seeded input generator package
``synth``.

Modules (each function cites the part of the paper it follows):

* ``fermion``  -- Jordan--Wigner operators, the second-quantized Hamiltonian
  (Sec. 1.1, Eq. (hamil), (tvdef)) as a dense matrix on the N-particle
  subspace, and exact diagonalisation.
* ``mpo``      -- an exact matrix product operator for that Hamiltonian
  (Sec. 2.4, Thm. opranks) and its contraction to a dense matrix.
* ``bsmps``    -- block-sparse U(1) MPS (Sec. 2.3): sector sets, blocks,
  addition by block concatenation, exact operator application, inner
  products, orthogonalisation and trunc_eps (Sec. 2.2, Eq. (ttsvdquasiopt)).
* ``precond``  -- exponential-sum preconditioner (Sec. 4.2-4.3).
* ``pinvit``   -- one step of the perturbed inverse iteration (Alg. 2) with
  the adaptive residual (Sec. 5.3.1), the 2x2 Rayleigh--Ritz step (Remark
  omegamin) and the a-posteriori bounds (Sec. 5.4).
* ``joint``    -- joint block MPS of D vectors and the perturbed inverse
  subspace iteration (Alg. 4, Sec. 6).
* ``ozaki``    -- FP64 matrix product by exact integer slice products (the
  Ozaki scheme; not in the paper), pinned against exact rational arithmetic.
"""
