"""ORACLE — plain, slow, FP64 CPU restatement of the method. Test infrastructure only.

This package is the independent reference that the CUDA library is checked
against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the library itself never does, and this package
imports nothing from the library. The two share no code: the only module both
sides use is ``synthetic`` (seeded random inputs, no method arithmetic).

What it restates (sections and equations of arXiv:1905.01348):

* ``discretization`` — Gamma-point planewave basis on the periodic cell (Sec. 2,
  Sec. 4 cutoff); real/reciprocal transforms with dense FFTs.
* ``exchange`` — the Fock exchange operator of Eq. 3 (pair densities, screened
  Coulomb convolution by FFT, full N_e^2 pair loop as in Alg. 2) and its
  adaptively compressed (ACE) form (cited in Sec. 1; formulas below).
* ``hamiltonian`` — the Hamiltonian of Eq. 2 with Gaussian-well ions, Hartree,
  (1 - alpha) Slater exchange and alpha Fock exchange; density (Sec. 3.4),
  total energy, dipole.
* ``ptcn`` — one parallel-transport Crank-Nicolson step (Eq. 4, Eq. 5,
  Alg. 1, residual of Alg. 3), per-band Anderson mixing (Sec. 3.4),
  Cholesky orthonormalisation (Sec. 3.4).

Every function cites the passage it follows. Readings of passages that are
silent or ambiguous are stated where they are used. All arithmetic is
complex128 / float64. Pinned by ``tests/test_oracle_*.py`` against closed
forms, brute force and invariants. The library's FP64 path is compared with it
at 1e-10 relative; its mixed-precision path (which the paper does not have) at
bounds derived from FP32 rounding for single operations and, over trajectories,
at the stated accuracy targets (dipole 1e-6 a.u., energy 1e-6 Ha per atom over
20 steps), see the test headers.
"""
