"""Plain FP64 CPU oracle for the even-odd staggered multi-shift CG path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import anything under oracle/.
The product path (the CUDA library and its Python binding) never calls it and
shares no code with it; both sides only share the seeded input generator
(paper_1710_09178_gb300/inputs.py), which holds none of the method's arithmetic.

Everything here is numpy complex128 / float64, written to be read against the
paper (Gupta & Majumdar, arXiv:1710.09178) line by line rather than to be fast:

  lattice.py   site address and even/odd ordering            (Section 2, Section 3.2)
  staggered.py staggered operator D, D_oe, D_eo, A = 4m^2 - D_eo D_oe  (Section 3.2)
  solvers.py   CG and the shifted (multi-shift) CG            (Section 4, ref. [mcg])
  rational.py  partial-fraction rational approximations       (Eq. ratapprx, Appendix)
  encode16.py  16-bit fixed-point colour-vector storage       (Section 5 "half precision")
  force.py     fermion force dS_f/dU of phi^dagger r(A) phi   (Section 3.1 MD equations)
  rhmc.py      gauge action and force, heatbath, Omelyan MD, Metropolis (Section 3.1)
  linkcomp.py  8-real and 16-bit compressed SU(3) link storage   (Section 5 outlook)
  cpp/         plain FP64 C++ twin of lattice/staggered/solvers/encode16 (one-core and
               OpenMP builds), bound by cpp_oracle.py: the host-core timings and the
               full-size solves come from it

Each function names the passage it follows.  Where the paper is silent or
ambiguous the oracle takes one stated reading, given in the docstring of the
module or function that depends on it.
Parity status: every function here is pinned by tests in tests/test_oracle_*.py
against closed forms, invariants, dense linear algebra or brute force.
"""

from . import lattice, staggered, solvers, rational, encode16, force, rhmc, linkcomp  # noqa: F401
