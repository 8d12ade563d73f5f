"""CTR-IBIM oracle: plain FP64 CPU implementation -- TEST INFRASTRUCTURE ONLY.

A slow, literal implementation of the corrected-trapezoidal implicit
boundary integral method for the linearized Poisson-Boltzmann equation
(Izzo, Zhong, Runborg, Tsai, arXiv 2210.03699), used to check the CUDA path.
Only tests/, __graft_entry__.smoke() and bench.py (its CPU-baseline and
reference arms) may import, call or build anything here.  It shares no code,
header, table or constant generator with the CUDA path; the only module both
use is `synthetic`, the seeded input generator.

Modules:
  native      gcc build + ctypes loader of csrc/oracle_sums.c (FP64 loops)
  tables      correction-weight tables by the limit of Eq. (2.29)
  geometry    tube, finite-difference geometry, Jacobian, weights (Sec. 2.1)
  correction  correction nodes and weights (Sec. 2.4, Eqs. (2.19)-(2.28))
  system      the discrete operator of Eq. (2.30), right-hand side Eq. (2.12)
  gmres       textbook GMRES (modified Gram-Schmidt, Givens rotations)
  energy      reaction potential Eq. (2.31) and polarization energy Eq. (3.3)
  exact       closed forms used as pins (sphere solution, Kirkwood energy)
  treecode    far-field acceleration of the dense sum (Sec. 2.5): Chebyshev
              interpolation on well-separated clusters of an integer octree

Every parity-relevant function names the passage it follows.  Parity
status of each function is listed in the module docstrings.
"""
