"""FP64 CPU oracle for FPSA source iteration in 1D slab S_N (test infrastructure).

This package is the plain, slow, obviously-correct reference against which the
CUDA path is checked. It is TEST INFRASTRUCTURE ONLY: it may be imported by the
tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline / reference arm of
``bench.py``, and by nothing else. The product path (the C-ABI library and its
Python binding) never imports, links or calls anything in here, and this package
never imports the product path.

Everything is numpy / scipy in float64, written in the order and notation of
Patel, Warsa & Prinja, "Acceleration of the S_N equations with highly
anisotropic scattering using the Fokker-Planck equation" (arXiv:1907.13013):

- ``quadrature``  -- S_N Gauss-Legendre set, Legendre tables, the moment
  operators D and M (Eqs. phi-mom, treq), the MPD angular Laplacian (Eq. fp-mpd)
  and the WFD angular Laplacian (Eqs. fp-wdd, sph-weights, w_wfd).
- ``transport``   -- linear-discontinuous (LD) finite elements in space (Sec. 2.2,
  named but not written out in the paper; the Galerkin reading is stated in that
  module), the upwind per-ordinate sweep, and global sparse assembly of the
  streaming operator L_h, scattering operator S_h and Fokker-Planck operator F_h
  (Eqs. trop, fpop, fp-mpd-oper, wd-eq-oper).
- ``iterations``  -- source iteration (Eq. trsi), FPSA predict / correct /
  iterate (Eqs. predict, correct, iterate) with the FP operator solved by sparse
  LU as in Sec. 4, and the direct solve of the discrete system.
- ``adjoint``     -- sensitivities of the exit current (or of a linear functional
  of the flux moments) to every per-cell sigma_t and sigma_s,l, by implicit
  differentiation of the discrete solution (sparse LU of A^T).

Parity status of every function is stated in its docstring; every function here
is pinned by at least one test in ``tests/test_oracle_*.py`` against a closed
form, an invariant, a special case or brute force.
"""

from . import quadrature, transport, iterations, adjoint  # noqa: F401
