"""CPU float64 oracle for the boundary-element hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, dense restatement of what the GPU library
computes, used to prove the GPU results right.  Only the test-suite, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
may import it; the library itself never does, and the oracle imports nothing
from the library.  The two share no code: they only consume the same seeded
inputs from ``workloads``.

Method (lifted from the paper's 2-D TM system to three dimensions):
  * Galerkin discretisation of the single/double-layer operators (Sec. II,
    Eqs. 1-4) with piecewise-linear (RWG) bases on a triangulated boundary
    (Sec. III, the discretisation preceding Eq. 8);
  * the PMCHWT block system for a penetrable body (Eq. 7, its second and third
    rows, and the matrices P11..P22 listed after Eq. 8);
  * the free-space kernel, here the 3-D e^{-jkR}/(4 pi R) under the e^{+j w t}
    convention implied by H0^(2) in Sec. II and by the 1+j w tau Debye terms
    of Eq. 6;
  * a low-rank skeleton of well-separated blocks (the U V^T of Eq. 17), here by
    adaptive cross approximation.

Modules:
  quadrature  -- 7-point degree-5 triangle rule
  rwg         -- mesh -> RWG edge table
  potentials  -- closed-form integrals of R^-1, R, grad R^-1, grad R over a flat triangle
  operators   -- dense T_k, K_k, PMCHWT matrix, on-the-fly rows
  excitation  -- plane-wave right-hand sides
  power       -- absorbed / extinguished / scattered power
  mie         -- Mie series of a homogeneous and of a coated sphere (closed-form pins)
  multiregion -- layered bodies: PMCHWT written region by region
  tree        -- cluster tree and block partition
  aca         -- partial-pivot adaptive cross approximation
  debye       -- double-Debye permittivity (Eq. 6)
  planar      -- the paper's own two-dimensional TM pipeline: S, D, D*, N on a polygon,
                 PMCHWT, CFIE and its Calderon form, circulant counterpart, skeleton, Woodbury
"""
