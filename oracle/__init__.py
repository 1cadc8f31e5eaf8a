"""CPU oracle for the space-time hp-DG Maxwell slab residual (test infrastructure).

This package is the plain, slow, FP64 statement of what the method computes,
written from the paper's definitions (Lilienthal, Schnepp, Weiland,
"Non-dissipative space-time hp-discontinuous Galerkin method for the
time-dependent Maxwell equations"):

  * basis.py     -- orthonormal Legendre polynomials on [0,1], integrated
                    Legendre polynomials, Gauss rules (Sec. 5.1 basis).
  * geometry.py  -- trilinear element maps, Jacobians, inverse maps
                    (Sec. 2.3 covariant transformation).
  * stdg.py      -- the bilinear form C_h + S_h and the load L by full
                    space-time tensor Gauss quadrature in physical space
                    (Eq. bilinearform:C, Eq. bilinearform:S), the residual
                    R_h = B_h - L (Eq. residual), sparse assembly, slab
                    solve, discrete energy (Eq. stability:energydef) and the
                    L2 projection of initial data.

It is test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may use it; the product path never
imports it and shares no code with it.
"""
