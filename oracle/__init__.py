"""FP64 CPU oracle for fast Fourier-Bessel steerable PCA (Zhao, Shkolnisky &
Singer, "Fast Steerable Principal Component Analysis").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (``paper_1412_0781_gb300``) and imports nothing
from it.

The oracle is deliberately plain and slow: every quantity is computed from its
definition in the paper, in float64, with numpy matrix products as the only
library primitive on the data path (plus ``numpy.linalg.eigh`` for the
symmetric eigenproblems):

* ``special``  Bessel functions J_k by Bessel's integral, their zeros by
  bracketing + bisection, Gauss-Legendre rules by Golub-Welsch + Newton.
* ``fb``       the sampling criterion and quadrature sizes (Sec. II-A,
  Alg. 1 step 1), the radial tables (Alg. 1 step 2), the polar Fourier
  transform as a DIRECT non-uniform DFT (Eq. nufft), the angular DFT as a
  plain sum (Eq. 1DFFT), the radial Gauss-Legendre quadrature (Eq. a), the
  steerable covariance (Eqs. cov, ck, ck_0), its eigendecomposition
  (Alg. 2 step 4), component selection / shrinkage (Eq. compselect), and the
  exact adjoint of the whole map plus an analytic synthesis (Eq. IFT_FB).

Parity status: every function is pinned in ``tests/test_oracle_pins.py`` by a
check that does not re-run the oracle's own formula (library special cases,
the paper's worked example, closed forms, group identities, brute force).
"""
