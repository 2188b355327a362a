"""FP64 CPU oracle for the DG S_N transport sweep and the VEF closure pass.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this package.  The product path
(the CUDA library and its Python binding) never calls it and shares no code with it.

What it computes (plain, slow, FP64, NumPy + SciPy):
  * basis.py      1D Gauss-Lobatto / Gauss-Legendre rules and Lagrange bases
  * mesh.py       Q_m control points of the structured, sine-distorted mesh and the
                  geometric factors J, adj(F), n ds (paper Sec. "Mesh and Finite
                  Element Preliminaries")
  * transport.py  the upwind DG S_N operator L_d of each direction assembled as one
                  global sparse matrix and solved directly, psi_d = L_d^{-1} b_d
                  (paper Eq. transport / trans_bc with the DG space Y_p)
  * moments.py    phi, J, second moment P, Eddington tensor E, boundary factor E_b
                  and inflow partial current J_in (paper Eq. vef_disc and the
                  definitions that follow Eq. mlbc)
  * iteration.py  source iteration phi^{k+1} = sum_d w_d psi_d(phi^k)
  * adjoint.py    adjoint solves L_d^T lambda_d = w_d g and the sigma gradients
  * mms.py        the manufactured solution of the paper's MMS section
  * hrt.py        the hybridized Raviart-Thomas VEF discretisation: element-local
                  blocks, their elimination to the multiplier system H = C1 W C2,
                  the back substitution, and the global saddle-point solve
                  (paper Sec. "Hybridization")

The sweep's discrete equations are not written out in the paper (it defers to the
cited transport solvers).  The oracle follows the standard once-integrated upwind DG
weak form, with the upwind choice made pointwise at each face quadrature point.
No ordering, lagging or scheduling logic appears here: the result is the direct
solution of the global system.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, invariants, convergence orders and brute force; nothing here
is "parity unpinned".
"""
from . import basis, mesh, transport, moments, iteration, adjoint, mms, hrt  # noqa: F401
