"""Plain FP64 CPU oracle of the space-time Vanka-multigrid GMRES solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never calls it and shares no code
with it; the only module both sides use is ``stg_inputs`` (seeded synthetic
inputs, no solver arithmetic).

It follows the paper (Anselmann & Bause, "Efficiency of local Vanka smoother
geometric multigrid preconditioning for space-time finite element methods to
the Navier-Stokes equations"):

* ``timebasis``  -- Lagrange basis at the k+1 right Gauss-Radau points (Sec. 3).
* ``element``    -- Q2 / P1disc reference element and Gauss rules (Sec. 2).
* ``mesh``       -- structured level hierarchy and the map dof(K, mu) (Sec. 3).
* ``assemble``   -- the Newton/Oseen Jacobian of Eq. (3.3) with the blocks D_ab
                    and B_ab, built from A_h and B_GammaD of Sec. 2.
* ``vanka``      -- local matrices J_K, their LAPACK inverses and the averaged
                    smoothing loop (S0)-(S3) built on Eq. (3.4).
* ``transfer``   -- nested-space prolongation and its transpose.
* ``multigrid``  -- the V-cycle with a direct coarse solve on T_0.
* ``fgmres``     -- right-preconditioned flexible GMRES.
* ``newton``     -- nonlinear slab residual F_n, damped Newton (Sec. 3).
* ``functionals`` -- drag and lift on an obstacle (Sec. 4).
* ``cnn``        -- the warm-start network (3x3 convolutions, tanh, MSE loss,
                    Adam) and the next-slab features, targets and guess; the
                    paper has no learned part, its pins are closed forms.

Every part is pinned by the ``-m "not gpu"`` tests against closed forms,
invariants and brute-force dense linear algebra.
"""
from . import timebasis, element, mesh, assemble, vanka, transfer, multigrid, fgmres, newton, cnn, functionals  # noqa: F401
from .multigrid import Hierarchy  # noqa: F401
