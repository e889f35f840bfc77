"""CPU oracle for the preconditioned FR/CPR implicit hot path (Wang & Yu, arXiv 1903.06304).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct FP64 numpy code that
follows the paper's sections and equations step by step.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  It shares no code with the CUDA library: the only
shared module is the seeded input generator ``paper_1903_06304_gb300.inputs``,
which holds none of the method's arithmetic.

Every function accepts complex arrays so that exact directional derivatives can
be taken by the complex step (``abs``/``max``/``min`` branch on the real part).

Modules
-------
basis     Gauss points, Lagrange derivative/extrapolation, Radau corrections (Sec. 3.1)
physics   Eqs. convection, diffusion, shear_stress, jacobian, preconditioning,
          theta, eigenvalues(_para), eps_nonmove/eps_move, Rosanov (Secs. 2-3)
geometry  bilinear element map, metrics and grid velocity (Sec. 2.3)
residual  FR/CPR residual R(q^p), Eqs. cpr_ns / unsteady_pre_mov_cdomain_GCL (Sec. 3.1),
          far-field and adiabatic no-slip wall faces (Sec. 3.3), wall force (Sec. 4)
solver    JVP, element block Jacobian, restarted GMRES, BDF2 dual-time Newton and
          steady PTC with SER (Sec. 3.2); L2 and entropy errors (Sec. 4)
scale     per-equation residual magnitudes that parity tolerances are stated in (the
          summed-terms scale sigma and the flux-divergence scale)
adjoint   discrete adjoint of the BDF2 march for d(mean C_t)/d(plunge amplitude, Mach)
          of a plunging airfoil (Secs. 3.2, 4, 4.4; dense, small meshes)

Functions whose result is pinned by tests against the paper or mathematics are
listed in ``tests/test_oracle_*.py``.  Parity unpinned: none of the functions
above (the paper's tables need meshes that are not available and are not used).
"""
