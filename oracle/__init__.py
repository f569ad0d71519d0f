"""Plain, slow FP64 CPU oracle of the space-time DG-SEM method (arXiv:2201.05800).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path (different formulas
for the LGL constants, the weak instead of the strong form of the spatial
operator, complex-step instead of dual-number derivatives).

Modules
-------
lgl      LGL nodes/weights, differentiation matrix, temporal SBP matrices and
         the Lobatto IIIC tableau obtained from them (Sec. 4, Eq. SBP_to_RK).
physics  Convective fluxes (linear advection, Euler, Burgers) and the Rusanov /
         upwind numerical flux (Eq. flux:llf).
dgsem    The spatial DG-SEM operator F = M^-1 L_h in weak form (Eqs. elementint,
         surfaceint, ode) on a periodic Cartesian grid.
stdg     Space-time residual (Eq. DG_vs_RK:DG), method-of-lines Lobatto IIIC
         residual (Eq. DG_vs_RK:RK), exact Jacobian-vector products, dense and
         Newton-GMRES slab solvers, slab marching, norms and conserved sums.

Every function is FP64 and written for a reader checking it against the paper.
Parity status: every function listed above is pinned by ``tests/test_oracle_*``
(closed forms, Appendix B/D values, Tables 1-2 convergence orders, exact
solutions, invariants, brute force).  The Burgers branch of ``physics`` is
pinned by a finite-difference flux derivative and by the characteristic
solution of smooth 1D Burgers (order N+1), ``stdg.lgl_weighted_norm`` by exact
integrals of constants and of polynomials within the LGL exactness
(``tests/test_oracle_burgers_norm.py``).
"""
