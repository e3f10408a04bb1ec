"""Plain, slow FP64 CPU oracle for the implicit high-order Lagrangian hydrodynamics
residual, its Jacobian actions and the implicit Newton step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code, tables or constants with the CUDA
path: it builds its own quadrature rules, bases, mesh connectivity and physics.

Form of the oracle (see each module for the paper passage it follows):

* the discrete operators are formed from their definitions with dense per-element
  matrices (no sum factorisation, no fusion): Eq. (7) for M_V, M_E and F, with the
  quadrature-point stress of Eqs. (11), (13)-(20);
* the stage residual R(k; tau, u) of Eq. (21) at w = u + tau k;
* Jacobian actions by the complex-step derivative (exact to rounding for the analytic
  residual) and by central finite differences (Eq. (22) needs J = dR/dk);
* Newton with the backtracking line search of Sec. 3.5 and the implicit midpoint rule.

Parity status: every function is pinned by tests/test_oracle_*.py against closed forms,
invariants of the compatible discretisation and printed values of the paper; see the
module headers.
"""
