"""Plain, slow, obviously-correct FP64 CPU oracle for the per-time-step
modified-Helmholtz solve of Kropinski & Quaife (heat equation by Rothe's
method, Section 2; numerical methods, Section 3).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run it.  The CUDA library
(``paper_1007_5335_gb300``) never imports it and shares no code, table or
constant generator with it.

Modules
  special     K0, K1, I_n, K_n (library routines from scipy.special)
  quadrature  Gauss-Legendre rules, tensor Lagrange basis, trigonometric interpolation
  geometry    curves, spectral derivatives, normals, curvature, point classification
  alpert      hybrid Gauss-trapezoidal rule for log-singular integrands (loaded table)
  bie         Nystrom operator (eq. discrete_sys), dense GMRES, double-layer evaluation
  volume      direct volume potential with exact integrals of the leaf interpolant
  tree        adaptive quadtree, 2:1 balance and interaction lists
  step        IMEX (backward) Euler heat step (Section 2)
  pool        the independent per-target / per-row loops over spawned worker processes
  warmstart   learned initial guess for the boundary solve (Fourier features, MLP,
              closed-form start, Adam, minimum-residual judge)

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
closed forms, special cases and brute force (see each module's docstring).
Functions without such a pin say "parity unpinned" in their docstring.
"""
