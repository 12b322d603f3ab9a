"""Plain FP64 CPU oracle for the Jacobian-free Newton-Krylov loop of
Wang & Yu, "A comparative study of implicit Jacobian-free Rosenbrock-Wanner,
ESDIRK and BDF methods ... with high-order flux reconstruction" (arXiv 1904.04825).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no headers, tables or helpers); both sides take
their inputs from the seeded generators in ``synthetic``.

The oracle follows the paper's steps in its own notation, one function per
step, NumPy doing only library work (matrix products, dense solves, norms):

  basis      Gauss-Legendre points, Lagrange basis, Radau g_DG correction (Sec. 3)
  fr2d       Euler fluxes, Rusanov common flux, FR residual R(q) (Sec. 3, Eq. simplified_ode)
  ns2d       Navier-Stokes BR2 residual, walls, body force (Sec. 2-3)
  fr3d       3D Navier-Stokes FR residual on hexahedra, Taylor-Green
             dissipation rate (Sec. 3, Sec. 5)
  jfnk       FD Jacobian-vector product, brute-force Jacobian, element-Jacobi
             blocks, restarted right-preconditioned GMRES(m) (Sec. 4.5)
  tableaus   ROW / ESDIRK coefficient sets (Sec. 4.2, 4.3)
  steppers   ROW, ESDIRK + pseudo-transient continuation + SER, BDF2, SSPRK3 (Sec. 4.1-4.4)
  mlp        per-element MLP forward, backward, Adam (learned initial guess)
  vortex     exact isentropic vortex (Eq. VP_Solution) and the error norm of Sec. 5.1

Parity status of each function is stated in its module docstring; every
function listed above is pinned by a ``-m "not gpu"`` test against facts the
paper or mathematics fixes (see ``tests/test_oracle_*.py``).
"""
