"""CPU oracle for the reduced-Newton MG-MINRES path (test infrastructure only).

This package is a plain, slow, float64 restatement of what the paper defines, written with numpy/scipy so that a
reader can check it against the paper by eye. It is used ONLY by `tests/`, by `__graft_entry__.smoke()` and by the
CPU-baseline leg of `bench.py`. The product path (the CUDA library and its Python binding) never imports it, and it
imports nothing from the product path.

Modules
  fem      : Q1 hexahedral elasticity on a structured grid (Section 5.2 / Section 6): element stiffness by Gauss
             quadrature, node/element/dof maps, supports, CSR assembly of K(w) = sum_i w_i K_i (eq. (1)),
             trilinear (27-point) prolongation.
  pbm      : penalty-barrier function (eq. (103.1)), augmented Lagrangian of the dual VTS problem (eq. aug_lagr),
             its gradient and Hessian (eqs. lagr_grad_a, lagr_hess_a), the reduced Newton matrix S (eq. S), its
             right-hand side (eq. system), the recovery of the nu-step (eq. deltanu), the duality gap (eq. gap),
             Newton (Algorithm 2) and the outer PBM loop (Algorithm 1).
  solvers  : preconditioned MINRES (Paige-Saunders), a Galerkin V-cycle on CSR (Section 5.1), direct solves.
  doc      : the damped optimality-criteria method (Algorithm DOC): equilibrium solve and the bisection of the
             volume multiplier.
  ip       : the primal-dual interior-point method's Newton system (Section 4.1): perturbed KKT residual, its
             Jacobian (eq. gradres), the reduced matrix (eq. S_IP), its right-hand side and the recovery of the
             density and multiplier increments (eqs. Delta_rho, Delta_onu, Delta_unu).

Every function is pinned by a `-m "not gpu"` test against something other than itself (closed forms, invariants,
brute force, the paper's printed problem dimensions); see tests/test_oracle_*.py.
"""
