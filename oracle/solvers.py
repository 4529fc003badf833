"""Linear solvers of Section 5 (oracle; test infrastructure only).

  * `minres`      — preconditioned MINRES of Paige and Saunders: Lanczos with the preconditioner's inner product,
                    Givens QR of the tridiagonal matrix, three-term update of the search directions. Stops when the
                    true 2-norm residual satisfies ||b - A x|| <= rtol ||b|| (eq. cgstop; the norm is not named in
                    the paper, the 2-norm is the reading taken). The recurrence's residual estimate is only used to
                    decide when to look at the true residual.
  * `Hierarchy`   — geometric multigrid V-cycle (correction scheme) with Galerkin coarse operators
                    A_{k-1} = P^T A_k P, restriction = P^T, 27-point trilinear prolongation, identity transfer of the
                    extra unknown alpha (Section 5.2), damped Jacobi smoothing and an exact (Cholesky) solve on the
                    coarsest level. The paper smooths with Gauss-Seidel; damped Jacobi is a reading. Its weight on
                    level k is omega_k = theta / lambda_k, lambda_k the largest Ritz value of `lanczos_steps` Lanczos
                    steps on D_k^{-1/2} A_k D_k^{-1/2} from the normalised all-ones vector; theta = 1.2 restates the
                    weight 0.6 relative to the Jacobi stability limit 2 / lambda_max (a fixed 0.6 makes the V-cycle
                    indefinite on these operators, whose lambda_max(D^-1 A) is 3 to 13).
                    The Chebyshev variant (`smoother="chebyshev"`) replaces each smoothing pass of nu steps by nu
                    steps of Chebyshev acceleration of the Jacobi iteration (Saad, "Iterative Methods for Sparse
                    Linear Systems", Algorithm 12.1) on the interval [0.1, 1.4] lambda_k, which damps the upper
                    part of the spectrum of D_k^{-1} A_k; every eigenvalue up to (0.1 + 1.4) lambda_k is damped, so
                    the Lanczos estimate from below may be off by a third. The interval is a reading (the paper
                    smooths with Gauss-Seidel and names no polynomial smoother).
                    The Gauss-Seidel variant (`smoother="gauss_seidel"`, the paper's smoother made parallel) sweeps
                    24 dof colours 3 ((i mod 2) + 2 (j mod 2) + 4 (k mod 2)) + component (and, for S, the extra
                    unknown alpha as a 25th): x_c += D_c^-1 (b - A x)_c, colour after colour. Nodes of one node
                    colour share no element, so no two dofs of one colour are coupled and a sweep is point
                    Gauss-Seidel in the colour ordering. Pre-smoothing sweeps the colours forward, post-smoothing
                    backward, which keeps the V-cycle symmetric.
  * `direct_solve`— sparse LU (scipy SuperLU) or dense solve.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def direct_solve(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    if A.shape[0] <= 6000:
        return np.linalg.solve(A.toarray(), b)
    return spla.splu(A.tocsc(), permc_spec="COLAMD").solve(b)


@dataclass
class MinresResult:
    x: np.ndarray
    iters: int
    relres: float       # true ||b - A x|| / ||b||
    converged: bool
    breakdown: bool = False   # v^T M^{-1} v < 0: the preconditioner is not positive definite


def minres(A, b: np.ndarray, M=None, rtol: float = 1e-8, maxit: int = 1000, x0: np.ndarray | None = None
           ) -> MinresResult:
    """Preconditioned MINRES for symmetric A and symmetric positive definite M^{-1} (callables)."""
    M = (lambda v: v.copy()) if M is None else M
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return MinresResult(x, 0, 0.0, True)
    r = b - A(x)
    # Lanczos vectors in the unpreconditioned space: v_prev, v_cur; z = M^{-1} v
    v_prev = np.zeros_like(b)
    v_cur = r.copy()
    z = M(v_cur)
    if float(v_cur @ z) < 0.0:
        return MinresResult(x, 0, float(np.linalg.norm(r)) / bnorm, False, True)
    beta_cur = math.sqrt(float(v_cur @ z))
    if beta_cur == 0.0:
        return MinresResult(x, 0, float(np.linalg.norm(r)) / bnorm, bool(np.linalg.norm(r) <= rtol * bnorm))
    beta_prev = 0.0
    # Givens rotation state and the (preconditioned) residual-norm estimate eta
    c_prev, s_prev, c_cur, s_cur = 1.0, 0.0, 1.0, 0.0
    eta = beta_cur
    eta0 = beta_cur
    d_prev = np.zeros_like(b)   # search directions d_{k-1}, d_{k-2}
    d_prev2 = np.zeros_like(b)
    target = rtol           # relative target on the estimate; tightened if the true residual lags behind
    relres = float("inf")
    for it in range(1, maxit + 1):
        q = z / beta_cur                       # preconditioned Lanczos vector
        Aq = A(q)
        a_k = float(Aq @ q)                    # diagonal of the Lanczos tridiagonal
        v_next = Aq - (a_k / beta_cur) * v_cur - ((beta_cur / beta_prev) * v_prev if beta_prev > 0 else 0.0)
        z_next = M(v_next)
        vz = float(v_next @ z_next)
        if vz < 0.0:
            return MinresResult(x, it - 1, float(np.linalg.norm(b - A(x))) / bnorm, False, True)
        beta_next = math.sqrt(vz)
        # apply the two previous rotations to the new column (beta_cur, a_k, beta_next) of the tridiagonal
        e_k = s_prev * beta_cur                          # entry two above the diagonal
        g_tmp = c_prev * beta_cur                        # entry one above, before the latest rotation
        f_k = c_cur * g_tmp + s_cur * a_k                # entry one above the diagonal
        g_k = -s_cur * g_tmp + c_cur * a_k               # diagonal before the new rotation
        r_k = math.hypot(g_k, beta_next)                 # diagonal after the new rotation
        if r_k == 0.0:
            break
        c_new, s_new = g_k / r_k, beta_next / r_k
        d_new = (q - e_k * d_prev2 - f_k * d_prev) / r_k
        x = x + (c_new * eta) * d_new
        eta = -s_new * eta
        # shift
        d_prev2, d_prev = d_prev, d_new
        c_prev, s_prev, c_cur, s_cur = c_cur, s_cur, c_new, s_new
        v_prev, v_cur, z = v_cur, v_next, z_next
        beta_prev, beta_cur = beta_cur, beta_next
        if abs(eta) <= target * eta0 or beta_next == 0.0:
            relres = float(np.linalg.norm(b - A(x))) / bnorm
            if relres <= rtol or beta_next == 0.0:
                return MinresResult(x, it, relres, relres <= rtol)
            target = target * 0.5 * rtol / relres
    relres = float(np.linalg.norm(b - A(x))) / bnorm
    return MinresResult(x, it, relres, relres <= rtol)


def lanczos_lmax(A: sp.spmatrix, D: np.ndarray, steps: int = 10) -> float:
    """Largest Ritz value of `steps` Lanczos steps on D^{-1/2} A D^{-1/2}, started from the normalised all-ones
    vector (an estimate from below of lambda_max(D^{-1} A))."""
    n = A.shape[0]
    s = 1.0 / np.sqrt(D)
    v = np.full(n, 1.0 / math.sqrt(n))
    v_prev = np.zeros(n)
    beta = 0.0
    al, be = [], []
    for _ in range(steps):
        w = s * (A @ (s * v))
        a = float(w @ v)
        w = w - a * v - beta * v_prev
        al.append(a)
        beta = float(np.linalg.norm(w))
        if beta == 0.0:
            break
        be.append(beta)
        v_prev, v = v, w / beta
    k = len(al)
    T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
    return float(np.linalg.eigvalsh(T).max())


class Hierarchy:
    """Galerkin hierarchy on CSR matrices. Level 0 is the finest."""

    def __init__(self, grid: fem.Grid, A: sp.spmatrix, levels: int, has_alpha: bool, omega: float | None = None,
                 sweeps: int = 2, post_sweeps: int | None = None, theta: float = 1.2, lanczos_steps: int = 10,
                 smoother: str = "jacobi"):
        if smoother not in ("jacobi", "chebyshev", "gauss_seidel"):
            raise ValueError(smoother)
        self.smoother = smoother
        self.nu1 = sweeps
        self.nu2 = sweeps if post_sweeps is None else post_sweeps
        self.has_alpha = has_alpha
        self.grids = [grid]
        self.A = [A.tocsr()]
        self.P = []
        for _ in range(levels - 1):
            g = self.grids[-1]
            P = fem.prolongation(g)
            gc = g.coarse()
            if has_alpha:
                P = sp.block_diag([P, sp.identity(1)]).tocsr()
            Ac = (P.T @ self.A[-1] @ P).tocsr()
            fixed_c = gc.fixed_dofs()
            if has_alpha:
                fixed_c = np.concatenate([fixed_c, [False]])
            Ac = (Ac + sp.diags(fixed_c.astype(float))).tocsr()
            self.P.append(P)
            self.A.append(Ac)
            self.grids.append(gc)
        self.D = [Ak.diagonal() for Ak in self.A]
        if omega is None or smoother == "chebyshev":
            self.lmax = [lanczos_lmax(Ak, Dk, lanczos_steps) for Ak, Dk in zip(self.A[:-1], self.D[:-1])]
        if omega is None:
            self.omega = [theta / lm for lm in self.lmax]
        else:
            self.omega = [omega] * (len(self.A) - 1)
        if smoother == "gauss_seidel":
            self.colours = [node_colours(gk, has_alpha) for gk in self.grids]
        if smoother == "chebyshev":
            # eigenvalue interval [lo, hi] of D^-1 A that the polynomial damps: centre and half width
            self.cheb = [((0.1 * lm + 1.4 * lm) / 2.0, (1.4 * lm - 0.1 * lm) / 2.0) for lm in self.lmax]
        self.coarse_chol = sla.cho_factor(self.A[-1].toarray(), lower=True)

    def vcycle(self, b: np.ndarray, k: int = 0) -> np.ndarray:
        if k == len(self.A) - 1:
            return sla.cho_solve(self.coarse_chol, b)
        A, D, w = self.A[k], self.D[k], self.omega[k]
        if self.smoother == "gauss_seidel":
            ncol = int(self.colours[k].max()) + 1
            x = np.zeros_like(b)
            for _ in range(self.nu1):
                x = multicolour_gs_sweep(A, D, b, x, self.colours[k], range(ncol))
            r = b - A @ x
            xc = self.vcycle(self.P[k].T @ r, k + 1)
            x = x + self.P[k] @ xc
            for _ in range(self.nu2):
                x = multicolour_gs_sweep(A, D, b, x, self.colours[k], range(ncol - 1, -1, -1))
            return x
        if self.smoother == "chebyshev":
            x = chebyshev_smooth(A, D, b, np.zeros_like(b), *self.cheb[k], self.nu1)
        else:
            x = w * b / D
            for _ in range(self.nu1 - 1):
                x = x + w * (b - A @ x) / D
        r = b - A @ x
        xc = self.vcycle(self.P[k].T @ r, k + 1)
        x = x + self.P[k] @ xc
        if self.smoother == "chebyshev":
            return chebyshev_smooth(A, D, b, x, *self.cheb[k], self.nu2)
        for _ in range(self.nu2):
            x = x + w * (b - A @ x) / D
        return x


def node_colours(grid: fem.Grid, has_alpha: bool) -> np.ndarray:
    """Colour of every unknown: 3 (node colour) + component, the node colour (i mod 2) + 2 (j mod 2) + 4 (k mod 2);
    24 for alpha."""
    ijk = grid.node_ijk()
    c = (ijk[:, 0] % 2) + 2 * (ijk[:, 1] % 2) + 4 * (ijk[:, 2] % 2)
    c = (3 * c[:, None] + np.arange(3)[None, :]).ravel()
    return np.concatenate([c, [24]]) if has_alpha else c


def multicolour_gs_sweep(A, D: np.ndarray, b: np.ndarray, x: np.ndarray, colours: np.ndarray, order) -> np.ndarray:
    """One multicolour Gauss-Seidel sweep: for each colour c in `order`, x_c += D_c^-1 (b - A x)_c."""
    for c in order:
        r = b - A @ x
        x = x + np.where(colours == c, r / D, 0.0)
    return x


def chebyshev_smooth(A, D: np.ndarray, b: np.ndarray, x: np.ndarray, theta: float, delta: float,
                     steps: int) -> np.ndarray:
    """`steps` steps of Chebyshev acceleration of the Jacobi iteration for A x = b from x (Saad, Algorithm 12.1,
    preconditioner D): the eigenvalues of D^-1 A in [theta - delta, theta + delta] are damped by the Chebyshev
    polynomial of degree `steps` scaled to 1 at zero."""
    if steps <= 0:
        return x
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - A @ x
    d = r / D / theta
    x = x + d
    for _ in range(steps - 1):
        r = b - A @ x
        rho_next = 1.0 / (2.0 * sigma - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * (r / D)
        x = x + d
        rho = rho_next
    return x
