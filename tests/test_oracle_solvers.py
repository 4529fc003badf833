"""Pins for the oracle's solvers (Section 5): MINRES preconditioned by one V-cycle.

References: numpy's dense solve, the explicit two-grid error-propagation formula, and symmetry / definiteness of
the V-cycle operator assembled column by column.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem, pbm, solvers


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * np.geomspace(1.0, cond, n)) @ Q.T


@pytest.mark.parametrize("seed", range(3))
def test_minres_spd_matches_dense_solve(seed):
    A = _spd(60, seed)
    b = np.random.default_rng(seed + 10).standard_normal(60)
    r = solvers.minres(lambda v: A @ v, b, rtol=1e-12, maxit=500)
    assert r.converged and r.relres <= 1e-12
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(r.x - x) <= 1e-8 * np.linalg.norm(x)


def test_minres_symmetric_indefinite_and_preconditioned():
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    ev = np.concatenate([-np.geomspace(1, 50, 20), np.geomspace(1, 100, 30)])
    A = (Q * ev) @ Q.T
    b = rng.standard_normal(50)
    r = solvers.minres(lambda v: A @ v, b, rtol=1e-11, maxit=500)
    assert r.converged
    assert np.allclose(r.x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-9)
    # SPD preconditioner M^{-1} = diag(1/|a_ii|) on an SPD matrix: fewer iterations than unpreconditioned
    B = _spd(80, 5, 1e4) + np.diag(np.geomspace(1, 1e4, 80))
    b = rng.standard_normal(80)
    Dinv = 1.0 / np.diag(B)
    r0 = solvers.minres(lambda v: B @ v, b, rtol=1e-10, maxit=2000)
    r1 = solvers.minres(lambda v: B @ v, b, lambda v: Dinv * v, rtol=1e-10, maxit=2000)
    assert r0.converged and r1.converged
    assert np.allclose(r1.x, np.linalg.solve(B, b), rtol=1e-7, atol=1e-9)


def test_minres_zero_rhs():
    A = _spd(10, 0)
    r = solvers.minres(lambda v: A @ v, np.zeros(10))
    assert r.converged and r.iters == 0 and np.all(r.x == 0)


def _S_problem(bc="cantilever", nx=4, ny=2, nz=2, seed=3):
    g = fem.Grid(nx, ny, nz, bc)
    f = synthetic.load_vector(nx, ny, nz, "end_edge")
    d = synthetic.random_state(nx, ny, nz, seed, u_scale=0.5, fixed_dofs=g.fixed_dofs())
    pb = pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"])
    st = pbm.State.from_dict(d)
    return pb, st, pbm.assemble_S(pb, st)


def _vcycle_matrix(h, n):
    return np.column_stack([h.vcycle(np.eye(n)[:, j]) for j in range(n)])


@pytest.mark.parametrize("levels", [2, 3])
def test_vcycle_is_symmetric_positive_definite(levels):
    pb, st, S = _S_problem(nx=8, ny=4, nz=4)
    h = solvers.Hierarchy(pb.grid, S, levels, has_alpha=True, sweeps=2)
    M = _vcycle_matrix(h, S.shape[0])
    assert np.max(np.abs(M - M.T)) < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


@pytest.mark.parametrize("levels", [2, 3])
def test_chebyshev_vcycle_is_symmetric_positive_definite(levels):
    pb, st, S = _S_problem(nx=8, ny=4, nz=4)
    h = solvers.Hierarchy(pb.grid, S, levels, has_alpha=True, sweeps=2, smoother="chebyshev")
    M = _vcycle_matrix(h, S.shape[0])
    assert np.max(np.abs(M - M.T)) < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


@pytest.mark.parametrize("steps", [1, 2, 3, 5])
def test_chebyshev_smoother_error_is_scaled_chebyshev_polynomial(steps):
    """On A = diag(lambda) with D = I, `steps` steps from x0 leave the error p(lambda) (x0 - x*) with
    p(lambda) = T_steps((theta - lambda) / delta) / T_steps(theta / delta), T the Chebyshev polynomial of the first
    kind: the defining property of Chebyshev acceleration (the polynomial of least maximum on the interval
    [theta - delta, theta + delta] among those with p(0) = 1)."""
    rng = np.random.default_rng(steps)
    lam = rng.uniform(0.05, 4.0, 40)
    A = sp.diags(lam)
    b = rng.standard_normal(40)
    x0 = rng.standard_normal(40)
    theta, delta = 2.0, 1.8
    x = solvers.chebyshev_smooth(A, np.ones(40), b, x0, theta, delta, steps)
    xs = b / lam
    T = lambda t: np.polynomial.chebyshev.chebval(t, [0.0] * steps + [1.0])
    p = T((theta - lam) / delta) / T(theta / delta)
    assert np.allclose(x - xs, p * (x0 - xs), rtol=1e-11, atol=1e-12)


def test_multicolour_gs_sweep_is_sequential_gauss_seidel_in_colour_order():
    """On an operator with one unknown per node (a scalar 27-point Q1 stencil: nodes of one colour share no element,
    so a colour has no internal coupling) a multicolour sweep equals the textbook Gauss-Seidel sweep on the
    unknowns ordered by colour: x + (L + D)^-1 (b - A x), L the strictly lower triangle in that order."""
    g = fem.Grid(5, 4, 3, "free")
    n = g.nnode
    rng = np.random.default_rng(3)
    rows, cols, vals = [], [], []
    ijk = g.node_ijk()
    for e in g.elem_nodes():
        w = rng.uniform(0.5, 1.5)
        for a in e:
            for b_ in e:
                rows.append(a)
                cols.append(b_)
                vals.append(w * (8.0 if a == b_ else -1.0))
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr() + sp.identity(n) * 0.1
    D = A.diagonal()
    colours = (ijk[:, 0] % 2) + 2 * (ijk[:, 1] % 2) + 4 * (ijk[:, 2] % 2)
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    x = solvers.multicolour_gs_sweep(A, D, b, x0, colours, range(8))
    perm = np.argsort(colours, kind="stable")
    Ap = A[perm][:, perm]
    LD = sp.tril(Ap, format="csr")
    xp = x0[perm] + spla.spsolve_triangular(LD, (b - A @ x0)[perm], lower=True)
    assert np.allclose(x[perm], xp, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("has_alpha", [False, True])
def test_dof_colouring_sweep_is_point_gauss_seidel_on_elasticity(has_alpha):
    """With the 24 dof colours (and alpha as the 25th) no two unknowns of a colour are coupled in K or S, so the
    multicolour sweep of the V-cycle is exactly point Gauss-Seidel on the unknowns ordered by colour."""
    if has_alpha:
        pb, st, A = _S_problem(nx=6, ny=4, nz=4)
        g = pb.grid
    else:
        g = fem.Grid(6, 4, 4, "bridge_corners")
        w = np.random.default_rng(2).uniform(1e-3, 1.0, g.m)
        A = fem.assemble_K(g, w, fem.element_stiffness())
    A = sp.csr_matrix(A)
    colours = solvers.node_colours(g, has_alpha)
    same = colours[:, None] == colours[None, :]
    Ad = A.toarray()
    assert np.all(Ad[same & ~np.eye(len(colours), dtype=bool)] == 0.0)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(A.shape[0])
    x0 = rng.standard_normal(A.shape[0])
    x = solvers.multicolour_gs_sweep(A, A.diagonal(), b, x0, colours, range(int(colours.max()) + 1))
    perm = np.argsort(colours, kind="stable")
    LD = sp.tril(A[perm][:, perm], format="csr")
    xp = x0[perm] + spla.spsolve_triangular(LD, (b - A @ x0)[perm], lower=True)
    assert np.allclose(x[perm], xp, rtol=1e-10, atol=1e-10 * np.abs(xp).max())


@pytest.mark.parametrize("levels", [2, 3])
def test_gauss_seidel_vcycle_is_symmetric_positive_definite(levels):
    pb, st, S = _S_problem(nx=8, ny=4, nz=4)
    h = solvers.Hierarchy(pb.grid, S, levels, has_alpha=True, sweeps=1, smoother="gauss_seidel")
    M = _vcycle_matrix(h, S.shape[0])
    assert np.max(np.abs(M - M.T)) < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_fixed_weight_06_is_indefinite_on_S():
    """Why the Jacobi weight is scaled by lambda_max: with a fixed 0.6, omega * lambda_max(D^-1 S) > 2 and the
    V-cycle loses definiteness, which MINRES reports as a breakdown."""
    pb, st, S = _S_problem(nx=8, ny=4, nz=4)
    h = solvers.Hierarchy(pb.grid, S, 2, has_alpha=True, omega=0.6, sweeps=2)
    M = _vcycle_matrix(h, S.shape[0])
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() < 0


def test_lanczos_lmax_estimate():
    pb, st, S = _S_problem(nx=8, ny=4, nz=4)
    A = S.toarray()
    D = np.diag(A)
    exact = np.linalg.eigvalsh(A / np.sqrt(D)[:, None] / np.sqrt(D)[None, :]).max()
    est = solvers.lanczos_lmax(S, D, 10)
    assert 0.97 * exact <= est <= exact * (1 + 1e-12)
    # on a diagonal matrix Lanczos is exact once it has seen every distinct eigenvalue
    Dg = sp.diags(np.array([1.0, 2.0, 3.0, 5.0]))
    assert abs(solvers.lanczos_lmax(Dg, np.ones(4), 4) - 5.0) < 1e-12


def test_two_grid_equals_textbook_error_propagation():
    """With an exact coarse solve, one two-grid cycle from x = 0 returns (I - E) A^{-1} b with
    E = (I - w D^-1 A)^nu2 (I - P Ac^-1 P^T A) (I - w D^-1 A)^nu1."""
    pb, st, S = _S_problem()
    h = solvers.Hierarchy(pb.grid, S, 2, has_alpha=True, omega=0.6, sweeps=2)
    A = S.toarray()
    n = A.shape[0]
    P = h.P[0].toarray()
    Ac = h.A[1].toarray()
    # coarse supported dofs were set to identity rows; P has zero columns there, so they decouple
    Sm = np.eye(n) - 0.6 * (A / np.diag(A)[:, None])
    C = np.eye(n) - P @ np.linalg.solve(Ac, P.T @ A)
    E = Sm @ Sm @ C @ Sm @ Sm
    b = np.random.default_rng(0).standard_normal(n)
    expect = (np.eye(n) - E) @ np.linalg.solve(A, b)
    assert np.allclose(h.vcycle(b), expect, rtol=1e-10, atol=1e-10 * np.abs(expect).max())


def test_galerkin_coarse_alpha_border_is_restricted_border():
    pb, st, S = _S_problem()
    h = solvers.Hierarchy(pb.grid, S, 2, has_alpha=True)
    n, nc = S.shape[0] - 1, h.A[1].shape[0] - 1
    Pu = h.P[0][:n, :nc]
    assert np.allclose(h.A[1][:nc, nc].toarray().ravel(), Pu.T @ S[:n, n].toarray().ravel(), atol=1e-14)
    assert h.A[1][nc, nc] == S[n, n]


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners"])
def test_mg_minres_solves_reduced_system(bc):
    pb, st, S = _S_problem(bc, 8, 4, 4, 1)
    rhs = pbm.rhs_closed(pb, st)
    h = solvers.Hierarchy(pb.grid, S, 3, has_alpha=True)
    assert all(0.1 < w < 0.6 for w in h.omega)
    r = solvers.minres(lambda v: S @ v, rhs, h.vcycle, rtol=1e-12, maxit=200)
    assert r.converged
    x = solvers.direct_solve(S, rhs)
    assert np.linalg.norm(r.x - x) <= 1e-9 * np.linalg.norm(x)
    assert r.iters < 60
    # the direct solve satisfies the system
    assert np.linalg.norm(S @ x - rhs) <= 1e-12 * np.linalg.norm(rhs)


def test_direct_solve_sparse_branch():
    g = fem.Grid(16, 8, 8, "cantilever")
    K = fem.assemble_K(g, np.full(g.m, 0.3), fem.element_stiffness())
    f = synthetic.load_vector(16, 8, 8, "end_edge")
    f[g.fixed_dofs()] = 0
    x = solvers.direct_solve(K, f)      # n = 4131 -> dense; force sparse by a larger grid below
    assert np.linalg.norm(K @ x - f) < 1e-12 * np.linalg.norm(f)
    g2 = fem.Grid(24, 12, 12, "cantilever")
    K2 = fem.assemble_K(g2, np.full(g2.m, 0.3), fem.element_stiffness())
    f2 = synthetic.load_vector(24, 12, 12, "end_edge")
    x2 = solvers.direct_solve(K2, f2)
    assert K2.shape[0] > 6000
    assert np.linalg.norm(K2 @ x2 - f2) < 1e-11 * np.linalg.norm(f2)
