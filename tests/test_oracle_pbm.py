"""Pins for the oracle's PBM layer (Section 3): the penalty-barrier function eq. (103.1), the augmented Lagrangian
eq. (aug_lagr), its gradient and Hessian (eqs. lagr_grad_a, lagr_hess_a), the reduced Newton system eqs. (S),
(system), the nu-recovery eq. (deltanu), and Algorithms 1-2.

References other than the oracle itself: properties (phi1)-(phi4), finite differences of L, the explicit Schur
complement of the dense Hessian, the full (unreduced) Newton system solved densely, and an independent primal solve
of the convex minimum-compliance problem (eq. (1)) with scipy.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem, pbm


# ---------------------------------------------------------------------------------------------------------------
# penalty-barrier function
# ---------------------------------------------------------------------------------------------------------------

def test_phi_properties():
    assert pbm.phi(0.0) == 0.0                                           # (phi1)
    assert pbm.dphi(0.0) == 1.0                                          # (phi2)
    assert pbm.dphi(1e8) > 1e7                                           # (phi3), b = +inf
    assert 0 < pbm.dphi(-1e8) < 1e-8                                     # (phi4)
    t = np.linspace(-20, 5, 2001)
    assert np.all(np.diff(pbm.phi(t)) > 0)                               # strictly increasing
    assert np.all(pbm.ddphi(t) > 0)                                      # strictly convex


def test_phi_log_branch_closed_form_and_continuity():
    # with tau_hat = -1/2 the log branch is -1/4 log(-2 tau) - 3/8, derivative -1/(4 tau), second 1/(4 tau^2)
    t = np.array([-0.5000001, -0.7, -3.0, -1e3])
    assert np.allclose(pbm.phi(t), -0.25 * np.log(-2 * t) - 0.375, rtol=1e-14, atol=1e-15)
    assert np.allclose(pbm.dphi(t), -1 / (4 * t), rtol=1e-14)
    assert np.allclose(pbm.ddphi(t), 1 / (4 * t * t), rtol=1e-14)
    h = 1e-9
    for f in (pbm.phi, pbm.dphi, pbm.ddphi):
        assert abs(f(-0.5 - h) - f(-0.5 + h)) < 1e-8
    # derivative consistency by finite differences on both branches
    for x in (-2.0, -0.6, -0.4, 0.3, 2.0):
        e = 1e-6
        assert abs((pbm.phi(x + e) - pbm.phi(x - e)) / (2 * e) - pbm.dphi(x)) < 1e-8
        assert abs((pbm.dphi(x + e) - pbm.dphi(x - e)) / (2 * e) - pbm.ddphi(x)) < 1e-7


# ---------------------------------------------------------------------------------------------------------------
# gradient, Hessian, Schur complement
# ---------------------------------------------------------------------------------------------------------------

def _tiny(bc="cantilever", nx=2, ny=1, nz=1, seed=0, p=1.0, q=1.0, u_scale=1.0):
    g = fem.Grid(nx, ny, nz, bc)
    f = synthetic.load_vector(nx, ny, nz, "end_edge")
    d = synthetic.random_state(nx, ny, nz, seed, u_scale=u_scale, p=p, q=q, fixed_dofs=g.fixed_dofs())
    pb = pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"])
    return pb, pbm.State.from_dict(d)


def _pack(pb, st):
    free = np.flatnonzero(~pb.fixed)
    return np.concatenate([st.u[free], [st.alpha], st.nu_lo, st.nu_up]), free


def _unpack(pb, st, v, free):
    s = st.copy()
    nf, m = free.size, pb.m
    s.u = np.zeros(pb.n)
    s.u[free] = v[:nf]
    s.alpha = v[nf]
    s.nu_lo = v[nf + 1:nf + 1 + m].copy()
    s.nu_up = v[nf + 1 + m:].copy()
    return s


@pytest.mark.parametrize("seed,u_scale", [(0, 1.0), (1, 0.05), (2, 3.0)])
def test_gradient_matches_finite_differences(seed, u_scale):
    pb, st = _tiny(seed=seed, u_scale=u_scale)
    v, free = _pack(pb, st)
    g = pbm.gradient_dense(pb, st)
    h = 1e-6
    fd = np.empty_like(v)
    for k in range(v.size):
        e = np.zeros_like(v)
        e[k] = h
        fd[k] = (pbm.lagrangian(pb, _unpack(pb, st, v + e, free))
                 - pbm.lagrangian(pb, _unpack(pb, st, v - e, free))) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-6 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("seed,u_scale", [(0, 1.0), (3, 0.05)])
def test_hessian_matches_finite_differences(seed, u_scale):
    pb, st = _tiny(seed=seed, u_scale=u_scale)
    v, free = _pack(pb, st)
    H = pbm.hessian_dense(pb, st)
    h = 1e-6
    fd = np.empty_like(H)
    for k in range(v.size):
        e = np.zeros_like(v)
        e[k] = h
        fd[:, k] = (pbm.gradient_dense(pb, _unpack(pb, st, v + e, free))
                    - pbm.gradient_dense(pb, _unpack(pb, st, v - e, free))) / (2 * h)
    assert np.max(np.abs(fd - H)) < 1e-5 * max(1.0, np.abs(H).max())


def test_both_branches_exercised():
    pb, st = _tiny(nx=4, ny=2, nz=2, seed=5, u_scale=0.3)
    s = pbm.constraint_arg(pb, st)
    assert np.any(s < -0.5) and np.any(s >= -0.5)


@pytest.mark.parametrize("bc,seed,u_scale", [("cantilever", 0, 1.0), ("cantilever", 5, 0.3),
                                             ("bridge_corners", 7, 0.5)])
def test_closed_form_S_and_rhs_equal_dense_schur_complement(bc, seed, u_scale):
    pb, st = _tiny(bc, 4, 2, 2, seed, u_scale=u_scale)
    S_dense, rhs_dense = pbm.schur_dense(pb, st)
    free = np.flatnonzero(~pb.fixed)
    idx = np.concatenate([free, [pb.n]])
    S = pbm.assemble_S(pb, st).toarray()
    scale = np.abs(S_dense).max()
    assert np.max(np.abs(S[np.ix_(idx, idx)] - S_dense)) < 1e-12 * scale
    rhs = pbm.rhs_closed(pb, st)
    assert np.max(np.abs(rhs[idx] - rhs_dense)) < 1e-12 * max(1.0, np.abs(rhs_dense).max())
    # supported rows/cols are identity, rhs zero there
    fixed = np.flatnonzero(pb.fixed)
    assert np.allclose(S[np.ix_(fixed, fixed)], np.eye(fixed.size))
    assert np.all(rhs[fixed] == 0.0)
    # matrix-free application equals the assembled matrix
    x = np.random.default_rng(seed).standard_normal(pb.n + 1)
    assert np.allclose(pbm.apply_S_elementwise(pb, st, pbm.coeffs(pb, st), x), S @ x, rtol=1e-12, atol=1e-12)


def test_S_spd_and_sparsity():
    pb, st = _tiny("cantilever", 4, 2, 2, 4, u_scale=0.5)
    S = pbm.assemble_S(pb, st)
    assert abs(S - S.T).max() < 1e-13
    np.linalg.cholesky(S.toarray())
    # structural pattern of sum K_i: dof pairs that share an element (plus the identity on supported dofs)
    n = pb.n
    Kp = fem.assemble_unconstrained(pb.grid, np.ones(pb.m), np.ones((24, 24))).toarray() != 0
    Kp |= np.eye(n, dtype=bool)
    Su = S[:n, :n].toarray() != 0
    assert not np.any(Su & ~Kp)                  # u-block: sparsity of sum K_i (Section 3.2)
    border = S[:n, n].toarray().ravel()
    assert np.count_nonzero(border) > 0.5 * np.count_nonzero(~pb.fixed)


@pytest.mark.parametrize("seed,u_scale", [(0, 1.0), (6, 0.2)])
def test_reduced_solve_plus_nu_recovery_equals_full_newton(seed, u_scale):
    pb, st = _tiny("cantilever", 4, 2, 2, seed, u_scale=u_scale)
    H = pbm.hessian_dense(pb, st)
    g = pbm.gradient_dense(pb, st)
    full = np.linalg.solve(H, -g)
    cf = pbm.coeffs(pb, st)
    S = pbm.assemble_S(pb, st, cf)
    dz = np.linalg.solve(S.toarray(), pbm.rhs_closed(pb, st, cf))
    dl, du = pbm.delta_nu(pb, st, cf, dz)
    free = np.flatnonzero(~pb.fixed)
    red = np.concatenate([dz[free], [dz[pb.n]], dl, du])
    assert np.max(np.abs(red - full)) < 1e-10 * max(1.0, np.abs(full).max())


# ---------------------------------------------------------------------------------------------------------------
# Algorithms 1-2 against an independent primal solve
# ---------------------------------------------------------------------------------------------------------------

def _primal_reference(pb):
    """min_rho 1/2 f^T K(rho)^{-1} f  s.t. sum rho = V, rho_lo <= rho <= rho_up (eq. (1)), by SLSQP with the exact
    gradient -1/2 u^T K_i u."""
    def obj(r):
        K = fem.assemble_K(pb.grid, r, pb.Ke)
        u = spla.spsolve(K.tocsc(), pb.f)
        c = 0.5 * fem.element_energies(pb.grid, pb.Ke, u)
        return 0.5 * pb.f @ u, -c
    r0 = np.full(pb.m, pb.V / pb.m)
    res = so.minimize(obj, r0, jac=True, method="SLSQP", bounds=[(pb.rho_lo, pb.rho_up)] * pb.m,
                      constraints=[dict(type="eq", fun=lambda r: r.sum() - pb.V, jac=lambda r: np.ones_like(r))],
                      options=dict(ftol=1e-14, maxiter=2000))
    return res.x, res.fun


# ---------------------------------------------------------------------------------------------------------------
# the Newton stopping measure res_PBM (eq. resIP)
# ---------------------------------------------------------------------------------------------------------------

def test_res_pbm_hand_computed_state():
    """res_PBM on a 2x1x1 cantilever state whose three terms follow by hand from eq. (resIP), the gradient of
    eq. (lagr_grad_a) and the log branch of eq. (103.1) (tau_hat = -1/2: phi'(t) = -1/(4t)).

    u = 0, alpha = 1, nu_lo = nu_up = 1, p = q = 1, rho = 0.4, mu = 1, rho_lo = 1e-3, rho_up = 1, V = 0.6:
      * res_1 = -f (u = 0), so ||res_1|| / ||f|| = 1;
      * s_i = (0 - 1 + 1 - 1) / 1 = -1, phi'(-1) = 1/4, rho'_i = 0.1; res_2 = V - sum rho' = 0.4, |res_2| / V = 2/3;
      * mu'_lo = phi'(-1) = 1/4, res_3_i = -rho_lo + rho'_i - mu'_lo = -0.151 for both elements, so
        ||res_3|| / (||rho_lo e|| + ||rho_up e||) = 0.151 sqrt(2) / (1.001 sqrt(2)).
    A normalisation by m instead of ||.||_2 of the bound vectors, the +rho_lo sign printed in res_3, or res_4 in
    place of res_3 each change the value in the third digit."""
    g = fem.Grid(2, 1, 1, "cantilever")
    f = synthetic.load_vector(2, 1, 1, "end_edge")
    pb = pbm.Problem(g, f, 0.6, 1e-3, 1.0)
    m = g.m
    st = pbm.State(np.zeros(g.n), 1.0, np.ones(m), np.ones(m), np.full(m, 0.4), np.ones(m), np.ones(m))
    expected = 1.0 + 2.0 / 3.0 + 0.151 / 1.001
    assert abs(pbm.res_pbm(pb, st) - expected) < 1e-13 * expected


@pytest.mark.parametrize("seed,u_scale", [(0, 1.0), (4, 0.2)])
def test_res_pbm_from_finite_difference_gradient(seed, u_scale):
    """eq. (resIP) with res_1, res_2, res_3 taken as central finite differences of the augmented Lagrangian
    (not from the oracle's gradient): ||dL/du|| / ||f|| + |dL/dalpha| / V + ||dL/dnu_lo|| / (||rho_lo|| + ||rho_up||),
    the bound vectors of length m with 2-norms sqrt(m) |rho_lo|, sqrt(m) |rho_up|."""
    pb, st = _tiny(seed=seed, u_scale=u_scale)
    v, free = _pack(pb, st)
    h = 1e-6
    fd = np.empty_like(v)
    for k in range(v.size):
        e = np.zeros_like(v)
        e[k] = h
        fd[k] = (pbm.lagrangian(pb, _unpack(pb, st, v + e, free))
                 - pbm.lagrangian(pb, _unpack(pb, st, v - e, free))) / (2 * h)
    nf, m = free.size, pb.m
    r1, r2, r3 = fd[:nf], fd[nf], fd[nf + 1:nf + 1 + m]
    bound_norms = np.linalg.norm(np.full(m, pb.rho_lo)) + np.linalg.norm(np.full(m, pb.rho_up))
    expected = np.linalg.norm(r1) / np.linalg.norm(pb.f) + abs(r2) / pb.V + np.linalg.norm(r3) / bound_norms
    assert abs(pbm.res_pbm(pb, st) - expected) < 1e-7 * expected


def test_res_pbm_vanishes_at_a_stationary_point():
    """At a minimiser of the augmented Lagrangian (Newton with direct solves run to convergence) res_PBM is zero up
    to rounding, and so is the finite-difference gradient of L there."""
    nx, ny, nz = 4, 2, 2
    g = fem.Grid(nx, ny, nz, "cantilever")
    f = synthetic.load_vector(nx, ny, nz, "end_edge")
    pb = pbm.Problem(g, f, 0.3 * g.m, 1e-3, 1.0)
    m = g.m
    st0 = pbm.State(np.zeros(g.n), 1.0, np.ones(m), np.ones(m), np.full(m, 0.3), np.ones(m), np.ones(m))
    st, info, _ = pbm.newton(pb, st0, eps_nwt=1e-12, eps_mr=None, max_iter=60)
    assert pbm.res_pbm(pb, st) < 1e-11
    v, free = _pack(pb, st)
    h = 1e-6
    for k in np.random.default_rng(0).choice(v.size, 12, replace=False):
        e = np.zeros_like(v)
        e[k] = h
        d = (pbm.lagrangian(pb, _unpack(pb, st, v + e, free)) - pbm.lagrangian(pb, _unpack(pb, st, v - e, free)))
        assert abs(d / (2 * h)) < 1e-6
    # away from it the measure is not small
    assert pbm.res_pbm(pb, st0) > 0.1


# ---------------------------------------------------------------------------------------------------------------
# non-descent directions of inexact solves (Section 6) and their recovery
# ---------------------------------------------------------------------------------------------------------------

def _nondescent_case():
    """8x4x4 bridge, random state at penalties p = q = 1e-6 (late-PBM conditioning): the MINRES iterate at
    eps_MR = 0.5 is not a descent direction, the one at 0.05 is."""
    nx, ny, nz = 8, 4, 4
    g = fem.Grid(nx, ny, nz, "bridge_corners")
    f = synthetic.load_vector(nx, ny, nz, "top_traction")
    d = synthetic.random_state(nx, ny, nz, 9, u_scale=0.5, p=1e-6, q=1e-6, fixed_dofs=g.fixed_dofs())
    pb = pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"])
    return pb, pbm.State.from_dict(d)


def _fd_directional_derivative(pb, st, dz, dl, dup, h=1e-9):
    def L(t):
        s = st.copy()
        s.u = pbm.masked(pb, st.u + t * dz[:pb.n])
        s.alpha = st.alpha + t * dz[pb.n]
        s.nu_lo = st.nu_lo + t * dl
        s.nu_up = st.nu_up + t * dup
        return pbm.lagrangian(pb, s)
    return (L(h) - L(-h)) / (2 * h)


def test_loose_solve_gives_a_non_descent_direction():
    """The premise of the recovery, measured on L itself (central differences along the Newton direction, not the
    oracle's gradient): ascent at eps_MR = 0.5, descent at eps_MR = 0.05."""
    pb, st = _nondescent_case()
    cf = pbm.coeffs(pb, st)
    rhs = pbm.rhs_closed(pb, st, cf)
    signs = []
    for eps in (0.5, 0.05):
        dz, _ = pbm.solve_reduced(pb, st, cf, rhs, eps, 3)
        dl, dup = pbm.delta_nu(pb, st, cf, dz)
        signs.append(np.sign(_fd_directional_derivative(pb, st, dz, dl, dup)))
    assert signs == [1.0, -1.0]


def test_newton_recovers_from_a_non_descent_direction():
    """Algorithm 2 with the re-solve of Section 6's failure mode: one tightening (0.5 -> 0.05), then a descent
    step accepted by Armijo that lowers L."""
    pb, st = _nondescent_case()
    st1, info, eps = pbm.newton(pb, st, eps_nwt=0.0, eps_mr=0.5, levels=3, max_iter=1)
    assert info.resolves == 1 and abs(eps - 0.05) < 1e-15 and not info.stalled
    assert info.iters == 1 and info.slopes[0] < 0
    assert pbm.lagrangian(pb, st1) < pbm.lagrangian(pb, st)
    # at the floor there is no recovery: the loop stalls at the current iterate and leaves it unchanged
    st2, info2, _ = pbm.newton(pb, st, eps_nwt=0.0, eps_mr=0.5, levels=3, max_iter=1, eps_mr_min=0.5)
    assert info2.stalled and info2.iters == 0 and info2.resolves == 0
    assert np.array_equal(st2.u, st.u) and st2.alpha == st.alpha


@pytest.fixture(scope="module")
def pbm_run():
    nx, ny, nz = 4, 2, 2
    g = fem.Grid(nx, ny, nz, "cantilever")
    f = synthetic.load_vector(nx, ny, nz, "end_edge")
    pb = pbm.Problem(g, f, 0.3 * g.m, 1e-3, 1.0)
    return pb, pbm.pbm(pb, eps_pbm=1e-6)


def test_pbm_matches_independent_primal_solve(pbm_run):
    pb, res = pbm_run
    st = res.state
    _, comp_ref = _primal_reference(pb)
    comp = 0.5 * pb.f @ pbm.masked(pb, st.u)
    assert abs(comp - comp_ref) < 1e-4 * comp_ref
    # the PBM multiplier rho is the density (Theorem 1): its compliance equals the primal optimum
    K = fem.assemble_K(pb.grid, st.rho, pb.Ke)
    u_rho = spla.spsolve(K.tocsc(), pb.f)
    assert abs(0.5 * pb.f @ u_rho - comp_ref) < 1e-4 * comp_ref
    # dual objective at the optimum is -1/2 f^T u (Theorem 2 / eq. (gap))
    assert abs(pbm.dual_objective(pb, st) + comp_ref) < 1e-4 * comp_ref


def test_pbm_kkt_and_volume(pbm_run):
    pb, res = pbm_run
    st = res.state
    assert res.gap_ratio < 1e-6
    assert abs(st.rho.sum() - pb.V) / pb.V <= 1e-3          # volume error within 1 per mille (Section 6)
    assert np.all(st.rho >= pb.rho_lo * (1 - 1e-6)) and np.all(st.rho <= pb.rho_up * (1 + 1e-6))
    c = pbm.compliances(pb, st.u)
    inner = (st.rho > 1.01 * pb.rho_lo) & (st.rho < 0.99 * pb.rho_up)
    # c_i = alpha on elements strictly between the bounds
    assert np.all(np.abs(c[inner] - st.alpha) < 1e-2 * st.alpha)
    assert np.all(c[st.rho <= 1.01 * pb.rho_lo] <= st.alpha * (1 + 1e-2))
    assert np.all(c[st.rho >= 0.99 * pb.rho_up] >= st.alpha * (1 - 1e-2))
    assert res.newton >= res.outer >= 2
