"""Penalty-barrier multiplier (PBM) method for the dual VTS problem (oracle; test infrastructure only).

Written from Section 3 of the paper. Variables xi = (u, alpha, nu_lo, nu_up); multipliers (rho, mu_lo, mu_up);
penalties p, q_lo, q_up (scalars: they start at 1 and are updated uniformly, Algorithm 1).

Readings of the paper taken here, where it is silent or inconsistent (the CUDA path takes the same ones):
  * tau_hat = -1/2 in eq. (103.1) (the "pure logarithmic branch" the paper says it uses).
  * The nu-gradient signs are derived from the augmented Lagrangian eq. (aug_lagr) itself:
        dL/dnu_lo_i = -rho_lo_i + rho'_i - mu'_lo_i,     dL/dnu_up_i = rho_up_i - rho'_i - mu'_up_i
    (eq. lagr_grad_a prints +rho_lo in res_3).
  * The mu_lo multiplier update of Algorithm 1 uses phi'(-nu_lo/q_lo), consistent with h_lo = phi(-nu_lo/q_lo)
    and with the generic rule eq. (106) (Algorithm 1 prints phi'(nu_lo/q_lo)).
  * Supported dofs are eliminated; u has zeros there and every K_i u is restricted to the free dofs.
  * Armijo constants (not given): c1 = 1e-4, halving, kappa0 = 1, at most 30 halvings.
  * Non-descent directions (Section 6, the discussion of the BRIDGE examples with 7 levels: inexact solves of eq.
    (system) stopped being descent directions and the method stalled there). When grad L^T dxi >= 0 the reduced
    system is solved again from zero with eps_MR tightened tenfold, down to the floor eps_mr_min of Section 5.3; a
    direction that is still not one of descent at the floor ends the Newton loop at the current iterate (a stall,
    which the paper accepted as the nearly optimal solution).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import fem
from . import solvers

TAU_HAT = -0.5

# ----------------------------------------------------------------------------------------------------------------
# penalty-barrier function, eq. (103.1) with tau_hat = -1/2
# ----------------------------------------------------------------------------------------------------------------


def phi(t):
    t = np.asarray(t, dtype=np.float64)
    th = TAU_HAT
    quad = t + 0.5 * t * t
    with np.errstate(divide="ignore", invalid="ignore"):
        logb = -(1.0 + th) ** 2 * np.log((1.0 + 2.0 * th - t) / (1.0 + th)) + th + 0.5 * th * th
    return np.where(t >= th, quad, logb)


def dphi(t):
    t = np.asarray(t, dtype=np.float64)
    th = TAU_HAT
    with np.errstate(divide="ignore", invalid="ignore"):
        logb = (1.0 + th) ** 2 / (1.0 + 2.0 * th - t)
    return np.where(t >= th, 1.0 + t, logb)


def ddphi(t):
    t = np.asarray(t, dtype=np.float64)
    th = TAU_HAT
    with np.errstate(divide="ignore", invalid="ignore"):
        logb = (1.0 + th) ** 2 / (1.0 + 2.0 * th - t) ** 2
    return np.where(t >= th, np.ones_like(t), logb)


# ----------------------------------------------------------------------------------------------------------------
# problem and state
# ----------------------------------------------------------------------------------------------------------------


@dataclass
class Problem:
    grid: fem.Grid
    f: np.ndarray
    V: float
    rho_lo: float
    rho_up: float
    E: float = 1.0
    nu: float = 0.3

    def __post_init__(self):
        self.Ke = fem.element_stiffness(self.E, self.nu, self.grid.h)
        self.fixed = self.grid.fixed_dofs()
        self.dofs = self.grid.elem_dofs()
        self.f = np.where(self.fixed, 0.0, self.f)

    @property
    def m(self):
        return self.grid.m

    @property
    def n(self):
        return self.grid.n


@dataclass
class State:
    u: np.ndarray
    alpha: float
    nu_lo: np.ndarray
    nu_up: np.ndarray
    rho: np.ndarray
    mu_lo: np.ndarray
    mu_up: np.ndarray
    p: float = 1.0
    q_lo: float = 1.0
    q_up: float = 1.0

    def copy(self):
        return State(self.u.copy(), float(self.alpha), self.nu_lo.copy(), self.nu_up.copy(), self.rho.copy(),
                     self.mu_lo.copy(), self.mu_up.copy(), self.p, self.q_lo, self.q_up)

    @staticmethod
    def from_dict(d: dict) -> "State":
        return State(np.array(d["u"], dtype=float), float(d["alpha"]), np.array(d["nu_lo"], dtype=float),
                     np.array(d["nu_up"], dtype=float), np.array(d["rho"], dtype=float),
                     np.array(d["mu_lo"], dtype=float), np.array(d["mu_up"], dtype=float), float(d["p"]),
                     float(d["q_lo"]), float(d["q_up"]))


def masked(pb: Problem, u: np.ndarray) -> np.ndarray:
    return np.where(pb.fixed, 0.0, u)


def element_w(pb: Problem, u: np.ndarray) -> np.ndarray:
    """(m, 24) local vectors w_e = K_e u_e, with the supported dofs zeroed (K_i u restricted to free dofs)."""
    um = masked(pb, u)
    w = um[pb.dofs] @ pb.Ke
    return np.where(pb.fixed[pb.dofs], 0.0, w)


def compliances(pb: Problem, u: np.ndarray) -> np.ndarray:
    """c_i = 1/2 u^T K_i u."""
    um = masked(pb, u)
    return 0.5 * fem.element_energies(pb.grid, pb.Ke, um)


# ----------------------------------------------------------------------------------------------------------------
# augmented Lagrangian eq. (aug_lagr), gradient (eq. lagr_grad_a), Hessian (eq. lagr_hess_a)
# ----------------------------------------------------------------------------------------------------------------


def constraint_arg(pb: Problem, st: State, c: np.ndarray | None = None) -> np.ndarray:
    """s_i = (1/2 u^T K_i u - alpha + nu_lo_i - nu_up_i) / p."""
    if c is None:
        c = compliances(pb, st.u)
    return (c - st.alpha + st.nu_lo - st.nu_up) / st.p


def lagrangian(pb: Problem, st: State) -> float:
    um = masked(pb, st.u)
    s = constraint_arg(pb, st)
    val = st.alpha * pb.V - pb.f @ um - pb.rho_lo * st.nu_lo.sum() + pb.rho_up * st.nu_up.sum()
    val += np.sum(st.rho * st.p * phi(s))
    val += np.sum(st.mu_lo * st.q_lo * phi(-st.nu_lo / st.q_lo))
    val += np.sum(st.mu_up * st.q_up * phi(-st.nu_up / st.q_up))
    return float(val)


@dataclass
class Coeffs:
    """Per-element derivative factors of Section 3.2 (after eq. lagr_grad_a)."""
    c: np.ndarray        # 1/2 u^T K_i u
    s: np.ndarray        # argument of phi in g_i
    rho1: np.ndarray     # rho'  = rho phi'(s)
    rho2: np.ndarray     # rho'' = (rho/p) phi''(s)
    mul1: np.ndarray     # mu'_lo  = mu_lo phi'(-nu_lo/q_lo)
    mul2: np.ndarray     # mu''_lo = (mu_lo/q_lo) phi''(-nu_lo/q_lo)
    muu1: np.ndarray
    muu2: np.ndarray
    gl: np.ndarray       # dL/dnu_lo
    gu: np.ndarray       # dL/dnu_up
    det: np.ndarray      # det of the per-element 2x2 (nu_lo, nu_up) Hessian block
    d: np.ndarray        # Schur weight d_i = rho'' mu''_lo mu''_up / det
    eps: np.ndarray      # rhs weight eps_i = rho'' (mu''_up gl - mu''_lo gu) / det


def coeffs(pb: Problem, st: State) -> Coeffs:
    c = compliances(pb, st.u)
    s = constraint_arg(pb, st, c)
    rho1 = st.rho * dphi(s)
    rho2 = st.rho / st.p * ddphi(s)
    tl, tu = -st.nu_lo / st.q_lo, -st.nu_up / st.q_up
    mul1, mul2 = st.mu_lo * dphi(tl), st.mu_lo / st.q_lo * ddphi(tl)
    muu1, muu2 = st.mu_up * dphi(tu), st.mu_up / st.q_up * ddphi(tu)
    gl = -pb.rho_lo + rho1 - mul1
    gu = pb.rho_up - rho1 - muu1
    det = rho2 * (mul2 + muu2) + mul2 * muu2
    d = rho2 * mul2 * muu2 / det
    eps = rho2 * (muu2 * gl - mul2 * gu) / det
    return Coeffs(c, s, rho1, rho2, mul1, mul2, muu1, muu2, gl, gu, det, d, eps)


def gradient(pb: Problem, st: State, cf: Coeffs | None = None):
    """(g_u (n), g_alpha, g_nu_lo (m), g_nu_up (m)) — gradient of the augmented Lagrangian, supported dofs zero."""
    cf = coeffs(pb, st) if cf is None else cf
    um = masked(pb, st.u)
    gu_vec = -pb.f + fem.apply_K_elementwise(pb.grid, cf.rho1, pb.Ke, um)
    gu_vec = np.where(pb.fixed, 0.0, gu_vec)
    galpha = pb.V - cf.rho1.sum()
    return gu_vec, float(galpha), cf.gl.copy(), cf.gu.copy()


def hessian_dense(pb: Problem, st: State) -> np.ndarray:
    """Dense Hessian of the augmented Lagrangian over the free dofs, alpha, nu_lo, nu_up (tiny grids only).
    Blocks exactly as eq. (lagr_hess_a)."""
    cf = coeffs(pb, st)
    free = np.flatnonzero(~pb.fixed)
    nf, m = free.size, pb.m
    W = element_w(pb, st.u)                         # (m, 24) local K_e u_e (free dofs only)
    G = np.zeros((pb.n, m))                         # column i = K_i u (global)
    for i in range(m):
        np.add.at(G[:, i], pb.dofs[i], W[i])
    G = G[free]
    K1 = fem.assemble_unconstrained(pb.grid, cf.rho1, pb.Ke).toarray()[np.ix_(free, free)]
    N = nf + 1 + 2 * m
    H = np.zeros((N, N))
    ia, il, iu = nf, nf + 1, nf + 1 + m
    H[:nf, :nf] = (G * cf.rho2) @ G.T + K1                     # H11
    H[:nf, ia] = H[ia, :nf] = -(G @ cf.rho2)                    # H12
    H[:nf, il:il + m] = G * cf.rho2                             # H13
    H[il:il + m, :nf] = (G * cf.rho2).T
    H[:nf, iu:iu + m] = -G * cf.rho2                            # H14
    H[iu:iu + m, :nf] = -(G * cf.rho2).T
    H[ia, ia] = cf.rho2.sum()                                   # H22
    H[ia, il:il + m] = H[il:il + m, ia] = -cf.rho2              # H23
    H[ia, iu:iu + m] = H[iu:iu + m, ia] = cf.rho2               # H24
    H[il:il + m, il:il + m] = np.diag(cf.rho2 + cf.mul2)        # H33
    H[il:il + m, iu:iu + m] = H[iu:iu + m, il:il + m] = np.diag(-cf.rho2)   # H34
    H[iu:iu + m, iu:iu + m] = np.diag(cf.rho2 + cf.muu2)        # H44
    return H


def gradient_dense(pb: Problem, st: State) -> np.ndarray:
    gu_vec, ga, gl, gu = gradient(pb, st)
    free = np.flatnonzero(~pb.fixed)
    return np.concatenate([gu_vec[free], [ga], gl, gu])


def schur_dense(pb: Problem, st: State):
    """S and rhs of eq. (S)/(system) by explicit Schur complement of the dense Hessian (tiny grids only).
    Returned over (free dofs, alpha)."""
    H = hessian_dense(pb, st)
    g = gradient_dense(pb, st)
    nz = int((~pb.fixed).sum()) + 1
    Hzz, Hzn, Hnn = H[:nz, :nz], H[:nz, nz:], H[nz:, nz:]
    Hnn_inv = np.linalg.inv(Hnn)
    S = Hzz - Hzn @ Hnn_inv @ Hzn.T
    rhs = -g[:nz] + Hzn @ Hnn_inv @ g[nz:]
    return S, rhs


# ----------------------------------------------------------------------------------------------------------------
# closed-form reduced system over the full-grid layout (supported dofs eliminated as identity rows)
# ----------------------------------------------------------------------------------------------------------------


def assemble_S(pb: Problem, st: State, cf: Coeffs | None = None) -> sp.csr_matrix:
    """Bordered CSR S ((n+1) x (n+1)): [K(rho'), 0; 0, 0] + sum_i d_i g_i g_i^T with g_i = [K_i u; -1], supported
    rows/cols replaced by identity. Index n is alpha."""
    cf = coeffs(pb, st) if cf is None else cf
    n, m = pb.n, pb.m
    W = element_w(pb, st.u)
    K1 = fem.assemble_unconstrained(pb.grid, cf.rho1, pb.Ke)
    K1 = fem.apply_supports(K1, pb.fixed)
    K1 = sp.block_diag([K1, sp.csr_matrix((1, 1))]).tocsr()          # border row/column of the alpha unknown
    # rank-1 terms, element by element: local vector [w_e ; -1] on dofs [dofs_e ; n]
    idx = np.concatenate([pb.dofs, np.full((m, 1), n)], axis=1)            # (m, 25)
    vec = np.concatenate([W, -np.ones((m, 1))], axis=1)                    # (m, 25)
    vals = cf.d[:, None, None] * vec[:, :, None] * vec[:, None, :]
    rows = np.repeat(idx, 25, axis=1).ravel()
    cols = np.tile(idx, (1, 25)).ravel()
    R = sp.coo_matrix((vals.ravel(), (rows, cols)), shape=(n + 1, n + 1)).tocsr()
    return (K1 + R).tocsr()


def apply_S_elementwise(pb: Problem, st: State, cf: Coeffs, x: np.ndarray) -> np.ndarray:
    """Matrix-free S x (x of length n+1) from its closed form, element by element."""
    n = pb.n
    xu = masked(pb, x[:n])
    W = element_w(pb, st.u)
    xe = xu[pb.dofs]
    t = cf.d * (np.einsum("ej,ej->e", W, xe) - x[n])
    ye = cf.rho1[:, None] * (xe @ pb.Ke) + t[:, None] * W
    y = np.bincount(pb.dofs.ravel(), weights=ye.ravel(), minlength=n)
    y = np.where(pb.fixed, x[:n], y)
    return np.concatenate([y, [-t.sum()]])


def rhs_closed(pb: Problem, st: State, cf: Coeffs | None = None) -> np.ndarray:
    """rhs = [f - K(rho' - eps) u ; -V + sum(rho' - eps)] (length n+1, zero on supported dofs)."""
    cf = coeffs(pb, st) if cf is None else cf
    um = masked(pb, st.u)
    ru = pb.f - fem.apply_K_elementwise(pb.grid, cf.rho1 - cf.eps, pb.Ke, um)
    ru = np.where(pb.fixed, 0.0, ru)
    return np.concatenate([ru, [-pb.V + (cf.rho1 - cf.eps).sum()]])


def delta_nu(pb: Problem, st: State, cf: Coeffs, dz: np.ndarray):
    """eq. (deltanu): dnu_i = -B_i^{-1} (grad_nu_i L + rho''_i (w_i . du_i - dalpha) [1; -1])."""
    n = pb.n
    W = element_w(pb, st.u)
    du = masked(pb, dz[:n])
    proj = np.einsum("ej,ej->e", W, du[pb.dofs]) - dz[n]
    rl = cf.gl + cf.rho2 * proj
    ru = cf.gu - cf.rho2 * proj
    a11, a22, a12 = cf.rho2 + cf.mul2, cf.rho2 + cf.muu2, -cf.rho2
    det = a11 * a22 - a12 * a12
    dl = -(a22 * rl - a12 * ru) / det
    dup = -(-a12 * rl + a11 * ru) / det
    return dl, dup


def res_pbm(pb: Problem, st: State, cf: Coeffs | None = None) -> float:
    """eq. (resIP): ||res_1||/||f|| + |res_2|/V + ||res_3||/(||rho_lo|| + ||rho_up||)."""
    cf = coeffs(pb, st) if cf is None else cf
    gu_vec, ga, gl, _ = gradient(pb, st, cf)
    m = pb.m
    denom = math.sqrt(m) * (abs(pb.rho_lo) + abs(pb.rho_up))
    return float(np.linalg.norm(gu_vec) / np.linalg.norm(pb.f) + abs(ga) / pb.V + np.linalg.norm(gl) / denom)


# ----------------------------------------------------------------------------------------------------------------
# duality gap (eq. gap) and dual objective
# ----------------------------------------------------------------------------------------------------------------


def duality_gap(pb: Problem, st: State) -> float:
    um = masked(pb, st.u)
    c = compliances(pb, um)
    a = st.alpha - c
    return float(-0.5 * pb.f @ um + st.alpha * pb.V - np.sum(np.minimum(pb.rho_lo * a, pb.rho_up * a)))


def dual_objective(pb: Problem, st: State) -> float:
    um = masked(pb, st.u)
    return float(st.alpha * pb.V - pb.f @ um - pb.rho_lo * st.nu_lo.sum() + pb.rho_up * st.nu_up.sum())


# ----------------------------------------------------------------------------------------------------------------
# Newton (Algorithm 2) and PBM (Algorithm 1)
# ----------------------------------------------------------------------------------------------------------------


@dataclass
class NewtonInfo:
    iters: int = 0
    minres_iters: int = 0
    res: float = float("nan")
    kappas: list = field(default_factory=list)
    resolves: int = 0          # re-solves with a tightened eps_MR after a non-descent direction
    stalled: bool = False      # no descent direction even at eps_mr_min: the loop ended at the current iterate
    slopes: list = field(default_factory=list)


def solve_reduced(pb: Problem, st: State, cf: Coeffs, rhs: np.ndarray, eps_mr: float | None, levels: int,
                  theta: float = 1.2, sweeps: int = 2):
    """Solve S dz = rhs: direct (eps_mr None) or MG-preconditioned MINRES to ||r|| <= eps_mr ||rhs||."""
    S = assemble_S(pb, st, cf)
    if eps_mr is None:
        return solvers.direct_solve(S, rhs), 0
    hier = solvers.Hierarchy(pb.grid, S, levels, has_alpha=True, theta=theta, sweeps=sweeps)
    res = solvers.minres(lambda v: S @ v, rhs, hier.vcycle, rtol=eps_mr, maxit=10000)
    return res.x, res.iters


def newton(pb: Problem, st: State, eps_nwt: float, eps_mr: float | None = None, levels: int = 2,
           max_iter: int = 100, c1: float = 1e-4, max_halvings: int = 30, adapt_eps_mr: bool = False,
           info: NewtonInfo | None = None, eps_mr_min: float = 1e-9):
    """Algorithm 2: Newton with Armijo backtracking on the augmented Lagrangian until res_PBM < eps_nwt.
    Returns (state, info, eps_mr). A direction that is not one of descent is solved again with eps_MR / 10 (down to
    eps_mr_min); at the floor the loop stops at the current iterate (info.stalled)."""
    info = NewtonInfo() if info is None else info
    st = st.copy()
    res_prev = None
    for _ in range(max_iter):
        cf = coeffs(pb, st)
        res = res_pbm(pb, st, cf)
        info.res = res
        if res < eps_nwt:
            break
        if adapt_eps_mr and eps_mr is not None and res_prev is not None and res > 0.9 * res_prev:
            eps_mr = max(0.1 * eps_mr, eps_mr_min)
        res_prev = res
        rhs = rhs_closed(pb, st, cf)
        gu_vec, ga, gl, gu = gradient(pb, st, cf)
        while True:
            dz, its = solve_reduced(pb, st, cf, rhs, eps_mr, levels)
            info.minres_iters += its
            dl, dup = delta_nu(pb, st, cf, dz)
            slope = gu_vec @ masked(pb, dz[:pb.n]) + ga * dz[pb.n] + gl @ dl + gu @ dup
            if slope < 0.0 or eps_mr is None or eps_mr <= eps_mr_min:
                break
            eps_mr = max(0.1 * eps_mr, eps_mr_min)
            info.resolves += 1
        info.slopes.append(float(slope))
        if not slope < 0.0:
            info.stalled = True
            break
        L0 = lagrangian(pb, st)
        kappa = 1.0
        for _h in range(max_halvings + 1):
            trial = st.copy()
            trial.u = masked(pb, st.u + kappa * dz[:pb.n])
            trial.alpha = st.alpha + kappa * dz[pb.n]
            trial.nu_lo = st.nu_lo + kappa * dl
            trial.nu_up = st.nu_up + kappa * dup
            if lagrangian(pb, trial) <= L0 + c1 * kappa * slope:
                break
            kappa *= 0.5
        else:
            raise RuntimeError("line search failed")
        st = trial
        info.kappas.append(kappa)
        info.iters += 1
    else:
        info.res = res_pbm(pb, st)
    return st, info, eps_mr


def multiplier_update(pb: Problem, st: State, beta: float) -> State:
    """Multiplier update of Algorithm 1 with the safeguard beta*x <= x+ <= x/beta."""
    st = st.copy()
    s = constraint_arg(pb, st)
    rho_new = st.rho * dphi(s)
    mul_new = st.mu_lo * dphi(-st.nu_lo / st.q_lo)
    muu_new = st.mu_up * dphi(-st.nu_up / st.q_up)
    st.rho = np.clip(rho_new, beta * st.rho, st.rho / beta)
    st.mu_lo = np.clip(mul_new, beta * st.mu_lo, st.mu_lo / beta)
    st.mu_up = np.clip(muu_new, beta * st.mu_up, st.mu_up / beta)
    return st


@dataclass
class PbmResult:
    state: State
    outer: int
    newton: int
    minres: int
    gap_ratio: float
    history: list


def pbm(pb: Problem, eps_pbm: float = 1e-5, beta: float = 0.3, gamma: float = 0.3, p_min: float = 1e-8,
        eps_nwt: float = 1.0, eps_nwt_min: float = 1e-3, eps_mr: float | None = None, levels: int = 2,
        max_outer: int = 100, state: State | None = None) -> PbmResult:
    """Algorithm 1 with the paper's parameters and initial point (u = 0, alpha = 1, nu = e, rho = V/m, mu = e)."""
    m = pb.m
    st = state.copy() if state is not None else State(np.zeros(pb.n), 1.0, np.ones(m), np.ones(m),
                                                      np.full(m, pb.V / m), np.ones(m), np.ones(m))
    total_newton = total_mr = 0
    hist = []
    ratio = float("nan")
    outer = 0
    for outer in range(1, max_outer + 1):
        st, ninfo, eps_mr = newton(pb, st, eps_nwt, eps_mr, levels, adapt_eps_mr=True)
        total_newton += ninfo.iters
        total_mr += ninfo.minres_iters
        gap = duality_gap(pb, st)
        dual = dual_objective(pb, st)
        ratio = abs(gap / dual)
        hist.append(dict(outer=outer, gap=gap, dual=dual, ratio=ratio, newton=ninfo.iters, res=ninfo.res,
                         p=st.p))
        if ratio < eps_pbm:
            break
        st = multiplier_update(pb, st, beta)
        st.p, st.q_lo, st.q_up = max(gamma * st.p, p_min), max(gamma * st.q_lo, p_min), max(gamma * st.q_up, p_min)
        eps_nwt = max(min(100.0 * ratio, eps_nwt), eps_nwt_min)
    st, ninfo, eps_mr = newton(pb, st, 10.0 * eps_pbm, eps_mr, levels, adapt_eps_mr=True)
    total_newton += ninfo.iters
    total_mr += ninfo.minres_iters
    s = constraint_arg(pb, st)
    rho_new = st.rho * dphi(s)
    st.rho = np.clip(rho_new, beta * st.rho, st.rho / beta)
    return PbmResult(st, outer, total_newton, total_mr, ratio, hist)
