"""Reduced Newton system of the primal-dual interior-point (IP) method for the VTS problem (oracle; test
infrastructure only: only tests/, __graft_entry__.smoke() and bench.py's CPU legs import this package).

Written from Section 4.1 of the paper. The unknowns are z = (u, alpha, rho, nu_lo, nu_up); the barrier parameters
r, s > 0 perturb the two complementarity conditions of the KKT system of eq. (1):
    res_1 = K(rho) u - f                                  (n)
    res_2 = sum(rho) - V                                  (1)
    res_3 = 1/2 u^T K_i u + alpha + nu_lo_i - nu_up_i     (m)
    res_4 = nu_lo_i (rho_i - rho_lo) - r                  (m)
    res_5 = nu_up_i (rho_up - rho_i) - s                  (m)
One Newton step solves J dz = -res with J the Jacobian of eq. (gradres). Eliminating (dnu_lo, dnu_up) and then
drho (two Schur complements) leaves the bordered system of eq. (S_IP),
    S = [K(rho), 0; 0, 0] + sum_i d_i g_i g_i^T,  g_i = [K_i u; 1],  d_i = 1 / (nu_lo_i / (rho_i - rho_lo)
                                                                          + nu_up_i / (rho_up - rho_i)),
with right-hand side  -[res_1; res_2] - sum_i d_i c_i g_i,  c_i = res_3 - res_4 / (rho_i - rho_lo)
+ res_5 / (rho_up - rho_i), and the increments follow back:
    drho_i   = d_i (w_i . du + dalpha + c_i),                     w_i = K_i u,
    dnu_up_i = ((rho_i - rho_lo)(w_i . du + dalpha + res_3) - (nu_lo_i - nu_up_i) drho_i - res_4 - res_5)
               / (rho_up - rho_lo)       (the form of eq. (Delta_onu)),
    dnu_lo_i = dnu_up_i - w_i . du - dalpha - res_3                (eq. (Delta_unu)).
Readings where the printed formulas disagree with one another (the CUDA path takes the same ones):
  * the nu_up column of the printed residual carries +e_i in res_3 and (rho_up - rho_i) e_i in res_4; the KKT
    conditions and the Jacobian eq. (gradres) put -e_i in res_3 and (rho_up - rho_i) e_i in res_5, as above;
  * the right-hand side and drho are derived from J dz = -res: the printed eq. (IP_system) and eq. (Delta_rho)
    differ from that derivation (and from each other) in the signs of the res_3 .. res_5 terms;
  * eq. (Delta_onu) prints (U_nu - O_nu) rho where the elimination gives (U_nu - O_nu) drho.
Supported dofs are eliminated (identity rows, zero increments), as in the PBM part.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem
from .pbm import Problem, element_w, masked


@dataclass
class IPState:
    u: np.ndarray
    alpha: float
    rho: np.ndarray
    nu_lo: np.ndarray
    nu_up: np.ndarray


def residual(pb: Problem, st: IPState, r: float, s: float):
    """(res_1 (n, zero on supported dofs), res_2, res_3, res_4, res_5) of the perturbed KKT system."""
    um = masked(pb, st.u)
    r1 = fem.apply_K_elementwise(pb.grid, st.rho, pb.Ke, um) - pb.f
    r1 = np.where(pb.fixed, 0.0, r1)
    r2 = float(st.rho.sum() - pb.V)
    c = 0.5 * fem.element_energies(pb.grid, pb.Ke, um)
    r3 = c + st.alpha + st.nu_lo - st.nu_up
    r4 = st.nu_lo * (st.rho - pb.rho_lo) - r
    r5 = st.nu_up * (pb.rho_up - st.rho) - s
    return r1, r2, r3, r4, r5


def pack(pb: Problem, st: IPState) -> np.ndarray:
    """z = [u (free dofs) ; alpha ; rho ; nu_lo ; nu_up]."""
    free = ~pb.fixed
    return np.concatenate([st.u[free], [st.alpha], st.rho, st.nu_lo, st.nu_up])


def unpack(pb: Problem, z: np.ndarray) -> IPState:
    free = ~pb.fixed
    nf, m = int(free.sum()), pb.m
    u = np.zeros(pb.n)
    u[free] = z[:nf]
    a = float(z[nf])
    return IPState(u, a, z[nf + 1:nf + 1 + m].copy(), z[nf + 1 + m:nf + 1 + 2 * m].copy(),
                   z[nf + 1 + 2 * m:nf + 1 + 3 * m].copy())


def residual_vector(pb: Problem, st: IPState, r: float, s: float) -> np.ndarray:
    r1, r2, r3, r4, r5 = residual(pb, st, r, s)
    return np.concatenate([r1[~pb.fixed], [r2], r3, r4, r5])


def jacobian_dense(pb: Problem, st: IPState) -> np.ndarray:
    """The Jacobian of eq. (gradres) over the free unknowns, assembled block by block (tiny grids)."""
    free = ~pb.fixed
    nf, m = int(free.sum()), pb.m
    K = fem.assemble_unconstrained(pb.grid, st.rho, pb.Ke).toarray()[np.ix_(free, free)]
    W = element_w(pb, st.u)                                  # (m, 24), supported dofs zeroed
    B = np.zeros((pb.n, m))
    for e in range(m):
        np.add.at(B[:, e], pb.dofs[e], W[e])
    B = B[free]
    N = nf + 1 + 3 * m
    J = np.zeros((N, N))
    iu, ia, ir, il, iv = 0, nf, nf + 1, nf + 1 + m, nf + 1 + 2 * m
    J[iu:ia, iu:ia] = K
    J[iu:ia, ir:il] = B
    J[ia, ir:il] = 1.0
    J[ir:il, iu:ia] = B.T
    J[ir:il, ia] = 1.0
    J[ir:il, il:iv] = np.eye(m)
    J[ir:il, iv:] = -np.eye(m)
    J[il:iv, ir:il] = np.diag(st.nu_lo)
    J[il:iv, il:iv] = np.diag(st.rho - pb.rho_lo)
    J[iv:, ir:il] = -np.diag(st.nu_up)
    J[iv:, iv:] = np.diag(pb.rho_up - st.rho)
    return J


@dataclass
class IPCoeffs:
    d: np.ndarray       # Schur weights of eq. (S_IP)
    c: np.ndarray       # res_3 - res_4 / (rho - rho_lo) + res_5 / (rho_up - rho)
    r3: np.ndarray
    r4: np.ndarray
    r5: np.ndarray


def coeffs(pb: Problem, st: IPState, r: float, s: float) -> IPCoeffs:
    _, _, r3, r4, r5 = residual(pb, st, r, s)
    gl, gu = st.rho - pb.rho_lo, pb.rho_up - st.rho
    d = 1.0 / (st.nu_lo / gl + st.nu_up / gu)
    return IPCoeffs(d, r3 - r4 / gl + r5 / gu, r3, r4, r5)


def assemble_S(pb: Problem, st: IPState, cf: IPCoeffs) -> sp.csr_matrix:
    """Bordered CSR S of eq. (S_IP): [K(rho), 0; 0, 0] + sum_i d_i g_i g_i^T, g_i = [K_i u; 1]; supported rows and
    columns the identity; index n is alpha."""
    n, m = pb.n, pb.m
    W = element_w(pb, st.u)
    K = fem.apply_supports(fem.assemble_unconstrained(pb.grid, st.rho, pb.Ke), pb.fixed)
    K = sp.block_diag([K, sp.csr_matrix((1, 1))]).tocsr()
    idx = np.concatenate([pb.dofs, np.full((m, 1), n)], axis=1)
    vec = np.concatenate([W, np.ones((m, 1))], axis=1)
    vals = cf.d[:, None, None] * vec[:, :, None] * vec[:, None, :]
    R = sp.coo_matrix((vals.ravel(), (np.repeat(idx, 25, axis=1).ravel(), np.tile(idx, (1, 25)).ravel())),
                      shape=(n + 1, n + 1)).tocsr()
    return (K + R).tocsr()


def apply_S(pb: Problem, st: IPState, cf: IPCoeffs, x: np.ndarray) -> np.ndarray:
    """Matrix-free S x of eq. (S_IP), element by element."""
    n = pb.n
    xu = masked(pb, x[:n])
    W = element_w(pb, st.u)
    xe = xu[pb.dofs]
    t = cf.d * (np.einsum("ej,ej->e", W, xe) + x[n])
    ye = st.rho[:, None] * (xe @ pb.Ke) + t[:, None] * W
    y = np.bincount(pb.dofs.ravel(), weights=ye.ravel(), minlength=n)
    y = np.where(pb.fixed, x[:n], y)
    return np.concatenate([y, [t.sum()]])


def rhs(pb: Problem, st: IPState, r: float, s: float, cf: IPCoeffs | None = None) -> np.ndarray:
    """Right-hand side of the reduced system: -[res_1; res_2] - sum_i d_i c_i [K_i u; 1] (zero on supported dofs)."""
    cf = coeffs(pb, st, r, s) if cf is None else cf
    r1, r2, _, _, _ = residual(pb, st, r, s)
    um = masked(pb, st.u)
    ru = -r1 - fem.apply_K_elementwise(pb.grid, cf.d * cf.c, pb.Ke, um)
    ru = np.where(pb.fixed, 0.0, ru)
    return np.concatenate([ru, [-r2 - float((cf.d * cf.c).sum())]])


def recover(pb: Problem, st: IPState, cf: IPCoeffs, dz: np.ndarray):
    """(drho, dnu_lo, dnu_up) from the reduced solution dz = [du; dalpha]."""
    n = pb.n
    du = masked(pb, dz[:n])
    da = float(dz[n])
    wdu = np.einsum("ej,ej->e", element_w(pb, st.u), du[pb.dofs])
    drho = cf.d * (wdu + da + cf.c)
    gl = st.rho - pb.rho_lo
    dnu_up = (gl * (wdu + da + cf.r3) - (st.nu_lo - st.nu_up) * drho - cf.r4 - cf.r5) / (pb.rho_up - pb.rho_lo)
    dnu_lo = dnu_up - wdu - da - cf.r3
    return drho, dnu_lo, dnu_up


def newton_full(pb: Problem, st: IPState, r: float, s: float):
    """The full Newton step J dz = -res by a dense solve (tiny grids): (du (n), dalpha, drho, dnu_lo, dnu_up)."""
    J = jacobian_dense(pb, st)
    dz = np.linalg.solve(J, -residual_vector(pb, st, r, s))
    d = unpack(pb, dz)
    return d.u, d.alpha, d.rho, d.nu_lo, d.nu_up


def state_from_dict(d: dict) -> IPState:
    return IPState(np.array(d["u"], dtype=float), float(d["alpha"]), np.array(d["rho"], dtype=float),
                   np.array(d["nu_lo"], dtype=float), np.array(d["nu_up"], dtype=float))
