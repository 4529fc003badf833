"""The damped optimality-criteria (DOC) method for the VTS problem (oracle; test infrastructure only: only tests/,
__graft_entry__.smoke() and bench.py's CPU legs import this package).

Written from Section 4.2 of the paper (Algorithm DOC). One iteration: the equilibrium displacement u of K(rho) u = f,
then the volume multiplier alpha by bisection on [0, 10^4], each trial density being
    rho_i^+ = min(max(rho_i (u^T K_i u)^q / alpha, rho_lo), rho_up),
raising the lower end while sum(rho^+) exceeds V and lowering the upper end otherwise, until
(alpha_hi - alpha_lo) / (alpha_hi + alpha_lo) <= tau_alpha; rho^+ is the density of the last trial. The run stops
when ||rho^+ - rho||_inf <= eps_DOC. Defaults: q = 1/2, tau_alpha = eps_DOC / 10.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse.linalg as sla

from . import fem
from .pbm import Problem, masked


def energies(pb: Problem, u: np.ndarray) -> np.ndarray:
    """u^T K_i u per element (supported dofs masked)."""
    return fem.element_energies(pb.grid, pb.Ke, masked(pb, u))


def density_update(rho: np.ndarray, e: np.ndarray, V: float, rho_lo: float, rho_up: float, q: float,
                   tau_alpha: float, alpha_hi: float = 1e4):
    """The bisection of Algorithm DOC: (rho^+, alpha of the last trial, number of trials)."""
    w = rho * np.power(e, q)
    lo, hi = 0.0, alpha_hi
    rho_new, alpha, trials = rho.copy(), 0.0, 0
    while (hi - lo) / (hi + lo) > tau_alpha:
        alpha = 0.5 * (hi + lo)
        rho_new = np.minimum(np.maximum(w / alpha, rho_lo), rho_up)
        trials += 1
        if rho_new.sum() > V:
            lo = alpha
        else:
            hi = alpha
    return rho_new, alpha, trials


@dataclass
class DocResult:
    rho: np.ndarray
    u: np.ndarray
    iterations: int
    change: float
    converged: bool


def doc(pb: Problem, rho0: np.ndarray, q: float = 0.5, eps_doc: float = 1e-3, tau_alpha: float | None = None,
        max_iter: int = 1000) -> DocResult:
    """Algorithm DOC with exact (direct) equilibrium solves."""
    tau = 0.1 * eps_doc if tau_alpha is None else tau_alpha
    rho = rho0.copy()
    u = np.zeros(pb.n)
    change = np.inf
    for it in range(1, max_iter + 1):
        K = fem.assemble_K(pb.grid, rho, pb.Ke)
        u = sla.spsolve(K.tocsc(), pb.f)
        rho_new, _, _ = density_update(rho, energies(pb, u), pb.V, pb.rho_lo, pb.rho_up, q, tau)
        change = float(np.abs(rho_new - rho).max())
        if change <= eps_doc:
            return DocResult(rho, u, it, change, True)
        rho = rho_new
    return DocResult(rho, u, max_iter, change, False)
