"""Pins of the DOC oracle (oracle/doc.py, Algorithm DOC): the bisection against an independent root finder, and
the DOC fixed point against the optimality conditions of the VTS problem and the PBM oracle's optimum."""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse.linalg as sla

import synthetic
from oracle import doc, fem, pbm


def test_bisection_brackets_the_root_of_the_volume_equation():
    rng = np.random.default_rng(0)
    m = 500
    rho = rng.uniform(0.05, 0.9, m)
    e = rng.uniform(1e-3, 2.0, m)
    V, lo, hi, q, tau = 0.3 * m, 1e-3, 1.0, 0.5, 1e-6
    rho_new, alpha, trials = doc.density_update(rho, e, V, lo, hi, q, tau)
    g = lambda a: np.clip(rho * e ** q / a, lo, hi).sum() - V
    root = so.brentq(g, 1e-8, 1e4, xtol=1e-15, rtol=1e-15)
    assert abs(alpha - root) <= 4 * tau * root
    assert np.all(rho_new >= lo) and np.all(rho_new <= hi)
    assert abs(rho_new.sum() - V) <= 1e-4 * V
    # each trial halves [lo, hi] from [0, 1e4]; it stops once the width is below 2 tau alpha
    assert abs(trials - np.log2(1e4 / (2 * tau * root))) <= 2


def test_bisection_stops_when_the_relative_interval_is_small():
    rho = np.full(10, 0.5)
    e = np.full(10, 1.0)
    _, alpha, trials = doc.density_update(rho, e, 5.0, 1e-3, 1.0, 0.5, 0.5)
    # [0, 1e4] -> first trial at 5e3, ...: stops once (hi - lo)/(hi + lo) <= 1/2, i.e. after hi = 3 lo
    assert trials >= 1 and alpha > 0


def test_doc_fixed_point_satisfies_the_optimality_conditions_and_matches_pbm():
    nx, ny, nz = 4, 2, 2
    g = fem.Grid(nx, ny, nz, "cantilever")
    f = synthetic.load_vector(nx, ny, nz, "end_edge")
    V = 0.4 * g.m
    pb = pbm.Problem(g, f, V, 1e-3, 1.0)
    res = doc.doc(pb, np.full(g.m, V / g.m), q=0.5, eps_doc=1e-7, max_iter=3000)
    assert res.converged
    rho = res.rho
    assert abs(rho.sum() - V) <= 1e-5 * V
    # KKT of the VTS problem: u^T K_i u is the same for every element strictly between the bounds
    e = doc.energies(pb, res.u)
    mid = (rho > 1e-3 + 1e-4) & (rho < 1.0 - 1e-4)
    assert mid.sum() >= 2
    assert np.ptp(e[mid]) <= 1e-3 * e[mid].mean()
    # and the compliance equals the one at the PBM oracle's optimum
    out = pbm.pbm(pb, eps_pbm=1e-8)
    K = fem.assemble_K(g, out.state.rho, pb.Ke)
    c_pbm = pb.f @ sla.spsolve(K.tocsc(), pb.f)
    c_doc = pb.f @ res.u
    assert abs(c_doc - c_pbm) <= 1e-4 * c_pbm
