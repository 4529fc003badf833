"""Pins of the interior-point oracle (oracle/ip.py, Section 4.1) against things other than itself: finite
differences of the residual, the dense Newton step of the full system, the dense Schur complements, and positive
definiteness."""
import numpy as np
import pytest

import synthetic
from oracle import fem, ip, pbm

CASES = [((3, 2, 2), "cantilever", 0), ((2, 2, 2), "bridge_corners", 1), ((4, 2, 1), "bridge_edges", 2)]


def make(dims, bc, seed):
    g = fem.Grid(*dims, bc)
    f = synthetic.load_vector(*dims, "end_edge")
    d = synthetic.ip_random_state(*dims, seed, fixed_dofs=g.fixed_dofs())
    pb = pbm.Problem(g, f, d["V"], d["rho_lo"], d["rho_up"])
    return pb, ip.state_from_dict(d), d["r"], d["s"]


@pytest.mark.parametrize("dims,bc,seed", CASES)
def test_jacobian_equals_finite_differences_of_the_residual(dims, bc, seed):
    pb, st, r, s = make(dims, bc, seed)
    J = ip.jacobian_dense(pb, st)
    z0 = ip.pack(pb, st)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for k in range(z0.size):
        zp, zm = z0.copy(), z0.copy()
        zp[k] += h
        zm[k] -= h
        Jfd[:, k] = (ip.residual_vector(pb, ip.unpack(pb, zp), r, s) -
                     ip.residual_vector(pb, ip.unpack(pb, zm), r, s)) / (2 * h)
    assert np.abs(J - Jfd).max() <= 1e-6 * max(1.0, np.abs(J).max())


@pytest.mark.parametrize("dims,bc,seed", CASES)
def test_reduced_solve_and_recovery_equal_the_full_newton_step(dims, bc, seed):
    pb, st, r, s = make(dims, bc, seed)
    cf = ip.coeffs(pb, st, r, s)
    S = ip.assemble_S(pb, st, cf).toarray()
    dz = np.linalg.solve(S, ip.rhs(pb, st, r, s, cf))
    drho, dnl, dnu = ip.recover(pb, st, cf, dz)
    fu, fa, frho, fnl, fnu = ip.newton_full(pb, st, r, s)
    scale = lambda v: max(1.0, np.abs(v).max())
    assert np.abs(dz[:pb.n] - fu).max() <= 1e-10 * scale(fu)
    assert abs(dz[pb.n] - fa) <= 1e-10 * max(1.0, abs(fa))
    assert np.abs(drho - frho).max() <= 1e-10 * scale(frho)
    assert np.abs(dnl - fnl).max() <= 1e-10 * scale(fnl)
    assert np.abs(dnu - fnu).max() <= 1e-10 * scale(fnu)


@pytest.mark.parametrize("dims,bc,seed", CASES)
def test_closed_form_S_equals_the_double_schur_complement(dims, bc, seed):
    pb, st, r, s = make(dims, bc, seed)
    J = ip.jacobian_dense(pb, st)
    free = ~pb.fixed
    nf, m = int(free.sum()), pb.m
    a = nf + 1                                   # (u, alpha) block, then rho, then (nu_lo, nu_up)
    A, B, C = J[:a + m, :a + m], J[:a + m, a + m:], J[a + m:, a + m:]
    D = J[a + m:, :a + m]
    S1 = A - B @ np.linalg.solve(C, D)          # eliminate the multipliers
    S2 = S1[:a, :a] - S1[:a, a:] @ np.linalg.solve(S1[a:, a:], S1[a:, :a])   # then rho
    # the rho block of S1 is -(U_rho^-1 U_nu + O_rho^-1 O_nu), so S2 = [K, 0; 0, 0] + [B; e^T] D [B^T, e]: compare
    # with the closed form on the free dofs and alpha
    assert np.all(np.linalg.eigvalsh(S1[a:, a:]) < 0)
    Sfull = ip.assemble_S(pb, st, ip.coeffs(pb, st, r, s)).toarray()
    keep = np.concatenate([np.flatnonzero(free), [pb.n]])
    assert np.abs(Sfull[np.ix_(keep, keep)] - S2).max() <= 1e-10 * np.abs(S2).max()


@pytest.mark.parametrize("dims,bc,seed", CASES)
def test_S_is_spd_and_the_matrix_free_apply_matches(dims, bc, seed):
    pb, st, r, s = make(dims, bc, seed)
    cf = ip.coeffs(pb, st, r, s)
    assert (cf.d > 0).all()
    S = ip.assemble_S(pb, st, cf)
    Sd = S.toarray()
    assert np.allclose(Sd, Sd.T, atol=1e-13 * np.abs(Sd).max())
    np.linalg.cholesky(Sd)
    x = np.random.default_rng(seed).standard_normal(pb.n + 1)
    assert np.abs(ip.apply_S(pb, st, cf, x) - S @ x).max() <= 1e-12 * np.abs(S @ x).max()
