"""Pins for the oracle's finite-element layer (Section 5.2, Section 6, eq. (1)).

Every check compares the oracle with something other than itself: the paper's printed problem dimensions
(Tables 2-5), an independent derivation of the element matrix from the weak form with 1D closed-form integrals,
the exact strain energy of constant-strain fields, rigid-body null spaces, and the nested-space identity between
Galerkin and rediscretised coarse operators.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_grid_dims.txt")
LAM = lambda E, nu: E * nu / ((1 + nu) * (1 - 2 * nu))
MU = lambda E, nu: E / (2 * (1 + nu))


def _paper_rows():
    rows = []
    with open(GOLD) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            kind, mx, my, mz, lv, m, n, src = line.split()
            rows.append((kind, int(mx), int(my), int(mz), int(lv), int(m), int(n), src))
    return rows


@pytest.mark.parametrize("row", _paper_rows(), ids=lambda r: f"{r[0]}-{r[1]}-{r[2]}-{r[3]}-{r[4]}")
def test_grid_dimensions_match_paper_tables(row):
    kind, mx, my, mz, lv, m, n, _ = row
    s = 2 ** (lv - 1)
    nx, ny, nz = mx * s, my * s, mz * s
    if nx * ny * nz > 2_200_000:
        # closed-form count for the largest rows (the node arrays would take too long on CPU): same support rule
        nnode = (nx + 1) * (ny + 1) * (nz + 1)
        fixed = (ny + 1) * (nz + 1) if kind == "CANT" else 4
        assert nx * ny * nz == m and 3 * (nnode - fixed) == n
        return
    g = fem.Grid(nx, ny, nz, "cantilever" if kind == "CANT" else "bridge_corners")
    assert g.m == m
    assert g.n_free() == n


def _Ke_weak_form(E, nu):
    """K^{cd}_{ab} = lam int d_c N_a d_d N_b + mu int d_d N_a d_c N_b + mu delta_cd int grad N_a . grad N_b,
    each integral a product of 1D closed forms on [0, 1]: int N'N' = S1, int N N = M1, int N_a' N_b = C1."""
    S1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    C1 = np.array([[-0.5, -0.5], [0.5, 0.5]])          # C1[a, b] = int N_a' N_b
    lam, mu = LAM(E, nu), MU(E, nu)
    off = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]

    def M(c, d, a, b):  # int d_c N_a d_d N_b over the unit cube
        val = 1.0
        for k in range(3):
            ia, ib = off[a][k], off[b][k]
            if k == c and k == d:
                val *= S1[ia, ib]
            elif k == c:
                val *= C1[ia, ib]
            elif k == d:
                val *= C1[ib, ia]
            else:
                val *= M1[ia, ib]
        return val

    K = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            for c in range(3):
                for d in range(3):
                    v = lam * M(c, d, a, b) + mu * M(d, c, a, b)
                    if c == d:
                        v += mu * sum(M(k, k, a, b) for k in range(3))
                    K[3 * a + c, 3 * b + d] = v
    return K


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (2.5, 0.1), (1.0, 0.45)])
def test_Ke_equals_weak_form_closed_form(E, nu):
    assert np.allclose(fem.element_stiffness(E, nu), _Ke_weak_form(E, nu), rtol=0, atol=1e-14 * E / (1 - 2 * nu))


def test_Ke_symmetric_psd_six_rigid_modes():
    K = fem.element_stiffness(1.0, 0.3)
    assert np.array_equal(K, K.T) or np.max(np.abs(K - K.T)) < 1e-15
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-12) == 6
    assert ev.min() > -1e-13
    R = fem.rigid_body_modes()
    assert np.max(np.abs(K @ R)) < 1e-13
    # the 6 modes span the null space exactly
    assert np.linalg.matrix_rank(R) == 6


def test_Ke_gauss_orders_agree_and_linear_in_E():
    K2 = fem.element_stiffness(1.0, 0.3, order=2)
    K3 = fem.element_stiffness(1.0, 0.3, order=3)
    assert np.max(np.abs(K2 - K3)) < 1e-14
    assert np.allclose(fem.element_stiffness(3.0, 0.3), 3.0 * K2, rtol=1e-14, atol=1e-15)


def test_Ke_scales_with_edge_length():
    # int B^T D B dx with B ~ 1/h and volume h^3: K_e(h) = h K_e(1)
    assert np.allclose(fem.element_stiffness(1.0, 0.3, h=2.0), 2.0 * fem.element_stiffness(1.0, 0.3), rtol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_Ke_constant_strain_energy(seed):
    """u(x) = G x (G any 3x3) has constant strain eps = sym(G); exact energy u^T K u = vol * eps : C : eps
    = lam tr(eps)^2 + 2 mu eps:eps on the unit cube."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((3, 3))
    X = fem.local_offsets().astype(float)
    u = (X @ G.T).ravel()
    eps = 0.5 * (G + G.T)
    E, nu = 1.0, 0.3
    exact = LAM(E, nu) * np.trace(eps) ** 2 + 2 * MU(E, nu) * np.sum(eps * eps)
    assert abs(u @ fem.element_stiffness(E, nu) @ u - exact) < 1e-13 * max(1.0, exact)


def test_node_element_dof_numbering():
    g = fem.Grid(3, 2, 2)
    en = g.elem_nodes()
    # element (1, 1, 1) = 1 + 3 (1 + 2 * 1) = 10; its local node a = ix + 2 iy + 4 iz sits at (1+ix, 1+iy, 1+iz)
    assert en[10].tolist() == [g.node_id(1 + (a & 1), 1 + ((a >> 1) & 1), 1 + ((a >> 2) & 1)) for a in range(8)]
    assert g.node_id(3, 2, 2) == g.nnode - 1
    assert g.elem_dofs()[10, 3 * 5 + 2] == 3 * en[10, 5] + 2


def test_supports():
    g = fem.Grid(4, 2, 2, "bridge_corners")
    assert g.fixed_nodes().sum() == 4
    g = fem.Grid(4, 2, 2, "cantilever")
    assert g.fixed_nodes().sum() == 9
    g = fem.Grid(4, 2, 2, "bridge_edges")
    assert g.fixed_nodes().sum() == 6


def test_single_element_assembly_is_Ke():
    g = fem.Grid(2, 2, 2, "free")
    Ke = fem.element_stiffness()
    w = np.zeros(g.m)
    w[5] = 1.0
    K = fem.assemble_K(g, w, Ke).toarray()
    d = g.elem_dofs()[5]
    assert np.allclose(K[np.ix_(d, d)], Ke, atol=1e-15)
    mask = np.ones(g.n, bool)
    mask[d] = False
    assert np.all(K[np.ix_(mask, mask)] == 0.0)


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners"])
def test_K_symmetric_pd_sparsity_and_matrix_free(bc):
    g = fem.Grid(4, 2, 2, bc)
    rng = np.random.default_rng(1)
    w = rng.uniform(1e-3, 1.0, g.m)
    Ke = fem.element_stiffness()
    K = fem.assemble_K(g, w, Ke)
    assert abs(K - K.T).max() < 1e-15
    assert np.linalg.eigvalsh(K.toarray()).min() > 0
    assert np.diff(K.indptr).max() <= 81            # at most 81 non-zeros per row in 3D (Section 5.2)
    x = rng.standard_normal(g.n)
    assert np.allclose(fem.apply_K_elementwise(g, w, Ke, x), K @ x, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners", "bridge_edges"])
def test_rows_at_nodes_equal_assembled_rows(bc):
    """The row-by-row product used for sampled checks at full size equals the rows of the assembled K(w) x (the
    plain definition), on every node of a small grid: interior, faces, edges, corners and supported nodes."""
    g = fem.Grid(5, 3, 2, bc)
    rng = np.random.default_rng(4)
    w = rng.uniform(1e-3, 1.0, g.m)
    Ke = fem.element_stiffness()
    x = rng.standard_normal(g.n)
    ref = (fem.assemble_K(g, w, Ke) @ x).reshape(-1, 3)
    nodes = np.arange(g.nnode)
    assert np.allclose(fem.apply_K_at_nodes(g, w, Ke, x, nodes), ref, rtol=1e-13, atol=1e-13)
    sub = rng.permutation(g.nnode)[:17]
    assert np.allclose(fem.apply_K_at_nodes(g, w, Ke, x, sub), ref[sub], rtol=1e-13, atol=1e-13)


def test_compliance_identity():
    """At equilibrium f^T u = u^T K(rho) u (eq. (1) with K(rho) u = f)."""
    g = fem.Grid(8, 4, 4, "cantilever")
    rng = np.random.default_rng(2)
    w = rng.uniform(1e-3, 1.0, g.m)
    K = fem.assemble_K(g, w, fem.element_stiffness())
    f = rng.standard_normal(g.n)
    f[g.fixed_dofs()] = 0.0
    u = spla.spsolve(K.tocsc(), f)
    assert abs(f @ u - u @ (K @ u)) < 1e-10 * abs(f @ u)


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners", "bridge_edges"])
def test_prolongation_reproduces_linear_fields(bc):
    fine = fem.Grid(4, 4, 2, bc)
    coarse = fine.coarse()
    P = fem.prolongation(fine)
    G = np.array([[0.3, -1.0, 0.5], [2.0, 0.1, -0.7], [0.0, 1.5, 1.0]])
    c0 = np.array([0.2, -0.4, 1.1])
    uc = (coarse.node_ijk() * coarse.h @ G.T + c0).ravel()
    uf = (fine.node_ijk() * fine.h @ G.T + c0).ravel()
    uc[coarse.fixed_dofs()] = 0.0
    free_f = ~fine.fixed_dofs()
    # on fine nodes whose parents are all free, interpolation is exact
    Pc = fem.prolongation(fem.Grid(4, 4, 2, "free"))
    got = Pc @ (fem.Grid(2, 2, 1, "free").node_ijk() * 2.0 @ G.T + c0).ravel()
    assert np.allclose(got, (fem.Grid(4, 4, 2, "free").node_ijk() @ G.T + c0).ravel(), atol=1e-14)
    # with supports, fixed fine rows are zero and P only reads free coarse dofs
    Pu = P @ uc
    assert np.all(Pu[~free_f] == 0.0)
    assert P.shape == (fine.n, coarse.n)
    assert np.all(P.toarray()[:, coarse.fixed_dofs()] == 0.0)
    # weights are products of 1D weights {1, 1/2}: only 1, 1/2, 1/4, 1/8 occur
    assert set(np.unique(P.data)) <= {1.0, 0.5, 0.25, 0.125}


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners", "bridge_edges"])
def test_galerkin_equals_rediscretisation_for_childwise_constant_density(bc):
    """For nested conforming spaces the Galerkin product P^T K_h P equals the coarse-grid assembly (edge 2h) of the
    same bilinear form when the density is constant on each coarse element."""
    fine = fem.Grid(4, 4, 4, bc)
    coarse = fine.coarse()
    rng = np.random.default_rng(3)
    wc = rng.uniform(0.1, 1.0, coarse.m)
    fe = fine.elem_ijk() // 2
    wf = wc[fe[:, 0] + coarse.nx * (fe[:, 1] + coarse.ny * fe[:, 2])]
    Kf = fem.assemble_K(fine, wf, fem.element_stiffness(h=1.0))
    P = fem.prolongation(fine)
    Kg = (P.T @ Kf @ P).toarray()
    fixed_c = coarse.fixed_dofs()
    Kg[fixed_c, fixed_c] = 1.0
    Kc = fem.assemble_K(coarse, wc, fem.element_stiffness(h=2.0)).toarray()
    assert np.max(np.abs(Kg - Kc)) < 1e-13
