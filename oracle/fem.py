"""Q1 hexahedral linear elasticity on a structured grid of unit cubes (oracle; test infrastructure only).

Follows Section 5.2 of the paper (trilinear displacements, piecewise-constant density, regular 8-way refinement,
27-point prolongation) and the problem statement of eq. (1): K(rho) = sum_i rho_i K_i, where K_i is the element
stiffness matrix of element i placed into the global dofs.

Conventions (identical to the library's ABI, which is documented in include/pbm.h):
    node id  = i + (nx+1) * (j + (ny+1) * k)
    dof      = 3 * node + c
    element  = i + nx * (j + ny * k)
    local node of an element: a = ix + 2*iy + 4*iz, at (i+ix, j+iy, k+iz)
    local dof: 3*a + c
Supports (Section 6): "cantilever" clamps every node on x = 0; "bridge_corners" clamps the four corner nodes of the
bottom face z = 0; "bridge_edges" clamps the two bottom edges x = 0 and x = nx of the face z = 0.
Supported (Dirichlet) dofs are eliminated: their rows and columns become those of the identity.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------------------------------------------
# element stiffness
# ----------------------------------------------------------------------------------------------------------------


def local_offsets() -> np.ndarray:
    """(8, 3) integer offsets (ix, iy, iz) of the local nodes a = ix + 2 iy + 4 iz."""
    return np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)


def isotropic_D(E: float, nu: float) -> np.ndarray:
    """6x6 isotropic elasticity matrix in Voigt order (xx, yy, zz, xy, yz, xz) with engineering shear strains."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for c in range(3):
        D[c, c] += 2.0 * mu
    for c in range(3, 6):
        D[c, c] = mu
    return D


def _shape_gradients(xi: np.ndarray) -> np.ndarray:
    """Gradients (8, 3) of the trilinear shape functions N_a(xi) = l_ix(x) l_iy(y) l_iz(z) on [0,1]^3,
    l_0(t) = 1 - t, l_1(t) = t."""
    off = local_offsets()
    g = np.zeros((8, 3))
    for a in range(8):
        l = [xi[d] if off[a, d] else 1.0 - xi[d] for d in range(3)]
        dl = [1.0 if off[a, d] else -1.0 for d in range(3)]
        g[a, 0] = dl[0] * l[1] * l[2]
        g[a, 1] = l[0] * dl[1] * l[2]
        g[a, 2] = l[0] * l[1] * dl[2]
    return g


def strain_displacement(xi: np.ndarray, h: float = 1.0) -> np.ndarray:
    """B (6 x 24): engineering strain at reference point xi of a cube of edge h, for the local dof order 3a + c."""
    G = _shape_gradients(xi) / h
    B = np.zeros((6, 24))
    for a in range(8):
        dx, dy, dz = G[a]
        B[0, 3 * a + 0] = dx
        B[1, 3 * a + 1] = dy
        B[2, 3 * a + 2] = dz
        B[3, 3 * a + 0], B[3, 3 * a + 1] = dy, dx
        B[4, 3 * a + 1], B[4, 3 * a + 2] = dz, dy
        B[5, 3 * a + 0], B[5, 3 * a + 2] = dz, dx
    return B


def element_stiffness(E: float = 1.0, nu: float = 0.3, h: float = 1.0, order: int = 2) -> np.ndarray:
    """24x24 Q1 element stiffness  K_e = int_cube B^T D B dx  by order x order x order Gauss quadrature.
    Two points per direction integrate this (degree <= 2 per direction) integrand exactly."""
    pts, wts = np.polynomial.legendre.leggauss(order)
    pts = 0.5 * (pts + 1.0)   # map [-1,1] -> [0,1]
    wts = 0.5 * wts
    D = isotropic_D(E, nu)
    K = np.zeros((24, 24))
    for a, wa in zip(pts, wts):
        for b, wb in zip(pts, wts):
            for c, wc in zip(pts, wts):
                B = strain_displacement(np.array([a, b, c]), h)
                K += (wa * wb * wc * h ** 3) * (B.T @ D @ B)
    return K


def rigid_body_modes(h: float = 1.0) -> np.ndarray:
    """(24, 6): three translations and three linearised rotations of one cube, sampled at its nodes."""
    X = local_offsets().astype(float) * h
    R = np.zeros((24, 6))
    for a in range(8):
        x, y, z = X[a]
        for c in range(3):
            R[3 * a + c, c] = 1.0
        R[3 * a:3 * a + 3, 3] = [-y, x, 0.0]   # rotation about z
        R[3 * a:3 * a + 3, 4] = [0.0, -z, y]   # rotation about x
        R[3 * a:3 * a + 3, 5] = [z, 0.0, -x]   # rotation about y
    return R


# ----------------------------------------------------------------------------------------------------------------
# structured grid
# ----------------------------------------------------------------------------------------------------------------


class Grid:
    """Structured nx x ny x nz grid of cubes of edge h with a support kind."""

    def __init__(self, nx: int, ny: int, nz: int, bc: str = "cantilever", h: float = 1.0):
        self.nx, self.ny, self.nz, self.bc, self.h = nx, ny, nz, bc, h
        self.nnode = (nx + 1) * (ny + 1) * (nz + 1)
        self.n = 3 * self.nnode
        self.m = nx * ny * nz

    def node_id(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def node_ijk(self) -> np.ndarray:
        """(nnode, 3) integer coordinates of every node, in node-id order."""
        k, j, i = np.meshgrid(np.arange(self.nz + 1), np.arange(self.ny + 1), np.arange(self.nx + 1),
                              indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def elem_ijk(self) -> np.ndarray:
        k, j, i = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def elem_nodes(self) -> np.ndarray:
        """(m, 8) node ids of every element in local order a = ix + 2 iy + 4 iz."""
        e = self.elem_ijk()
        off = local_offsets()
        out = np.empty((self.m, 8), dtype=np.int64)
        for a in range(8):
            out[:, a] = self.node_id(e[:, 0] + off[a, 0], e[:, 1] + off[a, 1], e[:, 2] + off[a, 2])
        return out

    def elem_dofs(self) -> np.ndarray:
        """(m, 24) global dofs of every element, local dof 3a + c."""
        nodes = self.elem_nodes()
        return (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(self.m, 24)

    def fixed_nodes(self) -> np.ndarray:
        """Boolean (nnode,) — True where the node is supported in all three directions."""
        ijk = self.node_ijk()
        i, j, k = ijk[:, 0], ijk[:, 1], ijk[:, 2]
        if self.bc == "cantilever":
            return i == 0
        if self.bc == "bridge_corners":
            return (k == 0) & ((i == 0) | (i == self.nx)) & ((j == 0) | (j == self.ny))
        if self.bc == "bridge_edges":
            return (k == 0) & ((i == 0) | (i == self.nx))
        if self.bc == "free":
            return np.zeros(self.nnode, dtype=bool)
        raise ValueError(self.bc)

    def fixed_dofs(self) -> np.ndarray:
        """Boolean (n,) Dirichlet mask."""
        return np.repeat(self.fixed_nodes(), 3)

    def n_free(self) -> int:
        return int(self.n - self.fixed_dofs().sum())

    def coarse(self) -> "Grid":
        assert self.nx % 2 == 0 and self.ny % 2 == 0 and self.nz % 2 == 0
        return Grid(self.nx // 2, self.ny // 2, self.nz // 2, self.bc, 2.0 * self.h)


# ----------------------------------------------------------------------------------------------------------------
# assembly and matrix-free application of K(w) = sum_i w_i K_i
# ----------------------------------------------------------------------------------------------------------------


def assemble_unconstrained(g: Grid, w: np.ndarray, Ke: np.ndarray) -> sp.csr_matrix:
    """sum_i w_i K_i as CSR (no supports applied). COO triplets -> CSR sums duplicates."""
    dofs = g.elem_dofs()
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    vals = (w[:, None, None] * Ke[None, :, :]).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(g.n, g.n)).tocsr()


def apply_supports(A: sp.spmatrix, fixed: np.ndarray) -> sp.csr_matrix:
    """Eliminate supported dofs: zero their rows and columns and put 1 on the diagonal."""
    free = (~fixed).astype(float)
    M = sp.diags(free)
    return (M @ A @ M + sp.diags(fixed.astype(float))).tocsr()


def assemble_K(g: Grid, w: np.ndarray, Ke: np.ndarray) -> sp.csr_matrix:
    """K(w) with supported dofs eliminated (identity rows/cols)."""
    return apply_supports(assemble_unconstrained(g, w, Ke), g.fixed_dofs())


def apply_K_elementwise(g: Grid, w: np.ndarray, Ke: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Matrix-free y = K(w) x with supported dofs eliminated: y = M (sum_e w_e G_e^T K_e G_e) M x + (I - M) x."""
    fixed = g.fixed_dofs()
    xm = np.where(fixed, 0.0, x)
    dofs = g.elem_dofs()
    ye = (xm[dofs] @ Ke) * w[:, None]           # Ke symmetric
    y = np.bincount(dofs.ravel(), weights=ye.ravel(), minlength=g.n)
    return np.where(fixed, x, y)


def apply_K_at_nodes(g: Grid, w: np.ndarray, Ke: np.ndarray, x: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Rows of y = K(w) x at the given node ids, shape (len(nodes), 3), each summed from the at most 8 elements
    around its node: the node is local corner a of element e, and y_node = sum_e w_e (K_e x_e)[3a : 3a + 3] with
    supported dofs of x zeroed; a supported node keeps y = x. For sampled checks at sizes where the full product
    is not wanted."""
    xm = np.where(g.fixed_dofs(), 0.0, x)
    fixed_n = g.fixed_nodes()
    off = local_offsets()
    out = np.zeros((len(nodes), 3))
    for r, nd in enumerate(np.asarray(nodes, dtype=np.int64)):
        i = nd % (g.nx + 1)
        j = (nd // (g.nx + 1)) % (g.ny + 1)
        k = nd // ((g.nx + 1) * (g.ny + 1))
        if fixed_n[nd]:
            out[r] = x[3 * nd:3 * nd + 3]
            continue
        for a in range(8):
            ei, ej, ek = i - off[a, 0], j - off[a, 1], k - off[a, 2]
            if not (0 <= ei < g.nx and 0 <= ej < g.ny and 0 <= ek < g.nz):
                continue
            e = ei + g.nx * (ej + g.ny * ek)
            xe = np.concatenate([xm[3 * q:3 * q + 3] for q in
                                 (g.node_id(ei + off[b, 0], ej + off[b, 1], ek + off[b, 2]) for b in range(8))])
            out[r] += w[e] * (Ke[3 * a:3 * a + 3] @ xe)
    return out


def element_energies(g: Grid, Ke: np.ndarray, u: np.ndarray, v: np.ndarray | None = None) -> np.ndarray:
    """Per-element bilinear forms  u_e^T K_e v_e  (v = u if omitted); u, v full-length nodal vectors."""
    dofs = g.elem_dofs()
    ue = u[dofs]
    ve = ue if v is None else v[dofs]
    return np.einsum("ei,ij,ej->e", ue, Ke, ve)


# ----------------------------------------------------------------------------------------------------------------
# 27-point prolongation (trilinear interpolation from a coarse grid to its 8-way refinement)
# ----------------------------------------------------------------------------------------------------------------


def prolongation(fine: Grid) -> sp.csr_matrix:
    """P (n_fine x n_coarse): a fine node at integer position (I, J, K) takes, per direction, the coarse node I/2 if I
    is even, or the average of coarse nodes (I-1)/2 and (I+1)/2 if I is odd; the 3D weight is the product.
    Supports are applied on both sides (P' = M_f P M_c, M = free-dof mask)."""
    coarse = fine.coarse()
    fijk = fine.node_ijk()
    rows, cols, vals = [], [], []
    for fn in range(fine.nnode):
        I = fijk[fn]
        per_dim = []
        for d in range(3):
            if I[d] % 2 == 0:
                per_dim.append([(I[d] // 2, 1.0)])
            else:
                per_dim.append([((I[d] - 1) // 2, 0.5), ((I[d] + 1) // 2, 0.5)])
        for (ci, wi) in per_dim[0]:
            for (cj, wj) in per_dim[1]:
                for (ck, wk) in per_dim[2]:
                    cn = coarse.node_id(ci, cj, ck)
                    for c in range(3):
                        rows.append(3 * fn + c)
                        cols.append(3 * cn + c)
                        vals.append(wi * wj * wk)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(fine.n, coarse.n))
    Mf = sp.diags((~fine.fixed_dofs()).astype(float))
    Mc = sp.diags((~coarse.fixed_dofs()).astype(float))
    return (Mf @ P @ Mc).tocsr()
