"""Seeded synthetic problem data for the reduced-Newton MG-MINRES workloads.

This module is shared by the CPU oracle's tests, the GPU parity tests and the benchmark. It holds only problem
*data*: grid shapes, the kind of support, nodal load vectors, density fields and the seeded synthetic Newton state.
None of the method's arithmetic lives here (no element stiffness, no penalty function, no operator, no solver), so
neither side of a parity test can inherit a mistake from the other through this file.

Layout conventions (the library's ABI, restated here only to place loads on nodes):
    node id  = i + (nx+1) * (j + (ny+1) * k),   0 <= i <= nx, 0 <= j <= ny, 0 <= k <= nz
    dof      = 3 * node + c,                     c = 0 (x), 1 (y), 2 (z)
    element  = i + nx * (j + ny * k),            0 <= i < nx, ...

The workloads follow the paper's two examples (Section 6: a cantilever clamped on the face x = 0 and loaded at the
far end; a "bridge" supported at the four bottom corners and loaded on the top face) on unit-cube grids.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "BATCH_WORKLOADS", "load_vector", "density_uniform_rescaled", "density_bumps",
    "density_for", "synthetic_state", "random_state", "smooth_displacement", "node_count", "dof_count", "elem_count",
    "supported_dofs", "state_displacement",
]


def node_count(nx: int, ny: int, nz: int) -> int:
    return (nx + 1) * (ny + 1) * (nz + 1)


def dof_count(nx: int, ny: int, nz: int) -> int:
    return 3 * node_count(nx, ny, nz)


def elem_count(nx: int, ny: int, nz: int) -> int:
    return nx * ny * nz


def supported_dofs(nx: int, ny: int, nz: int, bc: str) -> np.ndarray:
    """Boolean (n,) mask of the supported dofs of a workload's boundary condition (the placement of the supports,
    like the placement of the loads below): "cantilever" every node of the face x = 0; "bridge_corners" the four
    corner nodes of the bottom face z = 0; "bridge_edges" the two bottom edges {x = 0, z = 0} and {x = nx, z = 0};
    "free" none. All three dofs of a supported node are supported."""
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    if bc == "cantilever":
        node = i == 0
    elif bc == "bridge_corners":
        node = (k == 0) & ((i == 0) | (i == nx)) & ((j == 0) | (j == ny))
    elif bc == "bridge_edges":
        node = (k == 0) & ((i == 0) | (i == nx))
    elif bc == "free":
        node = np.zeros(i.size, dtype=bool)
    else:
        raise ValueError(f"unknown support {bc!r}")
    return np.repeat(node, 3)


def _face_weights(n: int) -> np.ndarray:
    """Consistent Q1 weights along one edge of a face: 1/2 at the two ends, 1 inside (they sum to n)."""
    w = np.ones(n + 1)
    w[0] = w[-1] = 0.5
    return w


def load_vector(nx: int, ny: int, nz: int, kind: str) -> np.ndarray:
    """Nodal load vector f (length 3*(nx+1)(ny+1)(nz+1), float64) for one load case.

    kinds
      end_edge     : -z, total 1, split equally over the nodes of the bottom edge at x = nx (k = 0, j = 0..ny).
      top_traction : -z uniform traction on the top face z = nz, consistent weights (1, 1/2, 1/4 interior/edge/corner)
                     scaled so that the total force is 1.
      point_end    : -z, magnitude 1, at node (nx, ny//2, nz//2).
      end_face     : -z, total 1, uniform traction on the face x = nx with consistent weights.
      torsion      : couple about the x axis on the face x = nx: nodal force s * (0, -(z - zc), (y - yc)) * weight,
                     net force 0, moment 1.
    """
    f = np.zeros(dof_count(nx, ny, nz))
    sx, sxy = nx + 1, (nx + 1) * (ny + 1)
    if kind == "end_edge":
        for j in range(ny + 1):
            f[3 * (nx + sx * j) + 2] -= 1.0 / (ny + 1)
    elif kind == "top_traction":
        wi, wj = _face_weights(nx), _face_weights(ny)
        t = 1.0 / (nx * ny)
        for j in range(ny + 1):
            for i in range(nx + 1):
                f[3 * (i + sx * j + sxy * nz) + 2] -= t * wi[i] * wj[j]
    elif kind == "point_end":
        f[3 * (nx + sx * (ny // 2) + sxy * (nz // 2)) + 2] -= 1.0
    elif kind == "end_face":
        wj, wk = _face_weights(ny), _face_weights(nz)
        t = 1.0 / (ny * nz)
        for k in range(nz + 1):
            for j in range(ny + 1):
                f[3 * (nx + sx * j + sxy * k) + 2] -= t * wj[j] * wk[k]
    elif kind == "torsion":
        wj, wk = _face_weights(ny), _face_weights(nz)
        yc, zc = ny / 2.0, nz / 2.0
        num = 0.0
        for k in range(nz + 1):
            for j in range(ny + 1):
                num += wj[j] * wk[k] * ((j - yc) ** 2 + (k - zc) ** 2)
        s = 1.0 / num
        for k in range(nz + 1):
            for j in range(ny + 1):
                node = nx + sx * j + sxy * k
                f[3 * node + 1] += -s * (k - zc) * wj[j] * wk[k]
                f[3 * node + 2] += s * (j - yc) * wj[j] * wk[k]
    else:
        raise ValueError(f"unknown load kind {kind!r}")
    return f


def density_uniform_rescaled(m: int, vf: float, seed: int, lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    """rho_i ~ U[lo, hi] (numpy PCG64, given seed), then an affine map toward `lo` so that mean(rho) = vf exactly
    while rho stays inside [lo, hi]:  rho <- lo + (rho - lo) * (vf - lo) / (mean(rho) - lo)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(lo, hi, size=m)
    rho = lo + (rho - lo) * (vf - lo) / (rho.mean() - lo)
    return rho


def density_bumps(nx: int, ny: int, nz: int, vf: float, seed: int, nbumps: int = 32, lo: float = 1e-3,
                  hi: float = 1.0) -> np.ndarray:
    """Smooth random field: sum of `nbumps` Gaussian bumps (centres uniform in the box, per-axis sigma uniform in
    [0.05, 0.2] * (nx, ny, nz), amplitudes uniform in [0.5, 1]); normalised to max 1; then a scale s found by
    bisection so that sum(clip(s * field, lo, hi)) = vf * m to 1e-12 relative."""
    rng = np.random.default_rng(seed)
    dims = np.array([nx, ny, nz], dtype=float)
    centres = rng.uniform(0.0, 1.0, size=(nbumps, 3)) * dims
    sig = rng.uniform(0.05, 0.2, size=(nbumps, 3)) * dims
    amp = rng.uniform(0.5, 1.0, size=nbumps)
    # element centres, element index e = i + nx*(j + ny*k)
    zc, yc, xc = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    xc, yc, zc = xc.ravel(), yc.ravel(), zc.ravel()
    field_ = np.zeros(nx * ny * nz)
    for b in range(nbumps):
        field_ += amp[b] * np.exp(-0.5 * (((xc - centres[b, 0]) / sig[b, 0]) ** 2
                                          + ((yc - centres[b, 1]) / sig[b, 1]) ** 2
                                          + ((zc - centres[b, 2]) / sig[b, 2]) ** 2))
    field_ /= field_.max()
    target = vf * field_.size

    def total(s):
        return np.clip(s * field_, lo, hi).sum()

    a, b = 0.0, 1.0
    while total(b) < target:
        b *= 2.0
    for _ in range(200):
        mid = 0.5 * (a + b)
        if total(mid) < target:
            a = mid
        else:
            b = mid
        if abs(total(b) - target) <= 1e-12 * target:
            break
    return np.clip(b * field_, lo, hi)


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: grid, support, loads, density recipe and solver settings."""
    name: str
    nx: int
    ny: int
    nz: int
    bc: str                      # "cantilever" | "bridge_corners" | "bridge_edges"
    loads: tuple                 # load kinds (one reduced system per load case)
    vf: float                    # volume fraction V / m
    density: str                 # "uniform" | "uniform_rescaled" | "bumps"
    seed: int = 0
    levels: int = 3
    rtol: float = 1e-8
    rho_lo: float = 1e-3
    rho_up: float = 1.0
    E: float = 1.0
    nu: float = 0.3
    extra: dict = field(default_factory=dict, hash=False, compare=False)

    @property
    def m(self) -> int:
        return elem_count(self.nx, self.ny, self.nz)

    @property
    def n(self) -> int:
        return dof_count(self.nx, self.ny, self.nz)

    @property
    def V(self) -> float:
        return self.vf * self.m


WORKLOADS = {
    # 16x8x8 cantilever, full PBM, MINRES to 1e-10, 3 levels (coarsest 4x2x2)
    "cant16": Workload("cant16", 16, 8, 8, "cantilever", ("end_edge",), 0.3, "uniform", 0, 3, 1e-10),
    # 64x32x32 cantilever, single reduced-Newton solve, 5 levels, rtol 1e-8
    "cant64": Workload("cant64", 64, 32, 32, "cantilever", ("end_edge",), 0.3, "uniform_rescaled", 0, 5, 1e-8),
    # 128x64x64 bridge (four bottom corners), top traction, Gaussian-bump density at vf 0.2, 6 levels (4x2x2 coarse);
    # its Newton state's displacement is the seeded smooth field (seed 5, max |u| = 1)
    "bridge128": Workload("bridge128", 128, 64, 64, "bridge_corners", ("top_traction",), 0.2, "bumps", 0, 6, 1e-8,
                          extra={"u": ("smooth", 5, 1.0)}),
    # 256x128x128 cantilever, distributed end load, vf 0.15, 7 levels
    "cant256": Workload("cant256", 256, 128, 128, "cantilever", ("end_face",), 0.15, "uniform", 0, 7, 1e-8),
    # small cases used by parity tests
    "cant8": Workload("cant8", 8, 4, 4, "cantilever", ("end_edge",), 0.3, "uniform_rescaled", 0, 2, 1e-10),
    "bridge16": Workload("bridge16", 16, 8, 8, "bridge_corners", ("top_traction",), 0.2, "bumps", 0, 3, 1e-10),
    "cant32": Workload("cant32", 32, 16, 16, "cantilever", ("end_edge",), 0.3, "uniform_rescaled", 0, 4, 1e-8),
}

# Twelve instances of uneven size (3 each of 32x16x16, 48x24x24, 64x32x32, 96x48x48), four load cases each.
_BATCH_LOADS = ("point_end", "end_face", "top_traction", "torsion")
BATCH_WORKLOADS = tuple(
    Workload(f"batch{idx}", *dims, "cantilever", _BATCH_LOADS, 0.3, "uniform_rescaled", idx,
             {32: 4, 48: 4, 64: 5, 96: 5}[dims[0]], 1e-8)
    for idx, dims in enumerate([(32, 16, 16)] * 3 + [(48, 24, 24)] * 3 + [(64, 32, 32)] * 3 + [(96, 48, 48)] * 3)
)


def density_for(w: Workload) -> np.ndarray:
    if w.density == "uniform":
        return np.full(w.m, w.vf)
    if w.density == "uniform_rescaled":
        return density_uniform_rescaled(w.m, w.vf, w.seed, w.rho_lo, w.rho_up)
    if w.density == "bumps":
        return density_bumps(w.nx, w.ny, w.nz, w.vf, w.seed, lo=w.rho_lo, hi=w.rho_up)
    raise ValueError(w.density)


def state_displacement(w: Workload) -> np.ndarray | None:
    """The displacement of a single-solve workload's synthetic Newton state when the recipe fixes it (the seeded
    smooth field of `smooth_displacement`, zero on the supported dofs); None when the state uses the equilibrium
    displacement of K(rho) u = f, which the caller computes."""
    spec = w.extra.get("u")
    if spec is None:
        return None
    kind, seed, amplitude = spec
    if kind != "smooth":
        raise ValueError(kind)
    return smooth_displacement(w.nx, w.ny, w.nz, seed, amplitude, supported_dofs(w.nx, w.ny, w.nz, w.bc))


def synthetic_state(w: Workload, u: np.ndarray) -> dict:
    """The synthetic Newton state of a single-solve workload: PBM multipliers all 1 (mu_lo = mu_up = 1), penalty
    parameters all 1, alpha = 1 and nu_lo = nu_up = 1 (the paper's initial values), rho from the density recipe,
    and u supplied by the caller (`state_displacement`, else the equilibrium displacement of K(rho) u = f)."""
    m = w.m
    return dict(u=np.asarray(u, dtype=np.float64), alpha=1.0, nu_lo=np.ones(m), nu_up=np.ones(m),
                rho=density_for(w), mu_lo=np.ones(m), mu_up=np.ones(m), p=1.0, q_lo=1.0, q_up=1.0,
                V=w.V, rho_lo=w.rho_lo, rho_up=w.rho_up)


def smooth_displacement(nx: int, ny: int, nz: int, seed: int, amplitude: float = 1.0,
                        fixed_dofs: np.ndarray | None = None) -> np.ndarray:
    """A seeded smooth nodal field (length 3 (nx+1)(ny+1)(nz+1)): per component the sum of 4 products of
    low-frequency sines in x, y and z with random wave numbers (1 to 3 half waves across the box), phases and
    amplitudes, scaled to max |u| = amplitude and zero on `fixed_dofs`."""
    rng = np.random.default_rng(seed)
    k, j, i = np.meshgrid(np.arange(nz + 1) / max(nz, 1), np.arange(ny + 1) / max(ny, 1),
                          np.arange(nx + 1) / max(nx, 1), indexing="ij")
    u = np.zeros((k.size, 3))
    for c in range(3):
        for _ in range(4):
            fx, fy, fz = rng.integers(1, 4, size=3)
            px, py, pz = rng.uniform(0.0, 2.0 * np.pi, size=3)
            u[:, c] += rng.uniform(0.5, 1.0) * (np.sin(np.pi * fx * i + px) * np.sin(np.pi * fy * j + py)
                                                * np.sin(np.pi * fz * k + pz)).ravel()
    u = u.ravel()
    u *= amplitude / np.abs(u).max()
    if fixed_dofs is not None:
        u[fixed_dofs] = 0.0
    return u


def random_state(nx: int, ny: int, nz: int, seed: int, u_scale: float = 1.0, p: float = 1.0, q: float = 1.0,
                 fixed_dofs: np.ndarray | None = None) -> dict:
    """A random (not optimal) Newton state for operator tests: u with zeros on `fixed_dofs`, alpha, nu, rho and mu
    drawn so that both branches of the penalty function are exercised."""
    rng = np.random.default_rng(seed)
    m, n = elem_count(nx, ny, nz), dof_count(nx, ny, nz)
    u = rng.standard_normal(n) * u_scale
    if fixed_dofs is not None:
        u[fixed_dofs] = 0.0
    return dict(u=u, alpha=float(rng.uniform(0.5, 2.0)), nu_lo=rng.uniform(0.0, 2.0, m),
                nu_up=rng.uniform(0.0, 2.0, m), rho=rng.uniform(1e-3, 1.0, m), mu_lo=rng.uniform(0.2, 2.0, m),
                mu_up=rng.uniform(0.2, 2.0, m), p=p, q_lo=q, q_up=q, V=0.3 * m, rho_lo=1e-3, rho_up=1.0)


def ip_random_state(nx: int, ny: int, nz: int, seed: int, fixed_dofs: np.ndarray | None = None, u_scale: float = 0.5,
                    rho_lo: float = 1e-3, rho_up: float = 1.0) -> dict:
    """A strictly feasible random point of the interior-point method for operator tests: rho inside (rho_lo, rho_up),
    nu_lo, nu_up > 0, u with zeros on `fixed_dofs`, and barrier parameters r, s."""
    rng = np.random.default_rng(seed)
    m, n = elem_count(nx, ny, nz), dof_count(nx, ny, nz)
    u = rng.standard_normal(n) * u_scale
    if fixed_dofs is not None:
        u[fixed_dofs] = 0.0
    rho = rho_lo + (rho_up - rho_lo) * rng.uniform(0.05, 0.95, m)
    return dict(u=u, alpha=float(rng.uniform(-1.0, 1.0)), rho=rho, nu_lo=rng.uniform(0.1, 2.0, m),
                nu_up=rng.uniform(0.1, 2.0, m), V=0.3 * m, rho_lo=rho_lo, rho_up=rho_up,
                r=float(rng.uniform(0.01, 0.1)), s=float(rng.uniform(0.01, 0.1)))

