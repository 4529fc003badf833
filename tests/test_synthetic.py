"""The seeded input recipes (synthetic/): each generator meets the contract its docstring states — load totals
and moments, exact volume fractions inside the density bounds, the supports of the displacement field — and is a
pure function of its seed (no GPU, no oracle arithmetic)."""
import numpy as np
import pytest

import synthetic
from oracle import fem


def _forces(f):
    return f.reshape(-1, 3)


@pytest.mark.parametrize("kind", ["end_edge", "top_traction", "point_end", "end_face"])
def test_loads_are_downward_with_unit_total(kind):
    nx, ny, nz = 8, 4, 6
    F = _forces(synthetic.load_vector(nx, ny, nz, kind))
    assert abs(F[:, 2].sum() + 1.0) < 1e-14
    assert np.all(F[:, 2] <= 0.0) and np.all(F[:, :2] == 0.0)
    g = fem.Grid(nx, ny, nz, "cantilever")
    ijk = g.node_ijk()
    loaded = F[:, 2] != 0.0
    if kind in ("end_edge", "point_end", "end_face"):
        assert np.all(ijk[loaded, 0] == nx)            # on the free end of the cantilever
    if kind == "top_traction":
        assert np.all(ijk[loaded, 2] == nz)


def test_torsion_is_a_pure_unit_couple():
    nx, ny, nz = 8, 4, 6
    F = _forces(synthetic.load_vector(nx, ny, nz, "torsion"))
    g = fem.Grid(nx, ny, nz, "cantilever")
    ijk = g.node_ijk().astype(float)
    assert np.abs(F.sum(axis=0)).max() < 1e-14         # net force zero
    y, z = ijk[:, 1] - ny / 2.0, ijk[:, 2] - nz / 2.0
    moment_x = (y * F[:, 2] - z * F[:, 1]).sum()
    assert abs(moment_x - 1.0) < 1e-13


def test_uniform_rescaled_density_has_exact_mean_inside_bounds():
    rho = synthetic.density_uniform_rescaled(4096, 0.3, 0)
    assert abs(rho.mean() - 0.3) < 1e-14
    assert rho.min() >= 1e-3 and rho.max() <= 1.0
    assert np.array_equal(rho, synthetic.density_uniform_rescaled(4096, 0.3, 0))
    assert not np.array_equal(rho, synthetic.density_uniform_rescaled(4096, 0.3, 1))


def test_bump_density_meets_volume_fraction_and_bounds():
    rho = synthetic.density_bumps(16, 8, 8, 0.2, 0)
    assert abs(rho.sum() - 0.2 * rho.size) <= 1e-10 * rho.size
    assert rho.min() >= 1e-3 and rho.max() <= 1.0


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners", "bridge_edges"])
def test_smooth_displacement_contract(bc):
    g = fem.Grid(8, 4, 4, bc)
    fixed = g.fixed_dofs()
    u = synthetic.smooth_displacement(8, 4, 4, 5, 0.7, fixed)
    assert u.shape == (g.n,)
    assert np.all(u[fixed] == 0.0)
    free = u[~fixed]
    assert 0.0 < np.abs(free).max() <= 0.7 + 1e-15
    assert np.array_equal(u, synthetic.smooth_displacement(8, 4, 4, 5, 0.7, fixed))


def test_workload_sizes_match_their_grids():
    for w in synthetic.WORKLOADS.values():
        assert w.m == w.nx * w.ny * w.nz
        assert w.n == 3 * (w.nx + 1) * (w.ny + 1) * (w.nz + 1)
        f = 1 << (w.levels - 1)
        assert w.nx % f == 0 and w.ny % f == 0 and w.nz % f == 0
        # the coarsest grid of every workload stays small enough for the dense bordered solve
        assert 3 * (w.nx // f + 1) * (w.ny // f + 1) * (w.nz // f + 1) <= 1500


@pytest.mark.parametrize("bc", ["cantilever", "bridge_corners", "bridge_edges", "free"])
def test_supported_dofs_match_the_oracle_grid(bc):
    for dims in ((8, 4, 4), (5, 3, 2)):
        assert np.array_equal(synthetic.supported_dofs(*dims, bc), fem.Grid(*dims, bc).fixed_dofs())


def test_state_displacement_recipes():
    w = synthetic.WORKLOADS["bridge128"]
    u = synthetic.state_displacement(w)
    assert u.shape == (w.n,) and abs(np.abs(u).max() - 1.0) < 1e-15
    assert np.all(u[synthetic.supported_dofs(w.nx, w.ny, w.nz, w.bc)] == 0.0)
    assert np.array_equal(u, synthetic.state_displacement(w))
    assert synthetic.state_displacement(synthetic.WORKLOADS["cant64"]) is None
