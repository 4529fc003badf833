"""pbm_apply_K_noalloc: K(w) x for callers that cannot allocate device memory.

Such callers (loops that must not allocate after start-up, host frameworks whose own allocator owns all device
memory, plug-ins inside such hosts) cannot create a grid handle, because pbm_create_grid allocates. The
no-allocation entry point keeps its scratch in a fixed device array inside the library. This file checks that its
result equals the handle-based pbm_apply_K and the oracle's element-by-element product on two calls in a row (the
array keeps the previous call's contents), that a different grid shape in between does not disturb it, that device
memory stays as it was around a call, and that a grid too large for the array is rejected before any launch. It
sorts last so that a run stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from oracle import fem

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.double().cpu().numpy() if isinstance(a, torch.Tensor) else a
    b = b.double().cpu().numpy() if isinstance(b, torch.Tensor) else b
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def pkg():
    from paper_1904_06556_gb300 import build
    build.build()
    import paper_1904_06556_gb300 as p
    return p


def _case(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    m, n = nx * ny * nz, 3 * (nx + 1) * (ny + 1) * (nz + 1)
    w, x = rng.uniform(1e-3, 1.0, m), rng.standard_normal(n)
    return w, x, torch.as_tensor(w, device="cuda"), torch.as_tensor(x, device="cuda")


def test_noalloc_apply_equals_handle_apply_and_oracle_on_two_calls(pkg):
    nx, ny, nz = 34, 10, 6
    w_h, x_h, w, x = _case(nx, ny, nz, 11)
    oref = fem.apply_K_elementwise(fem.Grid(nx, ny, nz, "bridge_corners"), w_h, fem.element_stiffness(), x_h)
    G = pkg.Grid(nx, ny, nz, 2, "bridge_corners")
    ref = G.apply_K(x, w)
    assert _rel(ref, oref) <= 1e-13
    y = torch.empty_like(x)
    for _ in range(2):
        y.fill_(float("nan"))
        pkg.apply_K_noalloc(nx, ny, nz, "bridge_corners", x, w, out=y)
        torch.cuda.synchronize()
        assert _rel(y, ref) <= 1e-13
        assert _rel(y, oref) <= 1e-13
    # another shape through the same array, then the first again
    w2_h, x2_h, w2, x2 = _case(16, 8, 8, 12)
    G2 = pkg.Grid(16, 8, 8, 3, "cantilever")
    y2 = pkg.apply_K_noalloc(16, 8, 8, "cantilever", x2, w2)
    torch.cuda.synchronize()
    assert _rel(y2, G2.apply_K(x2, w2)) <= 1e-13
    assert _rel(y2, fem.apply_K_elementwise(fem.Grid(16, 8, 8, "cantilever"), w2_h, fem.element_stiffness(),
                                            x2_h)) <= 1e-13
    pkg.apply_K_noalloc(nx, ny, nz, "bridge_corners", x, w, out=y)
    torch.cuda.synchronize()
    assert _rel(y, ref) <= 1e-13


def test_noalloc_call_leaves_device_memory_as_it_was(pkg):
    nx, ny, nz = 24, 12, 12
    _, _, w, x = _case(nx, ny, nz, 13)
    y = torch.empty_like(x)
    pkg.apply_K_noalloc(nx, ny, nz, "cantilever", x, w, out=y)   # the library's module is loaded by now
    torch.cuda.synchronize()
    before_torch = torch.cuda.memory_allocated()
    before_free = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        pkg.apply_K_noalloc(nx, ny, nz, "cantilever", x, w, out=y)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before_torch
    assert torch.cuda.mem_get_info()[0] == before_free


def test_noalloc_rejects_grids_beyond_the_static_array(pkg):
    """A 100 x 100 x 60 grid needs at least 96 bytes of plane-quad scratch per element (57.6 MB) against the 32 MiB
    array: rejected with PBM_EINVAL before any launch. The arrays passed are real buffers of the right length."""
    nx, ny, nz = 100, 100, 60
    m, n = nx * ny * nz, 3 * (nx + 1) * (ny + 1) * (nz + 1)
    w = torch.full((m,), 0.5, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    L = pkg.lib()
    rc = L.pbm_apply_K_noalloc(nx, ny, nz, 0, 1.0, 0.3, 1.0, C.c_void_p(w.data_ptr()), C.c_void_p(x.data_ptr()),
                               C.c_void_p(y.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == -1
    assert "too large" in L.pbm_last_error().decode()
    assert bool(torch.all(y == 7.0))
