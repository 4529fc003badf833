"""pbm_apply_K_noalloc: K(w) x for callers that cannot allocate device memory.

Such callers (code running during CUDA graph capture, loops that must not allocate after start-up, hosts whose own
allocator owns all device memory) cannot create a grid handle, because pbm_create_grid allocates. The no-allocation
entry point keeps its scratch in a fixed device array inside the library. This file checks that its result equals the
handle-based pbm_apply_K on two calls in a row (the array keeps the previous call's contents), that a different grid
shape in between does not disturb it, and that a grid too large for the array is rejected. It sorts last so that a run
stopping at the first failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
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
    w = torch.as_tensor(rng.uniform(1e-3, 1.0, m), dtype=torch.float64, device="cuda")
    x = torch.as_tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
    return w, x


def test_noalloc_apply_equals_handle_apply_on_two_calls(pkg):
    nx, ny, nz = 34, 10, 6
    w, x = _case(nx, ny, nz, 11)
    G = pkg.Grid(nx, ny, nz, 2, "bridge_corners")
    ref = G.apply_K(x, w)
    y = torch.empty_like(x)
    for _ in range(2):
        y.fill_(float("nan"))
        pkg.apply_K_noalloc(nx, ny, nz, "bridge_corners", x, w, out=y)
        torch.cuda.synchronize()
        assert _rel(y, ref) <= 1e-13
    # another shape through the same array, then the first again
    w2, x2 = _case(16, 8, 8, 12)
    G2 = pkg.Grid(16, 8, 8, 3, "cantilever")
    y2 = pkg.apply_K_noalloc(16, 8, 8, "cantilever", x2, w2)
    torch.cuda.synchronize()
    assert _rel(y2, G2.apply_K(x2, w2)) <= 1e-13
    pkg.apply_K_noalloc(nx, ny, nz, "bridge_corners", x, w, out=y)
    torch.cuda.synchronize()
    assert _rel(y, ref) <= 1e-13


def test_noalloc_rejects_grids_beyond_the_static_array(pkg):
    L = pkg.lib()
    dummy = C.c_void_p(1)   # never dereferenced: the size check comes first
    rc = L.pbm_apply_K_noalloc(256, 128, 128, 0, 1.0, 0.3, 1.0, dummy, dummy, dummy, None)
    assert rc == -1
    assert "too large" in L.pbm_last_error().decode()
