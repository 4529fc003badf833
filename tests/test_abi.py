"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every function include/pbm.h declares,
and rejects invalid descriptions with PBM_EINVAL before touching a device (no compute call is made here)."""
import ctypes as C

import pytest

from paper_1904_06556_gb300 import _lib, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _lib.header_symbols()
    for need in ("pbm_create_grid", "pbm_set_density", "pbm_apply_K", "pbm_vcycle", "pbm_minres_solve",
                 "pbm_newton_step", "pbm_compliance_grad", "pbm_destroy_grid", "pbm_set_state", "pbm_apply_S"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    for name in _lib.header_symbols():
        assert hasattr(lib, name), name


def test_default_desc(lib):
    d = _lib.GridDesc()
    assert lib.pbm_default_desc(C.byref(d), 16, 8, 8, 3, 0) == 0
    assert (d.nx, d.ny, d.nz, d.levels, d.precision) == (16, 8, 8, 3, 0)
    assert d.E == 1.0 and d.nu == 0.3 and d.pre_sweeps == 2 and d.post_sweeps == 2
    assert d.jacobi_theta == 1.2 and d.lanczos_steps == 10
    assert d.smoother == _lib.SMOOTHERS["jacobi"]


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 15, "divisible"), ("levels", 0, "levels"), ("levels", 1, "at least 2"), ("support", 9, "support"),
    ("precision", 7, "precision"), ("nu", 0.5, "material"), ("E", -1.0, "material"), ("jacobi_theta", 2.5, "theta"),
    ("lanczos_steps", 1, "lanczos"), ("pre_sweeps", -1, "sweeps"), ("smoother", 3, "smoother"),
])
def test_invalid_descriptions_rejected(lib, field, value, msg):
    d = _lib.GridDesc()
    lib.pbm_default_desc(C.byref(d), 16, 8, 8, 3, 0)
    setattr(d, field, value)
    h = C.c_void_p()
    assert lib.pbm_create_grid(C.byref(d), C.byref(h)) == _lib.PBM_EINVAL
    assert msg in lib.pbm_last_error().decode()
    assert not h.value


def test_chebyshev_steps_limit(lib):
    """A Chebyshev pass takes at most 9 steps (the coefficient table holds 8 after the first)."""
    d = _lib.GridDesc()
    lib.pbm_default_desc(C.byref(d), 16, 8, 8, 3, 0)
    d.smoother = _lib.SMOOTHERS["chebyshev"]
    d.post_sweeps = 10
    h = C.c_void_p()
    assert lib.pbm_create_grid(C.byref(d), C.byref(h)) == _lib.PBM_EINVAL
    assert "Chebyshev" in lib.pbm_last_error().decode()
    assert not h.value


def test_coarsest_too_large_rejected(lib):
    d = _lib.GridDesc()
    lib.pbm_default_desc(C.byref(d), 64, 32, 32, 2, 0)
    h = C.c_void_p()
    assert lib.pbm_create_grid(C.byref(d), C.byref(h)) == _lib.PBM_EINVAL
    assert "coarsest" in lib.pbm_last_error().decode()


def test_null_arguments(lib):
    assert lib.pbm_create_grid(None, None) == _lib.PBM_EINVAL
    assert lib.pbm_destroy_grid(None) == 0


def test_newton_params_defaults_and_rejection(lib):
    p = _lib.NewtonParams()
    assert lib.pbm_default_newton_params(C.byref(p)) == 0
    assert (p.eps_mr, p.eps_mr_min, p.max_halvings, p.maxit) == (1e-4, 1e-9, 30, 10000)
    info = _lib.NewtonInfo()
    assert lib.pbm_newton_step_ex(None, None, None, C.byref(p), C.byref(info), None) == _lib.PBM_EINVAL
    q = _lib.PbmParams()
    assert lib.pbm_default_pbm_params(C.byref(q)) == 0
    assert q.max_halvings == 30 and q.eps_mr_min == 1e-9 and q.max_newton == 100
