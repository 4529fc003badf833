"""GB300-native reduced-Newton MG-MINRES solver for the PBM method on 3D variable-thickness-sheet problems.

`Grid` wraps one handle of the C library (include/pbm.h). Vectors are torch CUDA tensors:
displacements (n = 3 (nx+1)(ny+1)(nz+1), float64), element arrays (m = nx ny nz, float64), and the
reduced-system vectors (n + 1, float64, alpha last). The library runs every step in its own kernels;
this module only passes pointers, sizes and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import PbmError, SolveInfo, NewtonInfo  # noqa: F401

__all__ = ["Grid", "Batch", "PbmError", "lib", "kernel_launches", "apply_K_noalloc"]

_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


def kernel_launches() -> int:
    """Number of CUDA kernels the library has launched in this process."""
    return int(lib().pbm_kernel_launches())


def apply_K_noalloc(nx: int, ny: int, nz: int, support: str, x: torch.Tensor, w: torch.Tensor,
                    out: torch.Tensor | None = None, E: float = 1.0, nu: float = 0.3, h: float = 1.0) -> torch.Tensor:
    """y = K(w) x like Grid.apply_K, for callers that cannot allocate device memory (pbm_apply_K_noalloc): no grid
    handle, and the library allocates nothing. Pass `out` to avoid the allocation of the result tensor too. x, w and
    out must be on one CUDA device; the call runs there, on that device's current stream."""
    L = lib()
    n, m = 3 * (nx + 1) * (ny + 1) * (nz + 1), nx * ny * nz
    y = torch.empty_like(x) if out is None else out
    for name, t in (("w", w), ("out", y)):
        if t.device != x.device:
            raise ValueError(f"{name} is on {t.device}, x on {x.device}: all three must be on one device")
    with torch.cuda.device(x.device):
        rc = L.pbm_apply_K_noalloc(nx, ny, nz, _lib.SUPPORTS[support], float(E), float(nu), float(h),
                                   _ptr(w, n=m, name="w"), _ptr(x, n=n, name="x"), _ptr(y, n=n, name="y"), _stream())
    if rc != 0:
        raise PbmError(rc, L.pbm_last_error().decode())
    return y


def fp32_plan_count() -> int:
    """Number of tile plans of the single-pass FP32 fine operator (pbm_fp32_plan_count)."""
    return int(lib().pbm_fp32_plan_count())


def fp32_tc_plan() -> int:
    """The plan that runs the element contraction on the tensor cores (pbm_fp32_tc_plan)."""
    return int(lib().pbm_fp32_tc_plan())


def fp32_coarse_plan_count() -> int:
    """Number of tile plans of the single-pass FP32 coarse operator (pbm_fp32_coarse_plan_count); the
    two-pass forms are plans -1 (rows split over eight threads) and -2 (one thread per element)."""
    return int(lib().pbm_fp32_coarse_plan_count())


def _ptr(t: torch.Tensor | None, dtype=torch.float64, n: int | None = None, name: str = "tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} entries, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Grid:
    """A structured grid with its multigrid hierarchy (see pbm_create_grid)."""

    def __init__(self, nx: int, ny: int, nz: int, levels: int, support: str = "cantilever",
                 precision: str = "fp64", E: float = 1.0, nu: float = 0.3, h: float = 1.0, pre_sweeps: int = 2,
                 post_sweeps: int = 2, jacobi_theta: float = 1.2, lanczos_steps: int = 10,
                 inner_rtol: float = 1e-4, smoother: str = "jacobi"):
        self._L = lib()
        d = _lib.GridDesc()
        self._check(self._L.pbm_default_desc(C.byref(d), nx, ny, nz, levels, _lib.SUPPORTS[support]))
        d.precision = _lib.PRECISIONS[precision]
        d.E, d.nu, d.h = E, nu, h
        d.pre_sweeps, d.post_sweeps = pre_sweeps, post_sweeps
        d.jacobi_theta, d.lanczos_steps, d.inner_rtol = jacobi_theta, lanczos_steps, inner_rtol
        d.smoother = _lib.SMOOTHERS[smoother]
        self.desc = d
        h_ = C.c_void_p()
        self._h = None
        self._check(self._L.pbm_create_grid(C.byref(d), C.byref(h_)))
        self._h = h_
        self.nx, self.ny, self.nz, self.levels = nx, ny, nz, levels
        self.nnode = (nx + 1) * (ny + 1) * (nz + 1)
        self.n = 3 * self.nnode
        self.m = nx * ny * nz
        self._level_n = [3 * ((nx >> k) + 1) * ((ny >> k) + 1) * ((nz >> k) + 1) for k in range(levels)]
        self._keep = []

    # --------------------------------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != 0:
            raise PbmError(rc, self._L.pbm_last_error().decode())

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._L.pbm_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --------------------------------------------------------------------------------------------
    def info(self) -> dict:
        gi = _lib.GridInfo()
        self._check(self._L.pbm_grid_info_get(self._h, C.byref(gi)))
        L = gi.levels
        return dict(levels=L, dims=[(gi.nx[k], gi.ny[k], gi.nz[k]) for k in range(L)], n=list(gi.n[:L]),
                    m=list(gi.m[:L]), n_free=gi.n_free, omega=list(gi.omega[:L]), lambda_max=list(gi.lambda_max[:L]),
                    device_bytes=gi.device_bytes, fine_chunk=list(gi.fine_chunk),
                    fp32_tile=[list(gi.fp32_tile[0]), list(gi.fp32_tile[1])],
                    coarse_plan=[list(gi.coarse_plan[0][1:max(1, L - 1)]), list(gi.coarse_plan[1][1:max(1, L - 1)])])

    def maps(self, level: int, which: str):
        import numpy as np
        nx, ny, nz = self.nx >> level, self.ny >> level, self.nz >> level
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        if which == "fixed_dofs":
            out = np.zeros(3 * nn, dtype=np.uint8)
        elif which == "elem_nodes":
            out = np.zeros((nx * ny * nz, 8), dtype=np.int32)
        elif which == "prolong":
            nnf = (2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1)
            buf = np.zeros(nnf * 8 * 4 + nnf * 8 * 8, dtype=np.uint8)
            self._check(self._L.pbm_get_maps(self._h, level, _lib.MAPS[which], buf.ctypes.data_as(C.c_void_p)))
            ids = buf[: nnf * 32].view(np.int32).reshape(nnf, 8)
            wts = buf[nnf * 32:].view(np.float64).reshape(nnf, 8)
            return ids, wts
        elif which == "Ke":
            out = np.zeros((24, 24), dtype=np.float64)
        else:
            raise ValueError(which)
        self._check(self._L.pbm_get_maps(self._h, level, _lib.MAPS[which], out.ctypes.data_as(C.c_void_p)))
        return out

    # --------------------------------------------------------------------------------------------
    def set_density(self, rho: torch.Tensor):
        self._check(self._L.pbm_set_density(self._h, _ptr(rho, n=self.m, name="rho"), _stream()))

    def apply_K(self, x: torch.Tensor, w: torch.Tensor | None = None, out: torch.Tensor | None = None,
                level: int = 0):
        """y = K(w) x on the fine level (w None: the set density), or, for level >= 1, the FP64 Galerkin operator
        of that level of the K(rho) hierarchy (pbm_apply_K)."""
        y = torch.empty_like(x) if out is None else out
        nl = self._level_n[level] if 0 <= level < self.levels else None
        self._check(self._L.pbm_apply_K(self._h, _ptr(w, n=self.m, name="w"), _ptr(x, n=nl, name="x"),
                                        _ptr(y, n=nl, name="y"), int(level), _stream()))
        return y

    def apply_K_f32(self, x: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None):
        y = torch.empty_like(x) if out is None else out
        f = torch.float32
        self._check(self._L.pbm_apply_K_f32(self._h, _ptr(w, f, self.m, "w"), _ptr(x, f, self.n, "x"),
                                            _ptr(y, f, self.n, "y"), _stream()))
        return y

    def apply_fine_f32(self, op: str, epilogue: str, x: torch.Tensor, b: torch.Tensor | None = None,
                       out: torch.Tensor | None = None, dot: bool = False):
        """One FP32 fine-level application of K or S with a fused epilogue (pbm_apply_fine_f32); returns
        (y, dot) where dot is the epilogue's reduced dot product (or None)."""
        f = torch.float32
        n = self.n + (1 if op == "S" else 0)
        y = out if out is not None else torch.empty(n, dtype=f, device=x.device)
        d = C.c_double(0.0)
        self._check(self._L.pbm_apply_fine_f32(self._h, _lib.OPS[op], _lib.EPILOGUES[epilogue], _ptr(x, f, n, "x"),
                                               _ptr(b, f, n, "b") if b is not None else None, _ptr(y, f, n, "y"),
                                               C.byref(d) if dot else None, _stream()))
        return y, (d.value if dot else None)

    def apply_level_f32(self, level: int, op: str, epilogue: str, x: torch.Tensor, b: torch.Tensor | None = None,
                        out: torch.Tensor | None = None, dot: bool = False):
        """pbm_apply_level_f32: one FP32 application of level `level`'s operator with a fused epilogue."""
        f = torch.float32
        # a level out of range is left to the library to reject (PBM_EINVAL)
        n = self._level_n[level] + (1 if op == "S" else 0) if 0 <= level < len(self._level_n) else None
        y = out if out is not None else torch.empty(n if n is not None else x.numel(), dtype=f, device=x.device)
        d = C.c_double(0.0)
        self._check(self._L.pbm_apply_level_f32(self._h, level, _lib.OPS[op], _lib.EPILOGUES[epilogue],
                                                _ptr(x, f, n, "x"), _ptr(b, f, n, "b") if b is not None else None,
                                                _ptr(y, f, n, "y"), C.byref(d) if dot else None, _stream()))
        return y, (d.value if dot else None)

    # ---- damped optimality criteria (pbm_doc_*) ----
    def _doc_params(self, V, rho_lo, rho_up, **kw):
        p = _lib.DocParams()
        self._check(self._L.pbm_default_doc_params(C.byref(p)))
        p.V, p.rho_lo, p.rho_up = float(V), float(rho_lo), float(rho_up)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown DOC parameter {k}")
            setattr(p, k, v)
        return p

    def doc_step(self, rho: torch.Tensor, f: torch.Tensor, u: torch.Tensor, V: float, rho_lo: float, rho_up: float,
                 **params) -> dict:
        """One iteration of Algorithm DOC (pbm_doc_step): rho (m) and u (n) FP64 CUDA tensors, updated in place."""
        p = self._doc_params(V, rho_lo, rho_up, **params)
        inf = _lib.DocInfo()
        self._check(self._L.pbm_doc_step(self._h, _ptr(rho, n=self.m, name="rho"), _ptr(f, n=self.n, name="f"),
                                         _ptr(u, n=self.n, name="u"), C.byref(p), C.byref(inf), _stream()))
        return {k: getattr(inf, k) for k, _ in _lib.DocInfo._fields_}

    def doc_solve(self, rho: torch.Tensor, f: torch.Tensor, u: torch.Tensor, V: float, rho_lo: float, rho_up: float,
                  check: bool = True, **params) -> dict:
        """Algorithm DOC until ||rho+ - rho||_inf <= eps_doc (pbm_doc_solve); rho and u updated in place."""
        p = self._doc_params(V, rho_lo, rho_up, **params)
        inf = _lib.DocInfo()
        rc = self._L.pbm_doc_solve(self._h, _ptr(rho, n=self.m, name="rho"), _ptr(f, n=self.n, name="f"),
                                   _ptr(u, n=self.n, name="u"), C.byref(p), C.byref(inf), _stream())
        if check:
            self._check(rc)
        out = {k: getattr(inf, k) for k, _ in _lib.DocInfo._fields_}
        out["rc"] = rc
        return out

    # ---- interior-point Newton system (pbm_ip_*) ----
    def ip_set_state(self, st: dict):
        """st: u (n), rho, nu_lo, nu_up (m) FP64 CUDA tensors; alpha, V, rho_lo, rho_up, r, s floats."""
        s = _lib.IPState(_ptr(st["u"], n=self.n, name="u").value, float(st["alpha"]),
                         _ptr(st["rho"], n=self.m, name="rho").value, _ptr(st["nu_lo"], n=self.m, name="nu_lo").value,
                         _ptr(st["nu_up"], n=self.m, name="nu_up").value, float(st["V"]), float(st["rho_lo"]),
                         float(st["rho_up"]), float(st["r"]), float(st["s"]))
        self._check(self._L.pbm_ip_set_state(self._h, C.byref(s), _stream()))

    def ip_apply_S(self, x: torch.Tensor, out: torch.Tensor | None = None):
        y = out if out is not None else torch.empty(self.n + 1, dtype=torch.float64, device=x.device)
        self._check(self._L.pbm_ip_apply_S(self._h, _ptr(x, n=self.n + 1, name="x"), _ptr(y, n=self.n + 1, name="y"),
                                           _stream()))
        return y

    def ip_reduced_rhs(self, f: torch.Tensor):
        rhs = torch.empty(self.n + 1, dtype=torch.float64, device=f.device)
        self._check(self._L.pbm_ip_reduced_rhs(self._h, _ptr(f, n=self.n, name="f"), _ptr(rhs, n=self.n + 1),
                                               _stream()))
        return rhs

    def ip_solve(self, rhs: torch.Tensor, rtol: float = 1e-8, maxit: int = 500, x0: torch.Tensor | None = None,
                 check: bool = True):
        dz = x0.clone() if x0 is not None else torch.zeros(self.n + 1, dtype=torch.float64, device=rhs.device)
        inf = _lib.SolveInfo()
        rc = self._L.pbm_ip_solve(self._h, _ptr(rhs, n=self.n + 1, name="rhs"), _ptr(dz, n=self.n + 1),
                                  float(rtol), int(maxit), C.byref(inf), _stream())
        if check:
            self._check(rc)
        return dz, {k: getattr(inf, k) for k, _ in _lib.SolveInfo._fields_}

    def ip_recover(self, dz: torch.Tensor):
        """(drho, dnu_lo, dnu_up) from the reduced solution dz (pbm_ip_recover)."""
        out = [torch.empty(self.m, dtype=torch.float64, device=dz.device) for _ in range(3)]
        self._check(self._L.pbm_ip_recover(self._h, _ptr(dz, n=self.n + 1, name="dz"), *[_ptr(t) for t in out],
                                           _stream()))
        return tuple(out)

    def set_fp32_plan(self, op: str, plan: int):
        """Overrides the autotuned tile plan of the FP32 fine operator for op (pbm_set_fp32_plan)."""
        self._check(self._L.pbm_set_fp32_plan(self._h, _lib.OPS[op], int(plan)))

    def set_fp32_coarse_plan(self, op: str, level: int, plan: int):
        """Overrides the autotuned form of the FP32 operator of coarse level `level` (pbm_set_fp32_coarse_plan)."""
        self._check(self._L.pbm_set_fp32_coarse_plan(self._h, _lib.OPS[op], int(level), int(plan)))

    def diag(self, level: int = 0) -> torch.Tensor:
        """Jacobi diagonal (n_level + 1 FP64 entries) of a level of the current hierarchy (pbm_get_diag)."""
        nl = self._level_n[level] + 1
        out = torch.empty(nl, dtype=torch.float64, device="cuda")
        self._check(self._L.pbm_get_diag(self._h, level, _ptr(out, n=nl, name="diag"), _stream()))
        return out

    def _state(self, st: dict) -> _lib.State:
        s = _lib.State()
        for key in ("u", "nu_lo", "nu_up", "rho", "mu_lo", "mu_up"):
            t = st[key]
            setattr(s, key + "_dev", _ptr(t, n=self.n if key == "u" else self.m, name=key))
        for key in ("alpha", "p", "q_lo", "q_up", "V", "rho_lo", "rho_up"):
            setattr(s, key, float(st[key]))
        return s

    def set_state(self, st: dict):
        """st: u (n), nu_lo, nu_up, rho, mu_lo, mu_up (m) CUDA float64 tensors; alpha, p, q_lo, q_up, V, rho_lo,
        rho_up floats."""
        s = self._state(st)
        self._check(self._L.pbm_set_state(self._h, C.byref(s), _stream()))

    def apply_S(self, x: torch.Tensor, out: torch.Tensor | None = None):
        y = torch.empty_like(x) if out is None else out
        self._check(self._L.pbm_apply_S(self._h, _ptr(x, n=self.n + 1, name="x"), _ptr(y, n=self.n + 1, name="y"),
                                        _stream()))
        return y

    def reduced_rhs(self, f: torch.Tensor, norms: bool = False):
        rhs = torch.empty(self.n + 1, dtype=torch.float64, device=f.device)
        nrm = (C.c_double * 3)()
        self._check(self._L.pbm_reduced_rhs(self._h, _ptr(f, n=self.n, name="f"), _ptr(rhs, n=self.n + 1),
                                            nrm if norms else None, _stream()))
        return (rhs, tuple(nrm)) if norms else rhs

    def vcycle(self, op: str, b: torch.Tensor):
        x = torch.empty_like(b)
        n = self.n + (1 if op == "S" else 0)
        self._check(self._L.pbm_vcycle(self._h, _lib.OPS[op], _ptr(b, n=n, name="b"), _ptr(x, n=n), _stream()))
        return x

    def minres_solve(self, op: str, b: torch.Tensor, rtol: float = 1e-8, maxit: int = 500,
                     x0: torch.Tensor | None = None, check: bool = True):
        n = self.n + (1 if op == "S" else 0)
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        inf = _lib.SolveInfo()
        rc = self._L.pbm_minres_solve(self._h, _lib.OPS[op], _ptr(b, n=n, name="b"), _ptr(x, n=n), float(rtol),
                                      int(maxit), C.byref(inf), _stream())
        info = {k: getattr(inf, k) for k, _ in _lib.SolveInfo._fields_}
        if check:
            self._check(rc)
        info["rc"] = rc
        return x, info

    def newton_step(self, st: dict, f: torch.Tensor, eps_mr: float, check: bool = True, **params):
        """One Newton step of Algorithm 2; updates st['u'], st['nu_lo'], st['nu_up'] in place and st['alpha'].
        Keyword arguments (eps_mr_min, max_halvings, maxit) override the defaults of pbm_newton_step_ex."""
        s = self._state(st)
        inf = _lib.NewtonInfo()
        prm = _lib.NewtonParams()
        self._check(self._L.pbm_default_newton_params(C.byref(prm)))
        prm.eps_mr = float(eps_mr)
        for k, v in params.items():
            if not hasattr(prm, k):
                raise TypeError(f"unknown Newton parameter {k}")
            setattr(prm, k, v)
        rc = self._L.pbm_newton_step_ex(self._h, C.byref(s), _ptr(f, n=self.n, name="f"), C.byref(prm), C.byref(inf),
                                        _stream())
        info = {k: getattr(inf, k) for k, _ in _lib.NewtonInfo._fields_}
        info["rc"] = rc
        if check:
            self._check(rc)
        st["alpha"] = s.alpha
        return info

    def profile(self, on: bool = True):
        """Start (or stop) timing every fine-level operator launch with CUDA events on its stream."""
        self._check(self._L.pbm_profile(self._h, 1 if on else 0))

    def profile_read(self, op: str = "S") -> dict:
        """Launches, total milliseconds, algorithmic bytes and operations of the fine-level kernel of operator `op`
        ("K" or "S") since its last read (synchronises)."""
        ps = _lib.ProfileStats()
        self._check(self._L.pbm_profile_read(self._h, _lib.OPS[op], C.byref(ps)))
        return {k: getattr(ps, k) for k, _ in _lib.ProfileStats._fields_}

    def pbm_solve(self, st: dict, f: torch.Tensor, check: bool = True, **params):
        """Algorithm 1 from the state `st` (updated in place; st['rho'] holds the densities on exit). Keyword
        arguments override the paper's parameters (eps_pbm, beta, gamma, p_min, eps_nwt, eps_nwt_min, eps_mr,
        eps_mr_min, max_outer, max_newton, max_halvings)."""
        prm = _lib.PbmParams()
        self._check(self._L.pbm_default_pbm_params(C.byref(prm)))
        for k, v in params.items():
            if not hasattr(prm, k):
                raise TypeError(f"unknown PBM parameter {k}")
            setattr(prm, k, v)
        s = self._state(st)
        inf = _lib.PbmInfo()
        rc = self._L.pbm_solve(self._h, C.byref(s), _ptr(f, n=self.n, name="f"), C.byref(prm), C.byref(inf),
                               _stream())
        info = {k: getattr(inf, k) for k, _ in _lib.PbmInfo._fields_}
        info["rc"] = rc
        if check:
            self._check(rc)
        for k in ("alpha", "p", "q_lo", "q_up"):
            st[k] = getattr(s, k)
        return info

    @staticmethod
    def initial_state(n: int, m: int, V: float, rho_lo: float, rho_up: float, device="cuda") -> dict:
        """The paper's initial point of Algorithm 1: u = 0, alpha = 1, nu = e, rho = V/m, mu = e, p = q = 1."""
        f64 = dict(dtype=torch.float64, device=device)
        return dict(u=torch.zeros(n, **f64), nu_lo=torch.ones(m, **f64), nu_up=torch.ones(m, **f64),
                    rho=torch.full((m,), V / m, **f64), mu_lo=torch.ones(m, **f64), mu_up=torch.ones(m, **f64),
                    alpha=1.0, p=1.0, q_lo=1.0, q_up=1.0, V=V, rho_lo=rho_lo, rho_up=rho_up)

    def compliance_grad(self, u: torch.Tensor, f: torch.Tensor | None = None):
        c = torch.empty(self.m, dtype=torch.float64, device=u.device)
        fTu = C.c_double(0.0)
        self._check(self._L.pbm_compliance_grad(self._h, _ptr(u, n=self.n, name="u"), _ptr(c, n=self.m),
                                                _ptr(f, n=self.n, name="f"), C.byref(fTu) if f is not None else None,
                                                _stream()))
        return (c, fTu.value) if f is not None else c


class Batch:
    """Several grids solved together, one launch per stage for all of them (see pbm_batch_create)."""

    def __init__(self, grids: list, op: str = "S"):
        self._L = lib()
        self.grids = list(grids)
        self.op = op
        arr = (C.c_void_p * len(self.grids))(*[g._h.value for g in self.grids])
        h = C.c_void_p()
        rc = self._L.pbm_batch_create(arr, len(self.grids), _lib.OPS[op], C.byref(h))
        if rc != 0:
            raise PbmError(rc, self._L.pbm_last_error().decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._L.pbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def minres_solve(self, bs: list, rtol: float = 1e-8, maxit: int = 1000, x0s: list | None = None,
                     check: bool = True):
        """Solves every system; returns (list of solutions, list of info dicts)."""
        ns = len(self.grids)
        xs = [torch.zeros_like(b) if x0s is None else x0s[i].clone() for i, b in enumerate(bs)]
        for g, b, x in zip(self.grids, bs, xs):
            n = g.n + (1 if self.op == "S" else 0)
            _ptr(b, n=n, name="b"), _ptr(x, n=n, name="x")
        barr = (C.c_void_p * ns)(*[b.data_ptr() for b in bs])
        xarr = (C.c_void_p * ns)(*[x.data_ptr() for x in xs])
        infos = (_lib.SolveInfo * ns)()
        rc = self._L.pbm_batch_minres_solve(self._h, barr, xarr, float(rtol), int(maxit), infos, _stream())
        out = [{k: getattr(inf, k) for k, _ in _lib.SolveInfo._fields_} for inf in infos]
        if check and rc != 0:
            raise PbmError(rc, self._L.pbm_last_error().decode())
        return xs, out
