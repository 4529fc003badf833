"""ctypes binding of libpbm.so (the C ABI of include/pbm.h).

Argument marshalling only: every computation runs in the library's CUDA kernels. Tensors passed in
must be contiguous CUDA tensors of the dtype each call documents; the current torch stream is passed
as the CUDA stream. There is no fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpbm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pbm.h")

PBM_OK, PBM_EINVAL, PBM_ENOMEM, PBM_ECUDA, PBM_EBREAKDOWN, PBM_ENOTCONV, PBM_ETIMEOUT, PBM_ELINESEARCH, \
    PBM_ENONFINITE, PBM_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
STATUS_NAMES = {0: "PBM_OK", -1: "PBM_EINVAL", -2: "PBM_ENOMEM", -3: "PBM_ECUDA", -4: "PBM_EBREAKDOWN",
                -5: "PBM_ENOTCONV", -6: "PBM_ETIMEOUT", -7: "PBM_ELINESEARCH", -8: "PBM_ENONFINITE",
                -9: "PBM_ESTATE"}
SUPPORTS = {"cantilever": 0, "bridge_corners": 1, "bridge_edges": 2, "free": 3}
PRECISIONS = {"fp64": 0, "mixed": 1}
SMOOTHERS = {"jacobi": 0, "chebyshev": 1, "gauss_seidel": 2}
OPS = {"K": 0, "S": 1}
EPILOGUES = {"apply": 0, "resid": 1, "jacobi": 2}
MAPS = {"fixed_dofs": 0, "elem_nodes": 1, "prolong": 2, "Ke": 3}


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("levels", C.c_int), ("support", C.c_int),
                ("precision", C.c_int), ("E", C.c_double), ("nu", C.c_double), ("h", C.c_double),
                ("pre_sweeps", C.c_int), ("post_sweeps", C.c_int), ("jacobi_theta", C.c_double),
                ("lanczos_steps", C.c_int), ("inner_rtol", C.c_double), ("smoother", C.c_int)]


class GridInfo(C.Structure):
    _fields_ = [("levels", C.c_int), ("nx", C.c_int * 16), ("ny", C.c_int * 16), ("nz", C.c_int * 16),
                ("n", C.c_int64 * 16), ("m", C.c_int64 * 16), ("n_free", C.c_int64), ("omega", C.c_double * 16),
                ("lambda_max", C.c_double * 16), ("device_bytes", C.c_int64), ("fine_chunk", C.c_int * 4),
                ("fp32_tile", (C.c_int * 5) * 2), ("coarse_plan", (C.c_int * 16) * 2)]


class State(C.Structure):
    _fields_ = [("u_dev", C.c_void_p), ("nu_lo_dev", C.c_void_p), ("nu_up_dev", C.c_void_p), ("rho_dev", C.c_void_p),
                ("mu_lo_dev", C.c_void_p), ("mu_up_dev", C.c_void_p), ("alpha", C.c_double), ("p", C.c_double),
                ("q_lo", C.c_double), ("q_up", C.c_double), ("V", C.c_double), ("rho_lo", C.c_double),
                ("rho_up", C.c_double)]


class IPState(C.Structure):
    _fields_ = [("u_dev", C.c_void_p), ("alpha", C.c_double), ("rho_dev", C.c_void_p), ("nu_lo_dev", C.c_void_p),
                ("nu_up_dev", C.c_void_p), ("V", C.c_double), ("rho_lo", C.c_double), ("rho_up", C.c_double),
                ("r", C.c_double), ("s", C.c_double)]


class DocParams(C.Structure):
    _fields_ = [("V", C.c_double), ("rho_lo", C.c_double), ("rho_up", C.c_double), ("q", C.c_double),
                ("eps_doc", C.c_double), ("tau_alpha", C.c_double), ("eps_mr", C.c_double), ("maxit", C.c_int),
                ("max_iter", C.c_int)]


class DocInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("minres", C.c_int), ("trials", C.c_int),
                ("alpha", C.c_double), ("change", C.c_double), ("compliance", C.c_double),
                ("minres_relres", C.c_double)]


class ProfileStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("total_ms", C.c_double), ("bytes", C.c_double), ("flops", C.c_double)]


class PbmParams(C.Structure):
    _fields_ = [("eps_pbm", C.c_double), ("beta", C.c_double), ("gamma", C.c_double), ("p_min", C.c_double),
                ("eps_nwt", C.c_double), ("eps_nwt_min", C.c_double), ("eps_mr", C.c_double),
                ("eps_mr_min", C.c_double), ("max_outer", C.c_int), ("max_newton", C.c_int),
                ("max_halvings", C.c_int)]


class PbmInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("outer", C.c_int), ("newton", C.c_int), ("minres", C.c_int),
                ("gap_ratio", C.c_double), ("compliance", C.c_double), ("volume", C.c_double),
                ("eps_mr", C.c_double), ("resolves", C.c_int), ("stalls", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("outer", C.c_int), ("relres", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


class NewtonInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("minres_iterations", C.c_int), ("halvings", C.c_int), ("kappa", C.c_double),
                ("res_pbm", C.c_double), ("slope", C.c_double), ("lagrangian_old", C.c_double),
                ("lagrangian_new", C.c_double), ("minres_relres", C.c_double), ("resolves", C.c_int),
                ("stalled", C.c_int), ("eps_mr", C.c_double)]


class NewtonParams(C.Structure):
    _fields_ = [("eps_mr", C.c_double), ("eps_mr_min", C.c_double), ("max_halvings", C.c_int), ("maxit", C.c_int)]


def header_symbols() -> list[str]:
    """Names of every function declared in include/pbm.h."""
    with open(HEADER) as fh:
        txt = fh.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(pbm_\w+)\s*\(", txt, flags=re.M)))


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libpbm.so is not built ({path}); run paper_1904_06556_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "pbm_default_desc": (i, [C.POINTER(GridDesc), i, i, i, i, i]),
        "pbm_create_grid": (i, [C.POINTER(GridDesc), C.POINTER(vp)]),
        "pbm_destroy_grid": (i, [vp]),
        "pbm_last_error": (C.c_char_p, []),
        "pbm_grid_info_get": (i, [vp, C.POINTER(GridInfo)]),
        "pbm_get_maps": (i, [vp, i, i, vp]),
        "pbm_set_density": (i, [vp, vp, vp]),
        "pbm_apply_K": (i, [vp, vp, vp, vp, i, vp]),
        "pbm_apply_K_f32": (i, [vp, vp, vp, vp, vp]),
        "pbm_apply_fine_f32": (i, [vp, i, i, vp, vp, vp, C.POINTER(C.c_double), vp]),
        "pbm_apply_level_f32": (i, [vp, i, i, i, vp, vp, vp, C.POINTER(C.c_double), vp]),
        "pbm_get_diag": (i, [vp, i, vp, vp]),
        "pbm_fp32_plan_count": (i, []),
        "pbm_fp32_tc_plan": (i, []),
        "pbm_ip_set_state": (i, [vp, C.POINTER(IPState), vp]),
        "pbm_default_doc_params": (i, [C.POINTER(DocParams)]),
        "pbm_doc_step": (i, [vp, vp, vp, vp, C.POINTER(DocParams), C.POINTER(DocInfo), vp]),
        "pbm_doc_solve": (i, [vp, vp, vp, vp, C.POINTER(DocParams), C.POINTER(DocInfo), vp]),
        "pbm_ip_apply_S": (i, [vp, vp, vp, vp]),
        "pbm_ip_reduced_rhs": (i, [vp, vp, vp, vp]),
        "pbm_ip_solve": (i, [vp, vp, vp, d, i, C.POINTER(SolveInfo), vp]),
        "pbm_ip_recover": (i, [vp, vp, vp, vp, vp, vp]),
        "pbm_set_fp32_plan": (i, [vp, i, i]),
        "pbm_fp32_coarse_plan_count": (i, []),
        "pbm_set_fp32_coarse_plan": (i, [vp, i, i, i]),
        "pbm_set_state": (i, [vp, C.POINTER(State), vp]),
        "pbm_apply_S": (i, [vp, vp, vp, vp]),
        "pbm_reduced_rhs": (i, [vp, vp, vp, C.POINTER(C.c_double), vp]),
        "pbm_vcycle": (i, [vp, i, vp, vp, vp]),
        "pbm_minres_solve": (i, [vp, i, vp, vp, d, i, C.POINTER(SolveInfo), vp]),
        "pbm_newton_step": (i, [vp, C.POINTER(State), vp, d, C.POINTER(NewtonInfo), vp]),
        "pbm_default_newton_params": (i, [C.POINTER(NewtonParams)]),
        "pbm_newton_step_ex": (i, [vp, C.POINTER(State), vp, C.POINTER(NewtonParams), C.POINTER(NewtonInfo), vp]),
        "pbm_compliance_grad": (i, [vp, vp, vp, vp, C.POINTER(C.c_double), vp]),
        "pbm_kernel_launches": (C.c_int64, []),
        "pbm_batch_create": (i, [C.POINTER(vp), i, i, C.POINTER(vp)]),
        "pbm_batch_destroy": (i, [vp]),
        "pbm_batch_minres_solve": (i, [vp, C.POINTER(vp), C.POINTER(vp), d, i, C.POINTER(SolveInfo), vp]),
        "pbm_default_pbm_params": (i, [C.POINTER(PbmParams)]),
        "pbm_solve": (i, [vp, C.POINTER(State), vp, C.POINTER(PbmParams), C.POINTER(PbmInfo), vp]),
        "pbm_apply_K_noalloc": (i, [i, i, i, i, d, d, d, vp, vp, vp, vp]),
        "pbm_profile": (i, [vp, i]),
        "pbm_profile_read": (i, [vp, i, C.POINTER(ProfileStats)]),
    }
    for name, (res, args) in sig.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
    return lib


class PbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
