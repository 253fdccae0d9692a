"""ctypes declarations of libbpmllg.so (include/bpm.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_uint8, c_uint32, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libbpmllg.so")

BPM_OK = 0
BPM_ERR_ARG, BPM_ERR_CUDA, BPM_ERR_OOM, BPM_ERR_TIMEOUT, BPM_ERR_NONFINITE, BPM_ERR_UNSTABLE, BPM_ERR_STATE = \
    -1, -2, -3, -4, -5, -6, -7
ERRORS = {-1: "BPM_ERR_ARG", -2: "BPM_ERR_CUDA", -3: "BPM_ERR_OOM", -4: "BPM_ERR_TIMEOUT",
          -5: "BPM_ERR_NONFINITE", -6: "BPM_ERR_UNSTABLE", -7: "BPM_ERR_STATE"}

TERM_EXCHANGE, TERM_ANISOTROPY, TERM_DEMAG, TERM_HEAD, TERM_UNIFORM, TERM_ALL = 1, 2, 4, 8, 16, 31
PREC_FP32, PREC_BF16X3, PREC_BF16, PREC_BF16X3_REF = 0, 1, 2, 3
ISLAND_NONFINITE = 1
OP_EXCHANGE_F32, OP_DEMAG_F64, OP_DEMAG_F32, OP_VOLUMES_F64, OP_NODAL_MS_F64, OP_NODAL_KU_F64 = range(6)
MESH_KEEP_F64 = 1


class bpm_region_mat(ctypes.Structure):
    _fields_ = [("Ms_A_per_m", c_double), ("Ku_J_per_m3", c_double), ("A_J_per_m", c_double)]


class bpm_island(ctypes.Structure):
    _fields_ = [("mesh_id", c_int32), ("Ms_scale", c_float), ("Ku_scale", c_float), ("u", c_float * 3),
                ("pos_nm", c_float * 2), ("Hext_T", c_float * 3)]


ISLAND_DTYPE = np.dtype([("mesh_id", "<i4"), ("Ms_scale", "<f4"), ("Ku_scale", "<f4"), ("u", "<f4", (3,)),
                         ("pos_nm", "<f4", (2,)), ("Hext_T", "<f4", (3,))])


class bpm_run_params(ctypes.Structure):
    _fields_ = [("dt_ps", c_double), ("substeps", c_int32), ("precision", c_int32), ("t0_ps", c_double),
                ("alpha", c_double), ("rise_ps", c_double), ("v_m_per_s", c_double), ("x0_nm", c_double),
                ("map_id", c_int32), ("term_mask", c_uint32), ("uniform_T", c_float * 3), ("pad_", c_float)]


class bpm_mesh_info(ctypes.Structure):
    _fields_ = [("n_nodes", c_int32), ("n_pad", c_int32), ("n_tets", c_int32), ("n_boundary", c_int32),
                ("nnz", c_int32), ("cg_iters_neumann", c_int32), ("cg_iters_dirichlet", c_int32),
                ("k_pad", c_int32), ("volume_nm3", c_double), ("exchange_lambda_max_T", c_double),
                ("field_bound_T", c_double), ("cg_residual_neumann", c_double),
                ("cg_residual_dirichlet", c_double)]


class bpm_mlp_cfg(ctypes.Structure):
    _fields_ = [("n_in", c_int32), ("width", c_int32), ("depth", c_int32), ("n_out", c_int32)]


class bpm_train_cfg(ctypes.Structure):
    _fields_ = [("epochs", c_int32), ("batch", c_int32), ("lr", c_float), ("weight_decay", c_float),
                ("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("pad_", c_int32)]


RASTER_AUTO, RASTER_M, RASTER_N = 0, 1, 2


class bpm_neb_params(ctypes.Structure):
    _fields_ = [("n_images", c_int32), ("max_iters", c_int32), ("climb_after", c_int32), ("precision", c_int32),
                ("map_id", c_int32), ("term_mask", ctypes.c_uint32), ("check_every", c_int32), ("pad_", c_int32),
                ("step", c_double), ("spring", c_double), ("force_tol", c_double), ("head_x_nm", c_double),
                ("uniform_T", c_double * 3)]


class bpm_pole_geometry(ctypes.Structure):
    _fields_ = [("pole_tip_width_nm", c_float), ("trailing_edge_angle_deg", c_float),
                ("side_edge_angle_deg", c_float), ("taper_angle_deg", c_float), ("abs_thickness_nm", c_float),
                ("yoke_edge_nm", c_float), ("Js_T", c_float), ("z_abs_nm", c_float), ("z_sul_nm", c_float),
                ("sul_image", c_int32), ("trailing_shield_gap_nm", c_float), ("shield_thickness_nm", c_float),
                ("shield_panel_nm", c_float), ("side_shield_gap_nm", c_float)]


class bpm_tuning(ctypes.Structure):
    _fields_ = [("gemm_tile_n", c_int32), ("stage_threads", c_int32), ("gemm_raster", c_int32), ("stage_islands", c_int32),
                ("gemm_k_block", c_int32), ("gemm_pair", c_int32), ("streams", c_int32),
                ("gemm_ms", c_double), ("stage_ms", c_double)]


# name -> (restype, argtypes); every function declared in include/bpm.h
PROTOTYPES = {
    "bpm_create": (c_int, [POINTER(c_void_p), c_int, c_void_p]),
    "bpm_destroy": (None, [c_void_p]),
    "bpm_context_stream": (c_int, [c_void_p, POINTER(c_void_p)]),
    "bpm_substeps_for_bound": (c_int, [c_double, c_double, c_double, POINTER(c_int32)]),
    "bpm_stable_substeps": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), POINTER(c_int32),
                                    POINTER(c_double)]),
    "bpm_last_error": (c_char_p, []),
    "bpm_version": (c_char_p, []),
    "bpm_mesh_upload": (c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_int32,
                                c_uint32, POINTER(c_int32)]),
    "bpm_mesh_info_get": (c_int, [c_void_p, c_int32, POINTER(bpm_mesh_info)]),
    "bpm_mesh_get_operator": (c_int, [c_void_p, c_int32, c_int32, c_void_p]),
    "bpm_head_field_solve": (c_int, [c_void_p, POINTER(bpm_pole_geometry), c_int32, c_int32, c_int32, c_float,
                                     c_void_p, c_void_p, c_int]),
    "bpm_mesh_release": (c_int, [c_void_p, c_int32]),
    "bpm_headmap_release": (c_int, [c_void_p, c_int32]),
    "bpm_headmap_upload": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p,
                                   POINTER(c_int32)]),
    "bpm_batch_create": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), POINTER(c_void_p)]),
    "bpm_batch_set_state": (c_int, [c_void_p, c_void_p, c_int32, c_double, c_int]),
    "bpm_batch_advance": (c_int, [c_void_p, c_int32]),
    "bpm_batch_read": (c_int, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "bpm_batch_field": (c_int, [c_void_p, c_double, c_uint32, c_void_p, c_int32, c_int]),
    "bpm_batch_kernel_times": (c_int, [c_void_p, c_int32, POINTER(c_double), POINTER(c_double),
                                       POINTER(c_double)]),
    "bpm_batch_autotune": (c_int, [c_void_p, c_int32, POINTER(bpm_tuning)]),
    "bpm_batch_set_tuning": (c_int, [c_void_p, POINTER(bpm_tuning)]),
    "bpm_debug_set_gemm_error": (c_int, [c_void_p, c_int32]),
    "bpm_debug_set_gemm_wait": (c_int, [c_void_p, c_double]),
    "bpm_batch_graph_kernels": (c_int, [c_void_p, POINTER(c_int32)]),
    "bpm_neb_run": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_neb_params), c_void_p, c_int32, c_void_p,
                            c_void_p, c_void_p, POINTER(c_int32), POINTER(c_double)]),
    "bpm_lhs_maximin": (c_int, [c_void_p, c_void_p, c_int32, c_int32, c_int32, POINTER(c_int32), c_void_p]),
    "bpm_gp_nll": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_double, c_void_p]),
    "bpm_gp_create": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_double, POINTER(c_int32),
                              c_void_p]),
    "bpm_gp_predict": (c_int, [c_void_p, c_int32, c_void_p, c_int64, c_double, c_void_p, c_void_p, c_void_p]),
    "bpm_gp_destroy": (c_int, [c_void_p, c_int32]),
    "bpm_batch_energy": (c_int, [c_void_p, c_void_p, c_void_p]),
    "bpm_batch_time": (c_int, [c_void_p, POINTER(c_double)]),
    "bpm_batch_destroy": (c_int, [c_void_p]),
    "bpm_run_batch": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), c_int32, c_void_p, c_int32,
                              c_void_p, c_void_p, c_void_p]),
    "bpm_run_batch_dev": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), c_int32, c_void_p, c_int32,
                                  c_void_p, c_void_p, c_void_p]),
    "bpm_run_plain": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), c_int32, c_void_p, c_int32,
                              c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    "bpm_run_plain_f64": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), c_int32, c_void_p, c_int32,
                                  c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    "bpm_surrogate_create": (c_int, [c_void_p, POINTER(bpm_mlp_cfg), c_void_p, POINTER(c_int32)]),
    "bpm_surrogate_param_count": (c_int, [c_void_p, c_int32, POINTER(c_int64)]),
    "bpm_surrogate_get_params": (c_int, [c_void_p, c_int32, c_void_p]),
    "bpm_surrogate_grad": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "bpm_surrogate_train": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_int64, POINTER(bpm_train_cfg),
                                    c_void_p]),
    "bpm_surrogate_infer": (c_int, [c_void_p, c_int32, c_void_p, c_int64, c_void_p, c_int]),
    "bpm_surrogate_screen": (c_int, [c_void_p, c_int32, c_void_p, c_int64, c_int32, c_void_p, c_int]),
    "bpm_surrogate_save": (c_int, [c_void_p, c_int32, c_char_p]),
    "bpm_surrogate_load": (c_int, [c_void_p, c_int32, c_char_p]),
    "bpm_surrogate_destroy": (c_int, [c_void_p, c_int32]),
    "bpm_llg_advance_noalloc": (c_int, [c_void_p, c_void_p, c_int32, POINTER(bpm_run_params), c_int32, c_void_p,
                                        c_int32, c_void_p]),
}

NOALLOC_SCRATCH_BYTES = 8 * 1024 * 1024

_lib = None


class BpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load the library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libbpmllg.so not built at {path}; run paper_1603_09493_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int):
    if code != BPM_OK:
        raise BpmError(code, load().bpm_last_error().decode())


def ptr(a) -> c_void_p:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return c_void_p(a.data_ptr())
    return a.ctypes.data_as(c_void_p)
