"""ctypes binding of libmg_gb300.so (the C ABI of include/mg.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  Loading fails loudly when the shared object is missing; there is
no fallback path.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmg_gb300.so")

MG_OK = 0
ERRORS = {-1: "MG_ERR_ARG", -2: "MG_ERR_BALANCE", -3: "MG_ERR_CUDA", -4: "MG_ERR_NOT_CONVERGED",
          -5: "MG_ERR_NAN", -6: "MG_ERR_TIMEOUT", -7: "MG_ERR_INCOMPATIBLE_RHS", -8: "MG_ERR_STATE",
          -9: "MG_ERR_UNSUPPORTED"}

# every entry point declared in include/mg.h
EXPORTS = ["mg_tree_create", "mg_tree_refine", "mg_tree_build_on", "mg_tree_built_on", "mg_tree_block_table",
           "mg_tree_num_levels", "mg_tree_level_info",
           "mg_tree_num_leaf_cells", "mg_tree_leaf_blocks", "mg_set_bc_plane", "mg_tree_finalize",
           "mg_tree_adapt", "mg_tree_build_times",
           "mg_set_rhs", "mg_set_eps", "mg_set_phi", "mg_get_phi", "mg_vcycle", "mg_fmg",
           "mg_residual_norm", "mg_solve", "mg_adjoint", "mg_adjoint_solve", "mg_apply_transpose",
           "mg_clean_adjoint", "mg_set_schedule", "mg_get_schedule", "mg_tune_schedule", "mg_tree_destroy",
           "mg_last_error",
           "mg_launch_count", "mg_set_wait_limit", "mg_time_sweeps", "mg_residual_norm_noalloc", "mg_sweep_variant",
           "mg_divergence", "mg_divergence_order", "mg_project", "mg_clean", "mg_set_sweep_variant", "mg_set_tail",
           "mg_batch_create", "mg_batch_leaf_offsets", "mg_batch_set_rhs", "mg_batch_set_eps",
           "mg_batch_set_phi", "mg_batch_get_phi", "mg_batch_vcycle", "mg_batch_fmg", "mg_batch_residual_norms",
           "mg_batch_solve", "mg_batch_launch_count", "mg_batch_num_segments", "mg_batch_segment_info",
           "mg_batch_time_sweeps", "mg_batch_set_tail", "mg_batch_coarse_info", "mg_batch_tune_schedule", "mg_batch_destroy"]


class MGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "MG_ERR"), code, msg))
        self.code = code


class mg_bc(C.Structure):
    _fields_ = [("type", C.c_int * 6), ("value", C.c_double * 6)]


class mg_params(C.Structure):
    _fields_ = [("n_down", C.c_int), ("n_up", C.c_int), ("precision", C.c_int), ("inner_cycles", C.c_int),
                ("smoother", C.c_int), ("omega", C.c_double), ("coarse_mode", C.c_int), ("coarse_max_it", C.c_int),
                ("coarse_abs_tol", C.c_double), ("coarse_rel_tol", C.c_double)]


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmg_gb300.so is not built: run __graft_entry__.build() "
                          "(or python -m paper_1901_11370_gb300.build)")
    L = C.CDLL(LIB_PATH)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    L.mg_tree_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(mg_bc), ip, dp, dp, C.c_int, C.c_double,
                                 C.POINTER(vp)]
    L.mg_tree_refine.argtypes = [vp, C.c_int, vp]
    L.mg_tree_num_levels.argtypes = [vp, ip]
    L.mg_tree_level_info.argtypes = [vp, C.c_int, vp, dp]
    L.mg_tree_num_leaf_cells.argtypes = [vp, C.POINTER(C.c_int64)]
    L.mg_tree_leaf_blocks.argtypes = [vp, vp]
    L.mg_tree_build_on.argtypes = [vp, C.c_int]
    L.mg_tree_built_on.argtypes = [vp, ip]
    L.mg_tree_block_table.argtypes = [vp, vp, vp]
    L.mg_set_bc_plane.argtypes = [vp, C.c_int, C.c_int, vp]
    L.mg_tree_finalize.argtypes = [vp, vp]
    L.mg_tree_adapt.argtypes = [vp, C.c_int, vp, C.c_int, vp, C.POINTER(vp)]
    L.mg_tree_build_times.argtypes = [vp, dp]
    for n in ("mg_set_rhs", "mg_set_eps", "mg_set_phi", "mg_get_phi"):
        getattr(L, n).argtypes = [vp, vp]
    L.mg_vcycle.argtypes = [vp, C.c_int, C.POINTER(mg_params)]
    L.mg_fmg.argtypes = [vp, C.POINTER(mg_params)]
    L.mg_residual_norm.argtypes = [vp, dp, dp, vp]
    L.mg_solve.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.POINTER(mg_params), ip, dp]
    L.mg_adjoint.argtypes = [vp, vp, vp, vp, C.POINTER(mg_params), C.c_int]
    L.mg_adjoint_solve.argtypes = [vp, vp, vp, vp, C.POINTER(mg_params), C.c_double, C.c_int, ip, dp]
    L.mg_apply_transpose.argtypes = [vp, vp, vp]
    L.mg_clean_adjoint.argtypes = [vp, vp, vp, C.POINTER(mg_params), C.c_double, C.c_int, ip, dp]
    L.mg_set_schedule.argtypes = [vp, C.c_int, vp, vp]
    L.mg_get_schedule.argtypes = [vp, C.c_int, vp, vp]
    L.mg_tune_schedule.argtypes = [vp, C.c_double, C.c_int, C.c_int, ip, dp]
    L.mg_tree_destroy.argtypes = [vp]
    L.mg_launch_count.argtypes = [vp, C.POINTER(C.c_int64)]
    L.mg_set_wait_limit.argtypes = [vp, C.c_int64]
    L.mg_time_sweeps.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp]
    L.mg_residual_norm_noalloc.argtypes = [vp, dp, dp]
    L.mg_sweep_variant.argtypes = [vp, C.c_int, C.c_int, ip]
    L.mg_set_sweep_variant.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.mg_set_tail.argtypes = [vp, C.c_int64]
    L.mg_batch_set_tail.argtypes = [vp, C.c_int64]
    L.mg_divergence.argtypes = [vp, vp, vp]
    L.mg_divergence_order.argtypes = [vp, vp, vp, C.c_int]
    L.mg_clean.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, C.c_int, C.POINTER(mg_params), ip, dp]
    L.mg_project.argtypes = [vp, vp, vp]
    L.mg_batch_create.argtypes = [C.c_int, vp, vp, C.POINTER(vp)]
    L.mg_batch_leaf_offsets.argtypes = [vp, vp]
    for n in ("mg_batch_set_rhs", "mg_batch_set_eps", "mg_batch_set_phi", "mg_batch_get_phi"):
        getattr(L, n).argtypes = [vp, vp]
    L.mg_batch_vcycle.argtypes = [vp, C.c_int, C.POINTER(mg_params)]
    L.mg_batch_fmg.argtypes = [vp, C.POINTER(mg_params)]
    L.mg_batch_residual_norms.argtypes = [vp, vp, vp]
    L.mg_batch_solve.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.POINTER(mg_params), ip, vp]
    L.mg_batch_launch_count.argtypes = [vp, C.POINTER(C.c_int64)]
    L.mg_batch_num_segments.argtypes = [vp, ip, ip]
    L.mg_batch_segment_info.argtypes = [vp, C.c_int, vp]
    L.mg_batch_time_sweeps.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp]
    L.mg_batch_coarse_info.argtypes = [vp, vp]
    L.mg_batch_tune_schedule.argtypes = [vp, C.c_double, C.c_int, C.c_int, ip, dp]
    L.mg_batch_destroy.argtypes = [vp]
    L.mg_last_error.restype = C.c_char_p
    _lib = L
    return L


def check(rc, allow=()):
    if rc != MG_OK and rc not in allow:
        raise MGError(rc, load().mg_last_error().decode(errors="replace"))
    return rc
