"""ctypes declarations of the C ABI in include/lh.h (argument marshalling only)."""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblh.so")

LH_OK, LH_EINVAL, LH_ECUDA, LH_ENOMEM, LH_ETANGLED, LH_ENOCONV, LH_ENONFINITE = range(7)
LH_FP64, LH_FP32, LH_FP32_LIN, LH_TF32, LH_BF16 = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "LH_OK", 1: "LH_EINVAL", 2: "LH_ECUDA", 3: "LH_ENOMEM", 4: "LH_ETANGLED",
                5: "LH_ENOCONV", 6: "LH_ENONFINITE"}

# every symbol include/lh.h declares
SYMBOLS = ["lh_mesh_desc_init", "lh_mesh_create", "lh_mesh_destroy", "lh_sizes", "lh_set_stream",
           "lh_initial_nodes", "lh_residual", "lh_jvp", "lh_jtvp", "lh_mass_apply", "lh_mass_solve",
           "lh_dt_estimate", "lh_energies", "lh_tg_velocity_error", "lh_newton_opts_init", "lh_newton_step", "lh_advance_opts_init", "lh_advance", "lh_advance_replay",
           "lh_explicit_opts_init", "lh_force", "lh_explicit_step", "lh_explicit_advance", "lh_stage_solve", "lh_sdirk_step", "lh_sdirk_tableau", "lh_last_error",
           "lh_probe_fma", "lh_profile_enable", "lh_profile_read", "lh_launch_count", "lh_qp_flops", "lh_record_len", "lh_dd_check", "lh_linearize", "lh_jvv_diagonal", "lh_qp_tangent_check", "lh_qp_adjoint_check", "lh_tc_status", "lh_tc_set_wait_polls", "lh_halo_len", "lh_halo_pack", "lh_halo_add", "lh_residual_noalloc", "lh_precond",
           "lh_mlp_create", "lh_mlp_destroy", "lh_mlp_num_params", "lh_mlp_params", "lh_mlp_forward",
           "lh_mlp_grad", "lh_mlp_train_step", "lh_mlp_last_error", "lh_mlp_features", "lh_mlp_apply_prediction"]
PROF_KINDS = ["residual", "jvp_fp64", "jvp_fp32", "jtvp", "mass_h1", "jvp_tc"]


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("order", C.c_int), ("quad_1d", C.c_int),
                ("rho0", C.POINTER(C.c_double)), ("gamma", C.POINTER(C.c_double)),
                ("rho0_value", C.c_double), ("gamma_value", C.c_double), ("bc_mask", C.c_uint),
                ("visc", C.c_int), ("q1", C.c_double), ("q2", C.c_double), ("psi0", C.c_double),
                ("eps_e", C.c_double), ("h0", C.c_double), ("h_coarse", C.c_double),
                ("tg_source", C.c_int), ("stream", C.c_void_p)]


class NewtonOpts(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_atol", C.c_double), ("gmres_rtol", C.c_double),
                ("newton_maxit", C.c_int), ("gmres_maxit", C.c_int), ("restart", C.c_int),
                ("max_halvings", C.c_int), ("jvp_prec", C.c_int), ("precond", C.c_int),
                ("forcing", C.c_int), ("eta_max", C.c_double), ("scaled_norm", C.c_int),
                ("cheb_degree", C.c_int), ("cheb_ratio", C.c_double), ("arnoldi", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("gmres_its_total", C.c_int), ("backtracks", C.c_int),
                ("residual_evals", C.c_int), ("jvp_evals", C.c_int), ("reorth", C.c_int), ("r0", C.c_double),
                ("rfinal", C.c_double), ("min_detj", C.c_double), ("newton_its_max", C.c_int)]


class AdvanceOpts(C.Structure):
    _fields_ = [("scheme", C.c_int), ("fs_cfl", C.c_double), ("dt0", C.c_double), ("grow", C.c_double),
                ("shrink", C.c_double), ("grow_its", C.c_int), ("reject_its", C.c_int), ("enlarge", C.c_int),
                ("max_steps", C.c_int), ("max_attempts", C.c_int), ("dt_min", C.c_double)]


class AdvanceAttempt(C.Structure):
    _fields_ = [("dt", C.c_double), ("h", C.c_double), ("newton_its", C.c_int), ("accepted", C.c_int)]


class AdvanceStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("rejected", C.c_int), ("attempts", C.c_int), ("t", C.c_double),
                ("dt_next", C.c_double), ("newton_its", C.c_longlong), ("gmres_its", C.c_longlong)]


class ExplicitOpts(C.Structure):
    _fields_ = [("scheme", C.c_int), ("visc_model", C.c_int), ("q1_exp", C.c_double), ("q2_exp", C.c_double),
                ("l0_exp", C.c_double), ("vorticity", C.c_int), ("cfl", C.c_double), ("mass_rtol", C.c_double),
                ("mass_maxit", C.c_int)]


class ExplicitStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("rejected", C.c_int), ("t", C.c_double), ("dt_last", C.c_double),
                ("force_evals", C.c_longlong), ("mass_iters", C.c_longlong)]


def load(path=LIB_PATH):
    """Load liblh.so and declare the signatures.  Raises OSError if it is missing."""
    lib = C.CDLL(path)
    vp, dp, ip, llp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
    i, d = C.c_int, C.c_double
    sig = {
        "lh_mesh_desc_init": (None, [C.POINTER(MeshDesc)]),
        "lh_mesh_create": (i, [C.POINTER(MeshDesc), C.POINTER(vp)]),
        "lh_mesh_destroy": (i, [vp]),
        "lh_sizes": (i, [vp, llp]),
        "lh_set_stream": (i, [vp, vp]),
        "lh_initial_nodes": (i, [vp, vp]),
        "lh_residual": (i, [vp, vp, vp, d, vp, dp]),
        "lh_jvp": (i, [vp, vp, vp, d, vp, vp, i]),
        "lh_jtvp": (i, [vp, vp, vp, d, vp, vp, i]),
        "lh_mass_apply": (i, [vp, i, vp, vp]),
        "lh_mass_solve": (i, [vp, i, vp, vp, d, i, ip]),
        "lh_dt_estimate": (i, [vp, vp, dp]),
        "lh_energies": (i, [vp, vp, dp, dp]),
        "lh_jvv_diagonal": (i, [vp, vp, vp, d, vp]),
        "lh_tg_velocity_error": (i, [vp, vp, dp]),
        "lh_newton_opts_init": (None, [C.POINTER(NewtonOpts)]),
        "lh_newton_step": (i, [vp, vp, vp, d, C.POINTER(NewtonOpts), C.POINTER(StepStats)]),
        "lh_stage_solve": (i, [vp, vp, vp, d, C.POINTER(NewtonOpts), C.POINTER(StepStats)]),
        "lh_advance_opts_init": (None, [C.POINTER(AdvanceOpts)]),
        "lh_explicit_opts_init": (None, [C.POINTER(ExplicitOpts)]),
        "lh_force": (i, [vp, vp, vp, C.POINTER(ExplicitOpts), vp, vp, dp]),
        "lh_explicit_step": (i, [vp, vp, d, C.POINTER(ExplicitOpts), C.POINTER(ExplicitStats)]),
        "lh_explicit_advance": (i, [vp, vp, d, i, C.POINTER(ExplicitOpts), C.POINTER(ExplicitStats)]),
        "lh_advance": (i, [vp, vp, vp, d, C.POINTER(NewtonOpts), C.POINTER(AdvanceOpts), C.POINTER(AdvanceStats),
                           C.POINTER(AdvanceAttempt), i]),
        "lh_advance_replay": (i, [ip, i, d, d, C.POINTER(AdvanceOpts), C.POINTER(AdvanceStats),
                                  C.POINTER(AdvanceAttempt), i]),
        "lh_sdirk_step": (i, [vp, i, vp, vp, d, C.POINTER(NewtonOpts), C.POINTER(StepStats)]),
        "lh_sdirk_tableau": (i, [i, ip, dp, dp]),
        "lh_last_error": (C.c_char_p, [vp]),
        "lh_probe_fma": (i, [i, dp]),
        "lh_profile_enable": (i, [vp, i]),
        "lh_profile_read": (i, [vp, dp, llp]),
        "lh_launch_count": (C.c_longlong, []),
        "lh_qp_flops": (i, [i, i, i, llp]),
        "lh_record_len": (i, [i, ip]),
        "lh_dd_check": (i, [i, i, C.c_uint, dp]),
        "lh_linearize": (i, [vp, vp, vp, d]),
        "lh_tc_status": (i, [vp]),
        "lh_tc_set_wait_polls": (C.c_uint, [C.c_uint]),
        "lh_qp_tangent_check": (i, [i, i, i, C.c_uint, dp, dp]),
        "lh_qp_adjoint_check": (i, [i, i, i, C.c_uint, dp]),
        "lh_halo_len": (i, [vp, i, C.POINTER(C.c_longlong)]),
        "lh_halo_pack": (i, [vp, i, vp, vp, i]),
        "lh_halo_add": (i, [vp, i, vp, vp, i]),
        "lh_residual_noalloc": (i, [C.POINTER(MeshDesc), vp, vp, vp, vp, d, vp]),
        "lh_precond": (i, [vp, i, d, vp, vp]),
        "lh_mlp_create": (i, [i, i, i, i, vp, vp, C.POINTER(vp)]),
        "lh_mlp_destroy": (i, [vp]),
        "lh_mlp_num_params": (C.c_longlong, [vp]),
        "lh_mlp_params": (i, [vp, vp]),
        "lh_mlp_forward": (i, [vp, vp, i, vp]),
        "lh_mlp_grad": (i, [vp, vp, vp, i, vp, dp]),
        "lh_mlp_train_step": (i, [vp, vp, vp, i, C.c_float, dp]),
        "lh_mlp_last_error": (C.c_char_p, [vp]),
        "lh_mlp_features": (i, [vp, vp, vp, d, vp, vp]),
        "lh_mlp_apply_prediction": (i, [vp, vp, d, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib
