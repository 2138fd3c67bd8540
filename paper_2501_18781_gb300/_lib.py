"""ctypes declarations of the C ABI in include/mfgb.h (argument marshalling only)."""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmfgb.so")

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_ENOTCONV, MF_ETIMEOUT, MF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
MF_F64, MF_F32, MF_F16, MF_BF16, MF_DF64 = 0, 1, 2, 3, 4
MF_INNER_TENSOR_CORES = 16
MF_OP_HELMHOLTZ, MF_OP_HEAT, MF_OP_OSEEN, MF_OP_REINIT = 0, 1, 2, 3
MF_HEAVISIDE_TANH, MF_HEAVISIDE_SINE = 0, 1
MF_COEF_INKERNEL, MF_COEF_QPOINT = 0, 1
MF_FIELD_PHI, MF_FIELD_T_PREV, MF_FIELD_BETA, MF_FIELD_K_QPOINT = 0, 1, 2, 3
MF_FIELD_RHOCP_QPOINT, MF_FIELD_BETA_QPOINT = 4, 5
MF_SOLVER_CG, MF_SOLVER_GMRES, MF_SOLVER_DEFECT_CORRECTION = 0, 1, 2
MF_OSEEN_THREE_PHASE, MF_OSEEN_DARCY, MF_OSEEN_TRACE_CORRECTION = 1, 2, 4
MF_PREC_NONE, MF_PREC_JACOBI, MF_PREC_CHEBYSHEV, MF_PREC_BLOCK_JACOBI, MF_PREC_BLOCK_TRIANGULAR = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "MF_OK", -1: "MF_EINVAL", -2: "MF_ENOMEM", -3: "MF_ECUDA", -4: "MF_ENOTCONV",
                -5: "MF_ETIMEOUT", -6: "MF_EUNSUPPORTED"}


class OpParams(C.Structure):
    _fields_ = [("kind", C.c_int), ("heaviside", C.c_int), ("coef_mode", C.c_int), ("reserved", C.c_int),
                ("eps", C.c_double), ("mass_coef", C.c_double), ("a_liquid", C.c_double), ("a_gas", C.c_double),
                ("rhocp", C.c_double), ("dt", C.c_double), ("k0", C.c_double), ("t_boil", C.c_double),
                ("sigma", C.c_double), ("rho_l", C.c_double), ("rho_g", C.c_double), ("mu_l", C.c_double),
                ("mu_g", C.c_double), ("dtau", C.c_double), ("rho_s", C.c_double), ("mu_s", C.c_double),
                ("t_solidus", C.c_double), ("t_liquidus", C.c_double), ("darcy_c", C.c_double),
                ("darcy_b", C.c_double), ("oseen_flags", C.c_int), ("reserved2", C.c_int)]


class SolverParams(C.Structure):
    _fields_ = [("solver", C.c_int), ("precond", C.c_int), ("inner_dtype", C.c_int), ("restart", C.c_int),
                ("cheby_degree", C.c_int), ("maxit", C.c_int), ("inner_maxit", C.c_int), ("use_graph", C.c_int),
                ("tol", C.c_double), ("inner_tol", C.c_double), ("cheby_ratio", C.c_double),
                ("lanczos_steps", C.c_int), ("fp64_arith", C.c_int), ("schur_maxit", C.c_int),
                ("velocity_steps", C.c_int), ("schur_tol", C.c_double), ("inner_arith", C.c_int),
                ("reserved3", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_iterations", C.c_int), ("rel_residual", C.c_double),
                ("lambda_max", C.c_double), ("seconds", C.c_double), ("inner_steps", C.c_int),
                ("reserved", C.c_int)]


class Evaporation(C.Structure):
    _fields_ = [("mass_flux", C.c_int), ("p_ambient", C.c_double), ("latent_heat", C.c_double),
                ("molar_mass", C.c_double), ("t_boil", C.c_double), ("sticking", C.c_double),
                ("tanasawa_coef", C.c_double), ("gas_constant", C.c_double), ("rhocp_liquid", C.c_double),
                ("rhocp_gas", C.c_double)]


class Laser(C.Structure):
    _fields_ = [("power", C.c_double), ("radius", C.c_double), ("x0", C.c_double), ("y0", C.c_double),
                ("absorptivity", C.c_double)]


class MeltPoolParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("eps", C.c_double), ("rho_l", C.c_double), ("rho_g", C.c_double),
                ("mu_l", C.c_double), ("mu_g", C.c_double), ("rhocp_l", C.c_double), ("rhocp_g", C.c_double),
                ("k_l", C.c_double), ("k_g", C.c_double), ("oseen_flags", C.c_int), ("laser_on", C.c_int),
                ("rho_s", C.c_double), ("mu_s", C.c_double), ("t_solidus", C.c_double), ("t_liquidus", C.c_double),
                ("darcy_c", C.c_double), ("darcy_b", C.c_double), ("evaporation", Evaporation),
                ("alpha0", C.c_double), ("alpha1", C.c_double), ("t_alpha", C.c_double), ("alpha_res", C.c_double),
                ("gravity", C.c_double * 3), ("laser_power", C.c_double), ("laser_radius", C.c_double),
                ("laser_absorptivity", C.c_double), ("laser_focus", C.c_double * 3),
                ("laser_direction", C.c_double * 3), ("reinit_steps", C.c_int), ("maxit", C.c_int),
                ("dtau", C.c_double), ("tol", C.c_double), ("flow_tol", C.c_double),
                ("flow_velocity_steps", C.c_int), ("flow_schur_maxit", C.c_int), ("flow_schur_tol", C.c_double),
                ("reinit_mixed", C.c_int), ("reserved", C.c_int)]


class MeltPoolInfo(C.Structure):
    _fields_ = [("advection_iterations", C.c_int), ("reinit_iterations", C.c_int), ("heat_iterations", C.c_int),
                ("flow_iterations", C.c_int), ("advection_residual", C.c_double), ("reinit_residual", C.c_double),
                ("heat_residual", C.c_double), ("flow_residual", C.c_double), ("seconds", C.c_double * 5)]


class MeltPoolTrace(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("u_star", "T_star", "phi_star", "u_gamma", "b_advection",
                                          "phi_advected", "r_heat", "b_flow", "T_update")]


P = C.c_void_p
I64 = C.c_int64
DP = C.POINTER(C.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "mf_last_error": (C.c_char_p, []),
    "mf_context_create": (C.c_int, [C.c_int, P, C.POINTER(P)]),
    "mf_context_destroy": (None, [P]),
    "mf_context_set_stream": (C.c_int, [P, P]),
    "mf_mesh_uniform": (C.c_int, [P, C.POINTER(C.c_int), DP, DP, C.POINTER(P)]),
    "mf_mesh_octree": (C.c_int, [P, C.c_int, C.c_int, DP, DP, C.POINTER(C.c_int32), I64, C.POINTER(P)]),
    "mf_mesh_destroy": (None, [P]),
    "mf_dofmap_create": (C.c_int, [P, C.c_int, C.c_uint32, C.POINTER(P)]),
    "mf_dofmap_destroy": (None, [P]),
    "mf_dofmap_query": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
    "mf_dofmap_export": (C.c_int, [P, C.POINTER(C.c_int32), C.POINTER(I64), C.POINTER(C.c_int32), DP, DP,
                                   C.POINTER(C.c_uint8)]),
    "mf_operator_create": (C.c_int, [P, C.POINTER(OpParams), C.POINTER(P), C.c_int, C.POINTER(P)]),
    "mf_operator_destroy": (None, [P]),
    "mf_operator_size": (C.c_int, [P, C.POINTER(I64)]),
    "mf_operator_set_field": (C.c_int, [P, C.c_int, P, C.c_int, I64]),
    "mf_apply": (C.c_int, [P, P, P, C.c_int, I64, C.c_int]),
    "mf_apply_transpose": (C.c_int, [P, P, P, C.c_int, I64, C.c_int]),
    "mf_apply_packed16": (C.c_int, [P, P, P, C.c_int, I64, C.c_int]),
    "mf_apply_tc": (C.c_int, [P, P, P, C.c_int, I64]),
    "mf_oseen_coupling": (C.c_int, [P, C.c_int, P, P, C.c_int]),
    "mf_interface_sources": (C.c_int, [P, C.POINTER(Evaporation), P, P, P, P]),
    "mf_diagonal": (C.c_int, [P, P, C.c_int]),
    "mf_dot": (C.c_int, [P, P, P, I64, I64, C.c_int, C.c_int, P]),
    "mf_dot_noalloc": (C.c_int, [P, P, I64, I64, C.c_int, C.c_int, P, P]),
    "mf_solve": (C.c_int, [P, C.POINTER(SolverParams), P, P, C.c_int, C.POINTER(SolveInfo)]),
    "mf_laser_load": (C.c_int, [P, C.POINTER(Laser), P, P]),
    "mf_heat_step_gradient": (C.c_int, [P, C.POINTER(Laser), C.POINTER(SolverParams), P, P, C.c_double, C.c_double,
                                        DP, DP, P, P, P]),
    "mf_autotune": (C.c_int, [P, C.c_char_p]),
    "mf_operator_variant": (C.c_char_p, [P]),
    "mf_operator_set_variant": (C.c_int, [P, C.c_char_p, C.c_int]),
    "mf_context_launch_count": (I64, [P]),
    "mf_meltpool_create": (C.c_int, [P, C.POINTER(MeltPoolParams), P, P, P, P, C.POINTER(P)]),
    "mf_meltpool_destroy": (None, [P]),
    "mf_meltpool_advance": (C.c_int, [P, P, P, P, P, P, P, P, P, P, C.POINTER(MeltPoolTrace),
                                      C.POINTER(MeltPoolInfo)]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libmfgb.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2501_18781_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status):
    if status != MF_OK:
        raise MFError(status, load().mf_last_error().decode())
    return status
