"""ctypes declarations of the C ABI in include/fe_hotpath.h (marshalling only)."""
import ctypes as ct

FE_OK = 0
STATUS = {0: "FE_OK", 1: "FE_ERR_ARG", 2: "FE_ERR_CUDA", 3: "FE_ERR_OOM",
          4: "FE_ERR_PATTERN_CHANGED", 5: "FE_ERR_NOT_CONVERGED", 6: "FE_ERR_BREAKDOWN",
          7: "FE_ERR_INVERTED", 8: "FE_ERR_TIMEOUT", 9: "FE_ERR_STATE"}
FE_TET4, FE_HEX8 = 0, 1
FE_SVK, FE_NEOHOOKE, FE_MOONEY_RIVLIN, FE_COROTATIONAL = 0, 1, 2, 3
FE_FP64, FE_MIXED = 0, 1


class FeMesh(ct.Structure):
    _fields_ = [("elem_type", ct.c_int32), ("n_nodes", ct.c_int64), ("n_elems", ct.c_int64),
                ("rest_xyz", ct.POINTER(ct.c_double)), ("conn", ct.POINTER(ct.c_int32)),
                ("n_fixed", ct.c_int64), ("fixed_nodes", ct.POINTER(ct.c_int32))]


class FeMaterial(ct.Structure):
    _fields_ = [("model", ct.c_int32), ("rho", ct.c_double),
                ("params", ct.POINTER(ct.c_double)), ("per_element", ct.c_int32)]


class FeOptions(ct.Structure):
    _fields_ = [("precision", ct.c_int32), ("tol", ct.c_double), ("max_iters", ct.c_int32),
                ("refactor_every", ct.c_int32), ("device_ptrs", ct.c_int32),
                ("stream", ct.c_void_p), ("keep_checkpoints", ct.c_int32),
                ("nd_leaf_nodes", ct.c_int32), ("inner_tol", ct.c_double),
                ("factor_timeout_s", ct.c_double), ("use_graph", ct.c_int32),
                ("profile_stages", ct.c_int32), ("newton_iters", ct.c_int32),
                ("newton_tol", ct.c_double), ("factor_tf32", ct.c_int32),
                ("precond_fp16", ct.c_int32), ("contact_sweeps", ct.c_int32), ("contact_tol", ct.c_double),
                ("factor_lag", ct.c_int32), ("dep_wait_s", ct.c_double), ("element_fp64", ct.c_int32),
                ("warm_start", ct.c_int32), ("spmv_variant", ct.c_int32), ("apply_sm_share", ct.c_double),
                ("update_bf16", ct.c_int32)]


class FeStepInfo(ct.Structure):
    _fields_ = [("iters", ct.c_int32), ("refinements", ct.c_int32), ("factor_age", ct.c_int32),
                ("rel_residual", ct.c_double), ("newton", ct.c_int32), ("newton_correction", ct.c_double)]


class FeInfo(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("nnz", ct.c_int64), ("ntrip", ct.c_int64), ("n_free", ct.c_int64),
                ("n_fronts", ct.c_int64), ("n_levels", ct.c_int64), ("y_nnz", ct.c_int64),
                ("factor_flops", ct.c_double), ("device_bytes", ct.c_int64), ("noalloc_bytes", ct.c_int64),
                ("ntrip_kept", ct.c_int64), ("n_blocks", ct.c_int64)]


STAGES = ["element", "assembly", "factor", "apply", "spmv", "vector", "residual", "integrate",
          "factor_update", "pcg_graph", "contact", "factor_update_bf16"]

P = ct.POINTER
CTX = ct.c_void_p
DP = P(ct.c_double)
I32P = P(ct.c_int32)

# name -> (restype, argtypes); the full exported surface of fe_hotpath.h
SIGNATURES = {
    "fe_options_default": (ct.c_int, [P(FeOptions)]),
    "fe_create": (ct.c_int, [P(FeMesh), P(FeMaterial), ct.c_double, ct.c_double, ct.c_double,
                             P(FeOptions), P(CTX)]),
    "fe_create_batch": (ct.c_int, [ct.c_int32, P(FeMesh), P(FeMaterial), ct.c_double, ct.c_double,
                                   ct.c_double, P(FeOptions), P(CTX)]),
    "fe_get_batch_layout": (ct.c_int, [CTX, P(ct.c_int32), P(I32P), P(P(ct.c_int64)), P(P(ct.c_int64))]),
    "fe_get_batch_stats": (ct.c_int, [CTX, I32P, DP]),
    "fe_build_pattern": (ct.c_int, [CTX]),
    "fe_get_pattern": (ct.c_int, [CTX, P(ct.c_int64), P(ct.c_int64), P(I32P), P(I32P),
                                  P(ct.c_int64), P(I32P)]),
    "fe_get_inverse_map": (ct.c_int, [CTX, P(P(ct.c_int64)), P(I32P)]),
    "fe_get_mass": (ct.c_int, [CTX, P(DP)]),
    "fe_get_ordering": (ct.c_int, [CTX, P(ct.c_int64), P(I32P), P(ct.c_int64), P(I32P), P(I32P),
                                   P(I32P), P(I32P), P(I32P)]),
    "fe_get_front_rows": (ct.c_int, [CTX, ct.c_int64, P(ct.c_int64), P(I32P)]),
    "fe_set_state": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p]),
    "fe_get_state": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p]),
    "fe_element_eval": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fe_assemble": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fe_factor_now": (ct.c_int, [CTX]),
    "fe_apply_preconditioner": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p]),
    "fe_set_contacts": (ct.c_int, [CTX, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fe_get_contact_forces": (ct.c_int, [CTX, ct.c_void_p]),
    "fe_apply_preconditioner_noalloc": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fe_step": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p, ct.c_void_p, P(FeStepInfo)]),
    "fe_get_info": (ct.c_int, [CTX, P(FeInfo)]),
    "fe_get_stage_times": (ct.c_int, [CTX, DP, P(ct.c_int64), P(ct.c_int64)]),
    "fe_reset_stage_times": (ct.c_int, [CTX]),
    "fe_get_update_flops": (ct.c_int, [CTX, DP]),
    "fe_get_update_bf16_flops": (ct.c_int, [CTX, DP]),
    "fe_get_update_bf16_tiles": (ct.c_int, [CTX, P(ct.c_int64)]),
    "fe_set_params": (ct.c_int, [CTX, ct.c_void_p]),
    "fe_adjoint": (ct.c_int, [CTX, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "fe_clear_checkpoints": (ct.c_int, [CTX]),
    "fe_num_checkpoints": (ct.c_int, [CTX, P(ct.c_int64)]),
    "fe_debug_hold_front": (ct.c_int, [CTX, ct.c_int64, ct.c_int32]),
    "fe_last_error": (ct.c_char_p, [CTX]),
    "fe_destroy": (None, [CTX]),
    "fe_trip_create": (ct.c_int, [ct.c_int64, P(ct.c_void_p)]),
    "fe_trip_assemble": (ct.c_int, [CTX, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int32,
                                    ct.c_void_p, P(ct.c_int32)]),
    "fe_trip_pattern": (ct.c_int, [CTX, P(ct.c_int64), P(I32P), P(I32P), P(I32P)]),
    "fe_trip_values": (ct.c_int, [CTX, ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "fe_trip_device_csr": (ct.c_int, [CTX, P(ct.c_void_p), P(ct.c_void_p), P(ct.c_void_p)]),
    "fe_trip_last_error": (ct.c_char_p, [CTX]),
    "fe_trip_destroy": (None, [CTX]),
}


def bind(lib):
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
