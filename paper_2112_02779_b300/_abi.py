"""ctypes mirrors of the structs in include/rimg.h (layout checked by a test
that compiles the header with gcc)."""
import ctypes

RIMG_MAX_LEVELS = 8
RIMG_FLAG_DEGENERATE = 1
RIMG_STATIC_SCRATCH_BYTES = 1 << 20

STATUS_NAMES = {0: "RIMG_OK", -1: "RIMG_ERR_INVALID_ARG", -2: "RIMG_ERR_LUT", -3: "RIMG_ERR_SIZE",
                -4: "RIMG_ERR_WORKSPACE", -5: "RIMG_ERR_CUDA", -6: "RIMG_ERR_MISMATCH"}


class rimg_level(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("n_bins", ctypes.c_int), ("tie_up", ctypes.c_int),
                ("bins_exact", ctypes.c_int), ("has_theta", ctypes.c_int), ("s_lo", ctypes.c_float), ("s_hi", ctypes.c_float), ("bin_scale", ctypes.c_float),
                ("w_over_2pi", ctypes.c_float),
                ("off_rows", ctypes.c_size_t), ("off_cols", ctypes.c_size_t), ("off_thu", ctypes.c_size_t),
                ("off_rank", ctypes.c_size_t), ("off_bnd", ctypes.c_size_t), ("off_bins", ctypes.c_size_t)]


class rimg_sensor(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("levels", ctypes.c_int), ("r0", ctypes.c_float),
                ("d_tables", ctypes.c_void_p), ("table_bytes", ctypes.c_size_t),
                ("level", rimg_level * RIMG_MAX_LEVELS)]


class rimg_params(ctypes.Structure):
    _fields_ = [("huber_delta", ctypes.c_float), ("max_corr_dist", ctypes.c_float),
                ("normal_rel_jump", ctypes.c_float), ("proj_iters", ctypes.c_int), ("kahan", ctypes.c_int),
                ("streams", ctypes.c_int), ("normal_method", ctypes.c_int)]


class rimg_group(ctypes.Structure):
    _fields_ = [("src", ctypes.POINTER(rimg_sensor)), ("dst", ctypes.POINTER(rimg_sensor)),
                ("n_pairs", ctypes.c_int), ("levels", ctypes.c_int), ("iters", ctypes.POINTER(ctypes.c_int)),
                ("params", ctypes.POINTER(rimg_params)), ("src_range", ctypes.c_void_p),
                ("dst_range", ctypes.c_void_p), ("T_init", ctypes.c_void_p), ("T_out", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


# Every function include/rimg.h declares (checked against the header and the
# library's exports by the CPU test-suite).
HEADER_FUNCTIONS = [
    "rimg_default_params", "rimg_status_string", "rimg_last_error",
    "rimg_sensor_table_bytes", "rimg_sensor_build", "rimg_unproject", "rimg_pyramid", "rimg_normals",
    "rimg_icp_workspace_bytes", "rimg_icp_step", "rimg_icp_step_static", "rimg_gn_update",
    "rimg_register_workspace_bytes", "rimg_register", "rimg_register_last_sums",
    "rimg_register_groups_workspace_bytes", "rimg_register_groups", "rimg_autotune", "rimg_autotune_register", "rimg_autotune_clear", "rimg_autotune_set",
    "rimg_register_host_workspace_bytes", "rimg_register_host", "rimg_register_host_async",
    "rimg_gemm_bf16", "rimg_profile_begin", "rimg_profile_end", "rimg_sdf_integrate", "rimg_points_to_range",
    "rimg_cnn_param_count", "rimg_cnn_state_bytes", "rimg_cnn_workspace_bytes", "rimg_cnn_init", "rimg_cnn_load",
    "rimg_propose", "rimg_cnn_grad", "rimg_cnn_train_step", "rimg_center_init",
]

# Learned pose proposal constants (rimg.h)
RIMG_CNN_IN_H, RIMG_CNN_IN_W = 8, 128
RIMG_CNN_RANGE_SCALE = 0.03125
RIMG_CNN_OMEGA_SCALE = 0.25
RIMG_CNN_T_SCALE = 3.0
RIMG_CNN_MAX_BATCH = 65536


class rimg_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("voxel", ctypes.c_float),
                ("origin", ctypes.c_float * 3)]


class rimg_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]
