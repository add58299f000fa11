"""GB300-native periodic corrector solver (arXiv 2007.06524 hot path).

Python binding of libsq (include/sq.h): argument marshalling only. Every step
of the solve runs in the library's CUDA kernels; PyTorch provides device
memory and streams. There is no CPU fallback: a missing or unloadable libsq.so
raises.
"""
from .sq import (  # noqa: F401
    SQ_EBADGUESS, SQ_ECUDA, SQ_EINVAL, SQ_ENOCONV, SQ_ENOMEM, SQ_ETIMEOUT, SQ_FP32_REFINE, SQ_FP64, SQ_OK,
    Batch, Coeffs, Net, sq_net_create, sq_net_grads, sq_net_params, sq_net_predict, sq_net_set_params,
    sq_net_train_step, Precond, SqError, Workspace, sq_batch_create, sq_pcg_solve_batched, lib_path, load_library, sq_apply_operator, sq_apply_operator_f32,
    sq_apply_precond, sq_apply_precond_f32, sq_build_coeffs, sq_coeffs_cells, sq_coeffs_from_host,
    sq_coeffs_regenerate, sq_coeffs_set_subcell, sq_coeffs_set_levels, sq_build_coeffs_levels, sq_coeffs_regenerate_levels, sq_coeffs_from_host_levels, sq_coeffs_shape, sq_ensemble_ahom, sq_coeffs_upload, sq_homogenized_matrix, sq_homogenized_matrix_noalloc, sq_profile_class_name,
    sq_profile_enable, sq_profile_read, sq_profile_work, sq_pcg_solve, sq_precond_factors, sq_precond_setup, sq_precond_setup_canonical, sq_precond_setup_tucker, sq_precond_info, sq_rhs, sq_set_option, sq_set_tiles, sq_strerror, SQ_OPT_STRIDED_TWO_STAGE,
    SQ_OPT_STENCIL_ROWS, SQ_OPT_INNER_TOL_EXP, SQ_OPT_WAIT_POLLS, SQ_OPT_MULTIPLIER_TABLE, SQ_OPT_CONV_TC,
    SQ_OPT_PCG_GRAPHS,
    sq_workspace_create, sq_launch_count, sq_probe_fma, sq_probe_copy,
    Coeffs2D, Precond2D, Workspace2D, sq2d_build_coeffs, sq2d_coeffs_from_host, sq2d_coeffs_set_subcell,
    sq2d_coeffs_cells, sq2d_precond_setup, sq2d_precond_factors, sq2d_workspace_create, sq2d_pcg_solve,
    sq2d_homogenized_matrix, sq2d_apply_operator, sq2d_rhs, sq2d_apply_precond,
)
