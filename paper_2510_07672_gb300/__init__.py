"""GB300-native Parareal with a convolutional coarse propagator for the classic
and mass-conservative Allen-Cahn equations (arXiv 2510.07672, Sec. 3).

The compute path is the C-ABI library ``libacpr.so`` (hand-written sm_103a CUDA,
declared in ``include/acpr.h``).  This package only builds and loads it and
marshals arguments: torch tensors supply device memory and the current CUDA
stream.  There is no CPU fallback; every call fails loudly if the library or a
GPU is missing.
"""
from .abi import (  # noqa: F401
    AC_CLASSIC, AC_MASS_CONSERVING, AC_F64, AC_F32, AC_ACT_TANH, AC_ACT_GELU,
    AcprError, load, lib_path,
    ac_fine_supported, ac_fine_step, ac_fine_propagate_slices, ac_cn_propagate_slices,
    ac_fine_workspace_bytes, ac_fine_propagate_slices_ws,
    ac_fine_variants, ac_fine_set_variant, ac_fine_get_variant, ac_fine_autotune, ac_fine_propagate_work,
    ac_fine_trajectory, ac_fine_adjoint, ac_energy, ac_energy_grad, ac_energy_gradient_ic,
    cnn_packed_bytes, cnn_work_bytes, cnn_pack_weights, cnn_coarse_step, ac_conv_status, ac_test_conv_stall, cnn_train_set_wgrad_tc,
    cnn_conv_variants, cnn_conv_set_variant, cnn_autotune,
    parareal_residual, parareal_residual_noalloc, ac_launch_count, parareal_solve_many, Parareal, CoarseNet, FineParams,
    TrainableCoarseNet, mse_loss_grad, coarse_step_function, fine_solve_function, fine_solve,
    Acnn, acnn_param_count, loss_acn, ac_fine3d_propagate,
)
