"""GB300 (sm_103a) library for the volume-integral-equation hot path of the
two-step radiative-transfer method of Ren, Zhang & Zhong (arXiv 1610.00835).

The compute lives in ``libvie.so`` (CUDA, built from ``csrc/``); this package
is its ctypes binding.  See ``include/vie.h`` for the C ABI.
"""
from .vie import (VIE_DISC_MII, VIE_DISC_MIII, VIE_KERNEL_AUTO, VIE_KERNEL_DISPLACEMENT,
                  VIE_KERNEL_GENERAL, VIE_KERNEL_SYMMETRIC)
from .vie import (VieUnet, vie_diffusion_precondition, vie_set_diffusion_preconditioner, vie_fft_precondition, vie_set_fft_preconditioner, vie_set_preconditioner, vie_unet_create, vie_unet_destroy,
                  vie_unet_forward, vie_unet_get_params, vie_unet_load, vie_unet_loss_grad,
                  vie_unet_num_params, vie_unet_save, vie_unet_set_params, vie_unet_train_step,
                  vie_unet_train_state, vie_unet_layer_io)
from .vie import (VIE_ERR_TIMEOUT, vie_check_device, vie_set_wait_limits, vie_set_preconditioner_on_diffusion,
                  vie_release_memory)
from .vie import (VieBatch, vie_batch_apply, vie_batch_autotune, vie_batch_config,
                  vie_batch_create, vie_batch_destroy)
from .vie import (VIE_OPERATOR_FMM, vie_assemble_fmm)
from .vie import (VIE_OPERATOR_BF16X3, VIE_OPERATOR_FP32, VIE_OPERATOR_PAIRS32, VIE_OPERATOR_SYM32, VIE_OPERATOR_OTF, VIE_OP_A_RAW, VIE_OP_I_MINUS_K, VIE_OP_K_SIGMA_S, VIE_PREC_FP32,
                  VIE_PREC_FP64, VIE_TAU_CLOSED, VIE_TAU_MARCH, VieError, VieHandle, ert_sweep,
                  load, vie_apply, vie_apply_noalloc, vie_get_kernel, vie_get_kernel_work, vie_assemble, vie_create, vie_destroy, vie_get_diagonal, vie_last_error,
                  vie_kernel_launches, vie_solve_gmres, vie_version)

__all__ = ["VIE_DISC_MII", "VIE_DISC_MIII", "VIE_KERNEL_AUTO", "VIE_KERNEL_DISPLACEMENT", "VIE_KERNEL_GENERAL",
           "VIE_KERNEL_SYMMETRIC", "VieUnet", "vie_diffusion_precondition", "vie_set_diffusion_preconditioner",
           "vie_fft_precondition", "vie_set_fft_preconditioner",
           "vie_set_preconditioner", "vie_unet_create", "vie_unet_destroy",
           "vie_unet_forward", "vie_unet_get_params", "vie_unet_load", "vie_unet_loss_grad",
           "vie_unet_num_params", "vie_unet_save", "vie_unet_set_params", "vie_unet_train_step",
           "vie_unet_train_state", "vie_unet_layer_io", "VIE_ERR_TIMEOUT", "vie_check_device", "vie_set_wait_limits",
           "vie_set_preconditioner_on_diffusion", "vie_release_memory",
           "VieBatch", "vie_batch_apply", "vie_batch_autotune", "vie_batch_config",
           "vie_batch_create", "vie_batch_destroy",
           "VIE_OPERATOR_FMM", "vie_assemble_fmm", "VIE_OPERATOR_BF16X3", "VIE_OPERATOR_FP32", "VIE_OPERATOR_PAIRS32", "VIE_OPERATOR_SYM32", "VIE_OPERATOR_OTF", "VIE_OP_A_RAW", "VIE_OP_I_MINUS_K", "VIE_OP_K_SIGMA_S", "VIE_PREC_FP32",
           "VIE_PREC_FP64", "VIE_TAU_CLOSED", "VIE_TAU_MARCH", "VieError", "VieHandle",
           "ert_sweep", "load", "vie_apply", "vie_apply_noalloc", "vie_get_kernel", "vie_get_kernel_work", "vie_assemble", "vie_create", "vie_destroy", "vie_get_diagonal",
           "vie_kernel_launches", "vie_last_error", "vie_solve_gmres", "vie_version"]
