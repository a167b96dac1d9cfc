"""librbgs: randomized block Gram-Schmidt (Balabanov & Grigori, arXiv 2111.14641)
on one NVIDIA GB300 (sm_103a).

The computation lives in the C-ABI library ``librbgs.so`` (hand-written CUDA
kernels, include/rbgs.h); this package is its Python binding.
"""
from .autotune import BatchTuner, rbgs_qr_batched_auto
from .rbgs import (NOALLOC_MAX_K, PREC, SKETCH, BatchedQRGraph, Op, QRGraph, QRStats, RbgsError, block_arnoldi, block_fom,
                   block_gmres, cholqr_postprocess, colmajor, embedding_check, launch_count, load, op_apply, philox,
                   rayleigh_ritz, rbgs_qr, rbgs_qr_batched, rbgs_qr_host, release_workspace, sketch_apply,
                   sparse_sign_columns, gaussian_entries, stencil_op, tall_update, tall_update_noalloc, version, UNet, adam_step,
                   block_fgmres, diffusion_faces, diffusion_op, unet_backward, unet_forward, unet_num_params,
                   unet_precondition, unet_residual_loss, unet_scale_inputs, unet_shape)

__all__ = ["BatchTuner", "rbgs_qr_batched_auto", "NOALLOC_MAX_K", "PREC", "SKETCH", "BatchedQRGraph", "Op", "QRGraph", "QRStats", "RbgsError", "block_arnoldi", "block_fom",
           "block_gmres", "cholqr_postprocess", "colmajor", "embedding_check", "launch_count", "load", "op_apply", "philox",
           "rayleigh_ritz", "rbgs_qr", "rbgs_qr_batched", "rbgs_qr_host", "release_workspace",
           "sketch_apply", "sparse_sign_columns", "gaussian_entries", "stencil_op", "tall_update", "tall_update_noalloc", "version",
           "UNet", "adam_step", "block_fgmres", "diffusion_faces", "diffusion_op", "unet_backward", "unet_forward",
           "unet_num_params", "unet_precondition", "unet_residual_loss", "unet_scale_inputs", "unet_shape"]
