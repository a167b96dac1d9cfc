"""librbgs: randomized block Gram-Schmidt (Balabanov & Grigori, arXiv 2111.14641)
on one NVIDIA GB300 (sm_103a).

The computation lives in the C-ABI library ``librbgs.so`` (hand-written CUDA
kernels, include/rbgs.h); this package is its Python binding.
"""
from .rbgs import (NOALLOC_MAX_K, PREC, SKETCH, QRStats, RbgsError, colmajor, launch_count, load, philox, rbgs_qr,
                   release_workspace, sketch_apply, tall_update, tall_update_noalloc, version)

__all__ = ["NOALLOC_MAX_K", "PREC", "SKETCH", "QRStats", "RbgsError", "colmajor", "launch_count", "load", "philox",
           "rbgs_qr", "release_workspace", "sketch_apply", "tall_update", "tall_update_noalloc", "version"]
