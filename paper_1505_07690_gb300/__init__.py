"""GB300-native invertible 3D orientation scores (arXiv 1505.07690).

The transform runs in libos3d.so (hand-written sm_103a CUDA behind a C ABI,
include/os3d.h); ``os3d`` is its ctypes binding and ``autograd`` wraps the
forward transform and its adjoint as a torch.autograd.Function.
"""
from .os3d import (Bank, OS3DError, os3d_adjoint, os3d_bank_coefficients, os3d_bank_minv,  # noqa: F401
                   os3d_default_params, os3d_destroy_bank, os3d_forward, os3d_icosa_orientations,
                   os3d_inverse, os3d_make_wavelets, new_score)
