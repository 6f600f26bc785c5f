"""Python binding of libos3d (include/os3d.h): argument marshalling only.

Every function here has the name of the C entry point it calls. Device
memory comes from torch tensors, streams from torch's current stream; all
arithmetic runs in the library's CUDA kernels. There is no fallback: if the
library is not built, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libos3d.so")

OS3D_U_C64 = 0
OS3D_U_BF16X2 = 1
_STATUS = {0: "OS3D_OK", 1: "OS3D_EINVAL", 2: "OS3D_ENOMEM", 3: "OS3D_ECUDA",
           4: "OS3D_ETIMEOUT", 5: "OS3D_EUNSUPPORTED"}
OS3D_EUNSUPPORTED = 5


class os3d_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("s_theta", ctypes.c_double), ("L", ctypes.c_int),
                ("N", ctypes.c_int), ("gamma", ctypes.c_double), ("eps", ctypes.c_double),
                ("fit_mode", ctypes.c_int), ("block_slots", ctypes.c_int),
                ("overlap", ctypes.c_int), ("profile", ctypes.c_int)]


class os3d_diffusion(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_int), ("D11", ctypes.c_double),
                ("D33", ctypes.c_double), ("D44", ctypes.c_double), ("sh_degree", ctypes.c_int)]


class os3d_server_config(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("udtype", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("bank_cache_bytes", ctypes.c_size_t)]


class OS3DError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)} "
                         f"({lib().os3d_status_string(status).decode()})")


_lib = None


def lib():
    """The loaded libos3d.so (ctypes)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_1505_07690_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.os3d_status_string.restype = ctypes.c_char_p
        L.os3d_status_string.argtypes = [i]
        L.os3d_default_params.argtypes = [ctypes.POINTER(os3d_params)]
        L.os3d_icosa_orientations.argtypes = [i, ctypes.POINTER(d), i, ctypes.POINTER(i)]
        L.os3d_octa_orientations.argtypes = [i, ctypes.POINTER(d), i, ctypes.POINTER(i)]
        L.os3d_approx_reconstruct.argtypes = [vp, vp, i, i, vp, vp]
        L.os3d_project.argtypes = [vp, vp, i, i, vp, vp, vp]
        L.os3d_soft_threshold.argtypes = [vp, vp, i, ctypes.c_longlong, d, vp]
        L.os3d_weighted_energy.argtypes = [vp, vp, i, ctypes.c_longlong, vp, vp, vp]
        L.os3d_weighted_energy_grad.argtypes = [vp, vp, i, ctypes.c_longlong, vp, vp, vp]
        L.os3d_upsilon.argtypes = [vp, vp, i, vp, d, vp, vp]
        L.os3d_default_diffusion.argtypes = [ctypes.POINTER(os3d_diffusion)]
        L.os3d_angular_propagator.argtypes = [ctypes.POINTER(d), i, i, d, ctypes.POINTER(d),
                                              ctypes.POINTER(i)]
        L.os3d_enhance_linear.argtypes = [vp, vp, i, vp, ctypes.POINTER(os3d_diffusion), vp, vp]
        L.os3d_make_wavelets.argtypes = [ctypes.POINTER(i), ctypes.POINTER(d), i,
                                         ctypes.POINTER(os3d_params), vp, ctypes.POINTER(vp)]
        L.os3d_forward.argtypes = [vp, vp, i, vp, i, vp, vp]
        L.os3d_inverse.argtypes = [vp, vp, i, i, vp, vp, vp]
        L.os3d_adjoint.argtypes = [vp, vp, i, i, vp, vp, vp]
        L.os3d_adjoint_weighted.argtypes = [vp, vp, vp, vp, i, i, vp, vp, vp]
        L.os3d_score_energy_grad.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, ctypes.c_size_t,
                                             vp, vp]
        L.os3d_score_energy_scratch.argtypes = [vp, i, ctypes.POINTER(ctypes.c_size_t)]
        L.os3d_scale_by.argtypes = [vp, vp, ctypes.c_longlong, vp, vp]
        L.os3d_bank_info.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]
        L.os3d_bank_resident_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.os3d_bank_wait_errors.argtypes = [vp, ctypes.POINTER(ctypes.c_uint), i]
        L.os3d_wait_selftest.argtypes = [d, i, ctypes.POINTER(ctypes.c_uint)]
        L.os3d_bank_coefficients.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.os3d_bank_minv.argtypes = [vp, vp, vp]
        L.os3d_destroy_bank.argtypes = [vp]
        L.os3d_launch_count.restype = ctypes.c_ulonglong
        L.os3d_launch_count.argtypes = []
        L.os3d_profile_enable.argtypes = [i]
        L.os3d_profile_read.argtypes = [i, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(d)]
        L.os3d_profile_reset.argtypes = []
        L.os3d_forward_static.argtypes = [vp, vp, i, vp, i, vp]
        L.os3d_server_default_config.argtypes = [ctypes.POINTER(os3d_server_config)]
        L.os3d_server_create.argtypes = [ctypes.POINTER(os3d_server_config),
                                         ctypes.POINTER(os3d_params), ctypes.POINTER(vp)]
        L.os3d_server_submit.argtypes = [vp, ctypes.POINTER(i), i, vp, vp,
                                         ctypes.POINTER(ctypes.c_longlong)]
        L.os3d_server_wait.argtypes = [vp, ctypes.c_longlong, d, ctypes.POINTER(d)]
        L.os3d_server_destroy.argtypes = [vp]
        L.os3d_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_longlong)]
        L.os3d_kernel_kind_name.restype = ctypes.c_char_p
        L.os3d_kernel_kind_name.argtypes = [i]
        for name in ("os3d_default_params", "os3d_icosa_orientations", "os3d_make_wavelets",
                     "os3d_forward", "os3d_inverse", "os3d_adjoint", "os3d_bank_info",
                     "os3d_bank_coefficients", "os3d_bank_minv", "os3d_destroy_bank",
                     "os3d_profile_enable", "os3d_profile_read", "os3d_profile_reset",
                     "os3d_forward_static", "os3d_server_default_config",
                     "os3d_server_create", "os3d_server_submit", "os3d_server_wait",
                     "os3d_server_destroy", "os3d_octa_orientations",
                     "os3d_approx_reconstruct", "os3d_project", "os3d_soft_threshold",
                     "os3d_upsilon", "os3d_default_diffusion", "os3d_enhance_linear",
                     "os3d_angular_propagator", "os3d_server_stats",
                     "os3d_bank_resident_bytes", "os3d_bank_wait_errors", "os3d_wait_selftest",
                     "os3d_weighted_energy", "os3d_weighted_energy_grad",
                     "os3d_adjoint_weighted", "os3d_score_energy_grad",
                     "os3d_score_energy_scratch", "os3d_scale_by"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def _check(status, where):
    if status != 0:
        raise OS3DError(status, where)


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def os3d_default_params(**overrides) -> os3d_params:
    p = os3d_params()
    _check(lib().os3d_default_params(ctypes.byref(p)), "os3d_default_params")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _orientations(fn, name, subdiv):
    n = ctypes.c_int(0)
    fn(int(subdiv), None, 0, ctypes.byref(n))
    if n.value <= 0:
        raise OS3DError(1, name)
    out = np.zeros((n.value, 3), dtype=np.float64)
    _check(fn(int(subdiv), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
              ctypes.byref(n)), name)
    return out


def os3d_icosa_orientations(subdiv: int) -> np.ndarray:
    return _orientations(lib().os3d_icosa_orientations, "os3d_icosa_orientations", subdiv)


def os3d_octa_orientations(subdiv: int) -> np.ndarray:
    return _orientations(lib().os3d_octa_orientations, "os3d_octa_orientations", subdiv)


class Bank:
    """Handle of a library-owned wavelet bank (os3d_bank*)."""

    def __init__(self, handle, dims, n_o, params):
        self.handle = handle
        self.dims = tuple(dims)
        self.n_o = n_o
        self.params = params
        ws, fp = ctypes.c_size_t(0), ctypes.c_size_t(0)
        _check(lib().os3d_bank_info(handle, ctypes.byref(ws), ctypes.byref(fp)), "os3d_bank_info")
        self.workspace_bytes = ws.value
        self.footprint_bytes_per_volume = fp.value

    def wait_errors(self, reset: bool = True) -> int:
        """Bounded waits that ran out in this bank's kernels (os3d_bank_wait_errors)."""
        n = ctypes.c_uint(0)
        _check(lib().os3d_bank_wait_errors(self.handle, ctypes.byref(n), 1 if reset else 0),
               "os3d_bank_wait_errors")
        return n.value

    def resident_bytes(self) -> int:
        """Device bytes the bank holds now (os3d_bank_resident_bytes)."""
        n = ctypes.c_size_t(0)
        _check(lib().os3d_bank_resident_bytes(self.handle, ctypes.byref(n)),
               "os3d_bank_resident_bytes")
        return n.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.os3d_destroy_bank(h)
            self.handle = None


def os3d_make_wavelets(dims, orient, params: os3d_params | None = None, stream=None) -> Bank:
    dims_c = (ctypes.c_int * 3)(*[int(d) for d in dims])
    o = np.ascontiguousarray(np.asarray(orient, dtype=np.float64).reshape(-1, 3))
    p = params if params is not None else os3d_default_params()
    h = ctypes.c_void_p(0)
    _check(lib().os3d_make_wavelets(dims_c, o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    len(o), ctypes.byref(p), _stream(stream), ctypes.byref(h)),
           "os3d_make_wavelets")
    return Bank(h, dims, len(o), p)


def os3d_destroy_bank(bank: Bank):
    if bank.handle:
        _check(lib().os3d_destroy_bank(bank.handle), "os3d_destroy_bank")
        bank.handle = None


def os3d_bank_coefficients(bank: Bank):
    L = bank.params.L
    b = np.zeros(L + 1)
    c = np.zeros(L + 1)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().os3d_bank_coefficients(bank.handle, b.ctypes.data_as(dp), c.ctypes.data_as(dp)),
           "os3d_bank_coefficients")
    return b, c


def os3d_bank_minv(bank: Bank, stream=None):
    import torch
    out = torch.empty(bank.dims, dtype=torch.float32, device="cuda")
    _check(lib().os3d_bank_minv(bank.handle, _ptr(out), _stream(stream)), "os3d_bank_minv")
    return out


def _udtype(U):
    import torch
    if U.dtype == torch.complex64:
        return OS3D_U_C64
    if U.dtype == torch.bfloat16 and U.shape[-1] == 2:
        return OS3D_U_BF16X2
    raise TypeError("U must be complex64, or bfloat16 with a trailing (re, im) axis of 2")


def _batch_of(x, nd, dims):
    if tuple(x.shape[-nd:]) != tuple(dims):
        raise ValueError(f"shape {tuple(x.shape)} does not end with {tuple(dims)}")
    return int(np.prod(x.shape[:-nd])) if x.dim() > nd else 1


def new_score(bank: Bank, batch: int, bf16: bool = False):
    import torch
    shape = (batch, bank.n_o) + bank.dims
    if bf16:
        return torch.empty(shape + (2,), dtype=torch.bfloat16, device="cuda")
    return torch.empty(shape, dtype=torch.complex64, device="cuda")


def _check_score(bank, U):
    if not (U.is_cuda and U.is_contiguous()):
        raise ValueError("U must be a contiguous CUDA tensor")
    ud = _udtype(U)
    core = U.shape[:-1] if ud == OS3D_U_BF16X2 else U.shape
    if tuple(core[-4:]) != (bank.n_o,) + bank.dims:
        raise ValueError(f"score shape {tuple(U.shape)} does not match the bank")
    batch = int(np.prod(core[:-4])) if len(core) > 4 else 1
    return ud, batch


def _ws_ptr(workspace):
    return ctypes.c_void_p(0) if workspace is None else _ptr(workspace)


def os3d_forward(bank: Bank, f, U=None, bf16: bool = False, workspace=None, stream=None):
    """U = W f (Eq. construction1Discrete) for real float32 volumes f."""
    import torch
    if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    batch = _batch_of(f, 3, bank.dims)
    if U is None:
        U = new_score(bank, batch, bf16)
    ud, ub = _check_score(bank, U)
    if ub != batch:
        raise ValueError("batch of U and f differ")
    _check(lib().os3d_forward(bank.handle, _ptr(f), batch, _ptr(U), ud, _ws_ptr(workspace),
                              _stream(stream)), "os3d_forward")
    return U


def os3d_forward_static(bank: Bank, f, U=None, bf16: bool = False, stream=None):
    """os3d_forward with the scratch in the library's fixed static device array
    instead of a workspace: allocates no device memory itself (U is
    allocated here only when the caller passes none). For volumes of at most
    64^3 voxels; concurrent calls race on the shared array."""
    import torch
    if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    batch = _batch_of(f, 3, bank.dims)
    if U is None:
        U = new_score(bank, batch, bf16)
    ud, ub = _check_score(bank, U)
    if ub != batch:
        raise ValueError("batch of U and f differ")
    _check(lib().os3d_forward_static(bank.handle, _ptr(f), batch, _ptr(U), ud, _stream(stream)),
           "os3d_forward_static")
    return U


def _backward(fn, name, bank, U, out, workspace, stream):
    import torch
    ud, batch = _check_score(bank, U)
    if out is None:
        out = torch.empty((batch,) + bank.dims, dtype=torch.float32, device="cuda")
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
            and out.numel() == batch * int(np.prod(bank.dims))):
        raise ValueError("output must be a contiguous float32 CUDA tensor of the batch's size")
    _check(fn(bank.handle, _ptr(U), ud, batch, _ptr(out), _ws_ptr(workspace), _stream(stream)), name)
    return out


def os3d_inverse(bank: Bank, U, f_out=None, workspace=None, stream=None):
    """Exact inverse (Eq. Reconstruction1Discrete, Sec. 3.1 clamp)."""
    return _backward(lib().os3d_inverse, "os3d_inverse", bank, U, f_out, workspace, stream)


def os3d_adjoint(bank: Bank, G, grad_f=None, workspace=None, stream=None):
    """Re W^* G: the gradient with respect to a real image."""
    return _backward(lib().os3d_adjoint, "os3d_adjoint", bank, G, grad_f, workspace, stream)


def os3d_adjoint_weighted(bank: Bank, U, w, g=None, grad_f=None, workspace=None, stream=None):
    """Re W^*(2 g w U), the gradient of g sum w |U|^2 at U = W f, with the
    weighting folded into the plane pass (complex64 U; OS3DError with
    OS3D_EUNSUPPORTED where the plane pass does not hold the grid's planes)."""
    import torch
    if g is None:
        g = torch.ones((), dtype=torch.float32, device="cuda")
    if not (g.is_cuda and g.dtype == torch.float32 and g.numel() == 1):
        raise ValueError("g must be a one-element float32 CUDA tensor")
    _, count, wp = _energy_operands(U, w)
    if w is None:
        raise ValueError("w is required (w = 1 is os3d_adjoint of 2 g U)")
    gc = g.contiguous()

    def fn(h, Up, ud, batch, out, ws, st):
        return lib().os3d_adjoint_weighted(h, Up, wp, _ptr(gc), ud, batch, out, ws, st)
    return _backward(fn, "os3d_adjoint_weighted", bank, U, grad_f, workspace, stream)


def os3d_score_energy_scratch(bank: Bank, batch: int) -> int:
    """Doubles of scratch os3d_score_energy_grad needs for `batch` volumes."""
    n = ctypes.c_size_t(0)
    _check(lib().os3d_score_energy_scratch(bank.handle, int(batch), ctypes.byref(n)),
           "os3d_score_energy_scratch")
    return int(n.value)


def os3d_score_energy_grad(bank: Bank, f, w, g=None, grad_f=None, scratch=None,
                           workspace=None, stream=None):
    """(L, grad_f): L = sum w |W f|^2 as a 0-dim float32 CUDA tensor and
    grad_f = Re W^*(2 g w W f), in one sweep that never stores the score
    (planes of the plane pass: square 16^2 to 128^2, 256^2 and 128 x 160;
    OS3DError with OS3D_EUNSUPPORTED elsewhere)."""
    import torch
    if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    batch = _batch_of(f, 3, bank.dims)
    n = batch * bank.n_o * int(np.prod(bank.dims))
    if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous() and w.numel() == n):
        raise ValueError("w must be a contiguous float32 CUDA tensor of the score's size")
    if g is not None and not (g.is_cuda and g.dtype == torch.float32 and g.numel() == 1):
        raise ValueError("g must be a one-element float32 CUDA tensor")
    if grad_f is None:
        grad_f = torch.empty_like(f)
    need = os3d_score_energy_scratch(bank, batch)
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.float64, device=f.device)
    if not (scratch.is_cuda and scratch.dtype == torch.float64 and scratch.is_contiguous()
            and scratch.numel() >= need):
        raise ValueError("scratch must be a float64 CUDA tensor of os3d_score_energy_scratch")
    loss = torch.empty((), dtype=torch.float32, device=f.device)
    gp = ctypes.c_void_p(None) if g is None else _ptr(g.contiguous())
    _check(lib().os3d_score_energy_grad(bank.handle, _ptr(f), _ptr(w), gp, batch, _ptr(loss),
                                        _ptr(grad_f), _ptr(scratch), scratch.numel(),
                                        _ws_ptr(workspace), _stream(stream)),
           "os3d_score_energy_grad")
    return loss, grad_f


def os3d_scale_by(x, g, out=None, stream=None):
    """g x (float32 CUDA tensor x, one-element float32 CUDA g); out may be x."""
    import torch
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    if not (g.is_cuda and g.dtype == torch.float32 and g.numel() == 1):
        raise ValueError("g must be a one-element float32 CUDA tensor")
    if out is None:
        out = torch.empty_like(x)
    if out.dtype != x.dtype or out.shape != x.shape or not out.is_contiguous():
        raise ValueError("out must match x")
    _check(lib().os3d_scale_by(_ptr(x), _ptr(out), x.numel(), _ptr(g.contiguous()),
                               _stream(stream)), "os3d_scale_by")
    return out


def os3d_approx_reconstruct(bank: Bank, U, f_out=None, stream=None):
    """Approximate reconstruction Re sum_i U_i / (N_o c_0)
    (Eq. Reconstruction2Approximation)."""
    import torch
    ud, batch = _check_score(bank, U)
    if f_out is None:
        f_out = torch.empty((batch,) + bank.dims, dtype=torch.float32, device="cuda")
    if not (f_out.is_cuda and f_out.dtype == torch.float32 and f_out.is_contiguous()
            and f_out.numel() == batch * int(np.prod(bank.dims))):
        raise ValueError("output must be a contiguous float32 CUDA tensor of the batch's size")
    _check(lib().os3d_approx_reconstruct(bank.handle, _ptr(U), ud, batch, _ptr(f_out),
                                         _stream(stream)), "os3d_approx_reconstruct")
    return f_out


def os3d_project(bank: Bank, U, U_out=None, workspace=None, stream=None):
    """P_psi U = W W^{*,ext} U (App. A); U_out may be U."""
    import torch
    ud, batch = _check_score(bank, U)
    if U_out is None:
        U_out = torch.empty_like(U)
    ud2, b2 = _check_score(bank, U_out)
    if ud2 != ud or b2 != batch:
        raise ValueError("U_out must match U")
    _check(lib().os3d_project(bank.handle, _ptr(U), ud, batch, _ptr(U_out), _ws_ptr(workspace),
                              _stream(stream)), "os3d_project")
    return U_out


def os3d_soft_threshold(U, power: float = 1.5, out=None, stream=None):
    """Phi(U) = |U|^p sgn(U) per real and imaginary part (Sec. 4.1); out may be U."""
    import torch
    ud = _udtype(U)
    if not (U.is_cuda and U.is_contiguous()):
        raise ValueError("U must be a contiguous CUDA tensor")
    if out is None:
        out = torch.empty_like(U)
    if out.dtype != U.dtype or out.shape != U.shape or not out.is_contiguous():
        raise ValueError("out must match U")
    count = U.numel() // 2 if ud == OS3D_U_BF16X2 else U.numel()
    _check(lib().os3d_soft_threshold(_ptr(U), _ptr(out), ud, count, float(power), _stream(stream)),
           "os3d_soft_threshold")
    return out


OS3D_ENERGY_SCRATCH_DOUBLES = 4097


def _energy_operands(U, w):
    import torch
    ud = _udtype(U)
    if not (U.is_cuda and U.is_contiguous()):
        raise ValueError("U must be a contiguous CUDA tensor")
    count = U.numel() // 2 if ud == OS3D_U_BF16X2 else U.numel()
    if w is not None:
        if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()
                and w.numel() == count):
            raise ValueError("w must be a contiguous float32 CUDA tensor, one weight per "
                             "complex element of U")
    return ud, count, (ctypes.c_void_p(None) if w is None else _ptr(w))


def os3d_weighted_energy(U, w=None, scratch=None, stream=None):
    """L = sum w |U|^2 (w = 1 when None) as a 0-dim float32 CUDA tensor, summed
    in FP32 over 16 terms and FP64 above; `scratch` (float64 CUDA tensor of
    OS3D_ENERGY_SCRATCH_DOUBLES) keeps the FP64 sum in scratch[0]."""
    import torch
    ud, count, wp = _energy_operands(U, w)
    if scratch is None:
        scratch = torch.empty(OS3D_ENERGY_SCRATCH_DOUBLES, dtype=torch.float64, device=U.device)
    if not (scratch.is_cuda and scratch.dtype == torch.float64 and scratch.is_contiguous()
            and scratch.numel() >= OS3D_ENERGY_SCRATCH_DOUBLES):
        raise ValueError("scratch must be a float64 CUDA tensor of OS3D_ENERGY_SCRATCH_DOUBLES")
    loss = torch.empty((), dtype=torch.float32, device=U.device)
    _check(lib().os3d_weighted_energy(_ptr(U), wp, ud, count, _ptr(scratch), _ptr(loss),
                                      _stream(stream)), "os3d_weighted_energy")
    return loss


def os3d_weighted_energy_grad(U, w=None, g=None, out=None, stream=None):
    """G = 2 g w U (PyTorch's gradient of sum w |U|^2 scaled by the upstream
    0-dim float32 CUDA tensor g, 1 when None); out may be U."""
    import torch
    ud, count, wp = _energy_operands(U, w)
    if g is None:
        g = torch.ones((), dtype=torch.float32, device=U.device)
    if not (g.is_cuda and g.dtype == torch.float32 and g.numel() == 1):
        raise ValueError("g must be a one-element float32 CUDA tensor")
    if out is None:
        out = torch.empty_like(U)
    if out.dtype != U.dtype or out.shape != U.shape or not out.is_contiguous():
        raise ValueError("out must match U")
    _check(lib().os3d_weighted_energy_grad(_ptr(U), wp, ud, count, _ptr(g.contiguous()), _ptr(out),
                                           _stream(stream)), "os3d_weighted_energy_grad")
    return out


def os3d_upsilon(bank: Bank, f, power: float = 1.5, f_out=None, workspace=None, stream=None):
    """Upsilon f = W^{*,ext} Phi W f (Sec. 4.1) without storing the score."""
    import torch
    if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    batch = _batch_of(f, 3, bank.dims)
    if f_out is None:
        f_out = torch.empty_like(f)
    if not (f_out.is_cuda and f_out.dtype == torch.float32 and f_out.is_contiguous()
            and f_out.numel() == f.numel()):
        raise ValueError("f_out must be a contiguous float32 CUDA tensor like f")
    _check(lib().os3d_upsilon(bank.handle, _ptr(f), batch, _ptr(f_out), float(power),
                              _ws_ptr(workspace), _stream(stream)), "os3d_upsilon")
    return f_out


def os3d_default_diffusion(**overrides) -> os3d_diffusion:
    d = os3d_diffusion()
    _check(lib().os3d_default_diffusion(ctypes.byref(d)), "os3d_default_diffusion")
    for k, v in overrides.items():
        setattr(d, k, v)
    return d


def os3d_angular_propagator(orient, tau: float, sh_degree: int = 0):
    """(exp(tau L) as an (n, n) array, degree used) for the discrete
    Laplace-Beltrami operator on the orientation set (host, FP64)."""
    o = np.ascontiguousarray(np.asarray(orient, dtype=np.float64).reshape(-1, 3))
    n = len(o)
    E = np.zeros((n, n))
    deg = ctypes.c_int(0)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().os3d_angular_propagator(o.ctypes.data_as(dp), n, int(sh_degree), float(tau),
                                         E.ctypes.data_as(dp), ctypes.byref(deg)),
           "os3d_angular_propagator")
    return E, deg.value


def os3d_enhance_linear(bank: Bank, f, diffusion: os3d_diffusion | None = None, f_out=None,
                        workspace=None, stream=None):
    """Upsilon f = W^{*,ext} Phi_t W f with the linear left-invariant diffusion
    Phi_t (Sec. 4.1), integrated per frequency without forming the score."""
    import torch
    if not (f.is_cuda and f.dtype == torch.float32 and f.is_contiguous()):
        raise ValueError("f must be a contiguous float32 CUDA tensor")
    batch = _batch_of(f, 3, bank.dims)
    d = diffusion if diffusion is not None else os3d_default_diffusion()
    if f_out is None:
        f_out = torch.empty_like(f)
    if not (f_out.is_cuda and f_out.dtype == torch.float32 and f_out.is_contiguous()
            and f_out.numel() == f.numel()):
        raise ValueError("f_out must be a contiguous float32 CUDA tensor like f")
    _check(lib().os3d_enhance_linear(bank.handle, _ptr(f), batch, _ptr(f_out), ctypes.byref(d),
                                     _ws_ptr(workspace), _stream(stream)), "os3d_enhance_linear")
    return f_out


OS3D_KIND_COUNT = 14


def os3d_wait_selftest(limit_s: float, arrive: bool) -> int:
    """Threads of the bounded-wait self-test whose wait ran out (64 or 0)."""
    n = ctypes.c_uint(0)
    _check(lib().os3d_wait_selftest(float(limit_s), 1 if arrive else 0, ctypes.byref(n)),
           "os3d_wait_selftest")
    return n.value


def os3d_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().os3d_launch_count())


def os3d_profile_enable(on: bool = True):
    _check(lib().os3d_profile_enable(1 if on else 0), "os3d_profile_enable")


def os3d_profile_reset():
    _check(lib().os3d_profile_reset(), "os3d_profile_reset")


def os3d_profile_read():
    """{kernel kind name: (launches, total ms)} since the last reset."""
    out = {}
    for k in range(OS3D_KIND_COUNT):
        n = ctypes.c_ulonglong(0)
        ms = ctypes.c_double(0.0)
        _check(lib().os3d_profile_read(k, ctypes.byref(n), ctypes.byref(ms)), "os3d_profile_read")
        out[lib().os3d_kernel_kind_name(k).decode()] = (int(n.value), float(ms.value))
    return out


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def os3d_server_default_config(**overrides) -> os3d_server_config:
    c = os3d_server_config()
    _check(lib().os3d_server_default_config(ctypes.byref(c)), "os3d_server_default_config")
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


class Server:
    """os3d_server: queued forward + inverse requests on one GPU. Host buffers
    are page-locked torch tensors kept alive until each request is waited for."""

    def __init__(self, config: os3d_server_config | None = None, params: os3d_params | None = None):
        self.handle = None
        cfg = config if config is not None else os3d_server_default_config()
        h = ctypes.c_void_p(0)
        _check(lib().os3d_server_create(ctypes.byref(cfg), None if params is None else ctypes.byref(params),
                                        ctypes.byref(h)), "os3d_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, f_host, subdiv: int, f_out=None) -> int:
        """Queue f_host (pinned float32 CPU tensor (nz, ny, nx)); returns the ticket."""
        import torch
        if f_host.device.type != "cpu" or f_host.dtype != torch.float32 or not f_host.is_contiguous():
            raise ValueError("f_host must be a contiguous float32 CPU tensor")
        if f_out is None:
            f_out = torch.empty_like(f_host).pin_memory()
        dims = (ctypes.c_int * 3)(*[int(x) for x in f_host.shape[-3:]])
        t = ctypes.c_longlong(0)
        _check(lib().os3d_server_submit(self.handle, dims, int(subdiv), _ptr(f_host), _ptr(f_out),
                                        ctypes.byref(t)), "os3d_server_submit")
        self._keep[t.value] = (f_host, f_out)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0):
        """(f_out tensor, latency in ms); raises OS3DError (OS3D_ETIMEOUT on timeout)."""
        lat = ctypes.c_double(0.0)
        st = lib().os3d_server_wait(self.handle, ctypes.c_longlong(ticket), float(timeout_s),
                                    ctypes.byref(lat))
        if st == 4:
            raise OS3DError(st, "os3d_server_wait")
        f_host, f_out = self._keep.pop(ticket)
        _check(st, "os3d_server_wait")
        return f_out, lat.value

    def stats(self):
        """(completed requests, graphs captured, graph replays)."""
        v = [ctypes.c_longlong(0) for _ in range(3)]
        _check(lib().os3d_server_stats(self.handle, *[ctypes.byref(x) for x in v]),
               "os3d_server_stats")
        return tuple(x.value for x in v)

    def close(self):
        if self.handle:
            _check(lib().os3d_server_destroy(self.handle), "os3d_server_destroy")
            self.handle = None
            self._keep.clear()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.os3d_server_destroy(self.handle)
            self.handle = None
