"""The workspace-free forward transform (os3d_forward_static) against the
ordinary one. Callers that cannot allocate device memory while they run the
transform use it; its scratch is a fixed array inside the library, shared by
all calls. This file sorts last so that a failure here comes after every
other test has run; it also passes when run on its own."""
import ctypes

import numpy as np
import pytest

from paper_1505_07690_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_07690_gb300 import build, os3d
    build.build()
    return os3d


@pytest.mark.parametrize("dims,subdiv", [((32, 32, 32), 1), ((64, 64, 64), 0)])
def test_static_scratch_forward_matches_forward(M, dims, subdiv):
    import torch
    V = M.os3d_icosa_orientations(subdiv)
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=12))
    f = torch.from_numpy(np.stack([synth.straight_tubes(dims, 3, seed=s) for s in (21, 22)])).cuda()
    ref = M.os3d_forward(bank, f)
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy()
    L = M.lib()
    for _ in range(2):   # two calls in a row share (and overwrite) the static array
        U = M.new_score(bank, 2)
        U.fill_(float("nan"))
        st = L.os3d_forward_static(bank.handle, ctypes.c_void_p(f.data_ptr()), 2,
                                   ctypes.c_void_p(U.data_ptr()), 0,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        assert rel(U.cpu().numpy(), ref_np) <= TOL


def test_static_scratch_rejects_larger_volumes(M):
    import torch
    dims = (96, 96, 96)
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(0), M.os3d_default_params(L=8))
    f = torch.zeros((1,) + dims, device="cuda")
    U = M.new_score(bank, 1)
    L = M.lib()
    st = L.os3d_forward_static(bank.handle, ctypes.c_void_p(f.data_ptr()), 1,
                               ctypes.c_void_p(U.data_ptr()), 0, None)
    assert st == 1   # OS3D_EINVAL: larger than the static scratch


@pytest.mark.parametrize("bf16", [False, True])
def test_static_scratch_forward_on_a_pencil_grid_against_the_oracle(M, bf16):
    """A 32 x 48 x 64 grid (non-square planes: the pencil passes, including
    the in-place y pass on the static scratch), through the Python wrapper,
    complex64 and BF16 scores, against the FP64 oracle; two calls in a row."""
    import torch
    from oracle import os3d_oracle as O
    dims = (32, 48, 64)
    f = synth.straight_tubes(dims, 3, seed=23, noise=0.1)
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(1), M.os3d_default_params(L=12))
    Uo = O.forward(f, O.Bank(dims, O.icosa_orientations(1), O.Params(L=12)))
    fd = torch.from_numpy(f).cuda()
    for _ in range(2):
        U = M.os3d_forward_static(bank, fd, bf16=bf16)
        torch.cuda.synchronize()
        if bf16:
            Ug = U.float().cpu().numpy()[0]
            Ug = Ug[..., 0] + 1j * Ug[..., 1]
        else:
            Ug = U.cpu().numpy()[0]
        assert rel(Ug, Uo) <= (5e-3 if bf16 else TOL)
        assert np.abs(Ug - Uo).max() <= (1e-2 if bf16 else 2e-5) * np.abs(Uo).max()


def test_static_scratch_forward_keeps_no_device_memory(M):
    """After the first call (which may load the library's device code and
    with it the static array), further calls leave the device's free memory
    unchanged: the entry point holds no allocation of its own."""
    import torch
    dims = (64, 64, 64)
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(1), M.os3d_default_params(L=12))
    f = torch.from_numpy(synth.straight_tubes(dims, 3, seed=24)).cuda()
    U = M.new_score(bank, 1)
    M.os3d_forward_static(bank, f, U)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        M.os3d_forward_static(bank, f, U)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
