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
