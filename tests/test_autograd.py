"""Differentiation: U = W f as a torch.autograd.Function whose backward is the
library's adjoint kernel path (Re W^* G). Loss = sum w |U|^2, w ~ U(0, 1)."""
import numpy as np
import pytest

from oracle import os3d_oracle as O
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


def test_gradient_matches_oracle_adjoint_batch8_96(M):
    """8 x 96^3 spline-tube volumes, 42 orientations, L = 16, the benchmark's
    differentiation workload: with the loss taken by torch's elementwise ops
    and with the fused weighted-energy kernels, the autograd gradient equals
    the oracle's Re W^*(2 w U) on every volume of the batch (relative L2 <=
    1e-5, element-wise <= 2e-5 of the largest value), and so does score_energy
    (the weighted adjoint, no stored gradient); the fused loss equals the
    oracle's energy (relative 2e-5)."""
    import torch
    from paper_1505_07690_gb300.autograd import orientation_score, weighted_energy
    dims = (96, 96, 96)
    f = np.stack([synth.workload_volume("splines96x8_no42", batch_index=b) for b in range(8)])
    w = synth.score_weights((8, 42) + dims, seed=1)
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(1), M.os3d_default_params(L=16))
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    U = orientation_score(ft, bank)
    loss = (wt * (U.real ** 2 + U.imag ** 2)).sum()
    loss.backward()
    torch.cuda.synchronize()
    g_torch = ft.grad.cpu().numpy()
    del U, loss
    ft.grad = None
    loss = weighted_energy(orientation_score(ft, bank), wt)
    loss.backward()
    g_fused = ft.grad.cpu().numpy()
    L_fused = loss.item()
    del loss
    from paper_1505_07690_gb300.autograd import score_energy
    ft.grad = None
    loss = score_energy(ft, bank, wt)
    loss.backward()
    g_score = ft.grad.cpu().numpy()
    assert loss.item() == L_fused
    del loss, wt
    torch.cuda.empty_cache()
    from _oracle_pool import energy_and_adjoint_of_weighted_score, oracle_map
    res = oracle_map(energy_and_adjoint_of_weighted_score,
                     [(f[b], w[b], dims, 1, 16) for b in range(8)])
    for b in range(8):
        ref = res[b][1]
        for g in (g_torch, g_fused, g_score):
            assert rel(g[b], ref) <= TOL, b
            assert np.abs(g[b] - ref).max() <= 2e-5 * np.abs(ref).max(), b
    L_ref = sum(r[0] for r in res)
    assert abs(L_fused - L_ref) <= 2e-5 * L_ref


def test_gradient_against_fp64_central_differences(M):
    """Central differences of the loss in FP64 (the oracle, eps = 1e-3) along
    random directions agree with the GPU gradient; the loss is quadratic in
    f, so central differences are exact up to rounding."""
    import torch
    from paper_1505_07690_gb300.autograd import orientation_score
    dims = (16, 16, 16)
    f = synth.workload_volume("splines96x8_no42")[40:56, 40:56, 40:56].copy()
    w = synth.score_weights((42,) + dims, seed=1)
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(1), M.os3d_default_params(L=16))
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    U = orientation_score(ft, bank)
    (torch.from_numpy(w).cuda() * U.abs() ** 2).sum().backward()
    g = ft.grad.cpu().numpy().astype(np.float64)
    ob = O.Bank(dims, O.icosa_orientations(1), O.Params(L=16))
    w64 = w.astype(np.float64)
    f64 = f.astype(np.float64)

    def loss(x):
        return float(np.sum(w64 * np.abs(O.forward(x, ob)) ** 2))

    rng = np.random.default_rng(3)
    eps = 1e-3
    for _ in range(3):
        d = rng.standard_normal(dims)
        fd = (loss(f64 + eps * d) - loss(f64 - eps * d)) / (2 * eps)
        assert abs(float(np.sum(g * d)) - fd) <= TOL * abs(fd)
