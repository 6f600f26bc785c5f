"""GPU parity of the weighted energy L = sum w |U|^2 of a score (the squared
L_2(R^3 x S^2) norm of Sec. 2) and of its gradient 2 g w U, through the C
ABI, against the FP64 oracle.

The sum is taken in FP32 over 16 terms and in FP64 above, so on FP32 inputs
it is within 1e-6 (relative) of the exact FP64 sum of the same values; the
gradient is two FP32 roundings of 2 g w U (relative 2.4e-7 per part), BF16
scores one more rounding to BF16 (2^-8)."""
import ctypes

import numpy as np
import pytest

from oracle import os3d_oracle as O
from paper_1505_07690_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_SUM = 1e-6
TOL_GRAD = 3e-7
TOL_GRAD_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_07690_gb300 import build, os3d
    build.build()
    return os3d


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _score(shape, seed):
    rng = np.random.default_rng(seed)
    U = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    w = rng.uniform(0, 1, shape).astype(np.float32)
    return U, w


def _bf16_pair(U):
    """(re, im) BF16 tensor of U and the FP64 values it holds."""
    import torch
    t = torch.view_as_real(_cuda(U)).to(torch.bfloat16).contiguous()
    back = t.float().cpu().numpy().astype(np.float64)
    return t, back[..., 0] + 1j * back[..., 1]


@pytest.mark.parametrize("shape", [(42, 32, 32, 32), (3, 5, 7, 4), (1237 * 4,), (4,)])
@pytest.mark.parametrize("weighted", [True, False])
def test_energy_and_gradient_c64(M, shape, weighted):
    """Several grid strides of blocks and a ragged tail (1237 quads), a single
    quad; with and without weights."""
    import torch
    U, w = _score(shape, seed=11)
    Ut = _cuda(U)
    wt = _cuda(w) if weighted else None
    scratch = torch.empty(M.OS3D_ENERGY_SCRATCH_DOUBLES, dtype=torch.float64, device="cuda")
    loss = M.os3d_weighted_energy(Ut, wt, scratch=scratch)
    ref = O.weighted_energy(U.astype(np.complex128), w if weighted else None)
    torch.cuda.synchronize()
    assert abs(scratch[0].item() - ref) <= TOL_SUM * ref
    assert loss.item() == np.float32(scratch[0].item())
    g = torch.tensor(0.625, device="cuda")
    G = M.os3d_weighted_energy_grad(Ut, wt, g).cpu().numpy()
    Go = O.weighted_energy_grad(U, w if weighted else None, 0.625)
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(G) - part(Go)) <= TOL_GRAD * np.abs(part(Go)) + 1e-30)


def test_energy_bf16_scores(M):
    import torch
    U, w = _score((42, 16, 16, 16), seed=12)
    Ub, Uv = _bf16_pair(U)
    wt = _cuda(w)
    scratch = torch.empty(M.OS3D_ENERGY_SCRATCH_DOUBLES, dtype=torch.float64, device="cuda")
    M.os3d_weighted_energy(Ub, wt, scratch=scratch)
    ref = O.weighted_energy(Uv, w)
    assert abs(scratch[0].item() - ref) <= TOL_SUM * ref
    G = M.os3d_weighted_energy_grad(Ub, wt, torch.tensor(1.5, device="cuda")).float().cpu().numpy()
    Go = O.weighted_energy_grad(Uv, w, 1.5)
    assert np.all(np.abs(G[..., 0] - Go.real) <= TOL_GRAD_BF16 * np.abs(Go.real) + 1e-30)
    assert np.all(np.abs(G[..., 1] - Go.imag) <= TOL_GRAD_BF16 * np.abs(Go.imag) + 1e-30)


def test_energy_is_bit_identical_from_call_to_call_and_in_place_gradient(M):
    import torch
    U, w = _score((42, 24, 24, 24), seed=13)
    Ut, wt = _cuda(U), _cuda(w)
    scratch = torch.empty(M.OS3D_ENERGY_SCRATCH_DOUBLES, dtype=torch.float64, device="cuda")
    vals = set()
    for _ in range(5):
        M.os3d_weighted_energy(Ut, wt, scratch=scratch)
        vals.add(scratch[0].item())
    assert len(vals) == 1
    G = M.os3d_weighted_energy_grad(Ut, wt)
    M.os3d_weighted_energy_grad(Ut, wt, out=Ut)
    assert torch.equal(G, Ut)


def test_energy_edge_cases_and_errors(M):
    import torch
    from paper_1505_07690_gb300.os3d import lib
    scratch = torch.full((M.OS3D_ENERGY_SCRATCH_DOUBLES,), 7.0, dtype=torch.float64, device="cuda")
    empty = torch.empty(0, dtype=torch.complex64, device="cuda")
    assert M.os3d_weighted_energy(empty, scratch=scratch).item() == 0.0
    assert scratch[0].item() == 0.0
    U = torch.zeros(8, dtype=torch.complex64, device="cuda")
    vp = ctypes.c_void_p
    p = vp(U.data_ptr())
    s = vp(scratch.data_ptr())
    assert lib().os3d_weighted_energy(p, vp(None), 0, 6, s, vp(None), vp(None)) != 0     # count % 4
    assert lib().os3d_weighted_energy(vp(U.data_ptr() + 8), vp(None), 0, 4, s, vp(None),
                                      vp(None)) != 0                                   # alignment
    assert lib().os3d_weighted_energy(p, vp(None), 0, 4, vp(None), vp(None), vp(None)) != 0
    assert lib().os3d_weighted_energy(p, vp(None), 5, 4, s, vp(None), vp(None)) != 0     # udtype
    assert lib().os3d_weighted_energy_grad(p, vp(None), 0, 4, vp(None), p, vp(None)) != 0  # no g
    with pytest.raises(ValueError):
        M.os3d_weighted_energy(U, torch.ones(7, device="cuda"))
    torch.cuda.synchronize()


def test_energy_of_a_transform_is_parseval_with_M(M):
    """sum_i sum_x |(W f)_i|^2 = (1/n^3) sum_w M |f_hat|^2 (Sec. 2: norm
    preservation when M = 1), GPU transform and GPU energy against the oracle's
    M and DFT, 64^3 spline tubes, 42 orientations."""
    import torch
    dims = (64, 64, 64)
    f = synth.workload_volume("splines96x8_no42")[16:80, 16:80, 16:80].copy()
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(1), M.os3d_default_params(L=16))
    U = M.os3d_forward(bank, _cuda(f)[None])
    e = M.os3d_weighted_energy(U).item()
    ob = O.Bank(dims, O.icosa_orientations(1), O.Params(L=16))
    ref = float(np.sum(ob.M() * np.abs(np.fft.fftn(f.astype(np.float64))) ** 2) / np.prod(dims))
    torch.cuda.synchronize()
    assert abs(e - ref) <= 2e-5 * ref


def test_energy_at_the_differentiation_workload_size(M):
    """8 x 42 x 96^3 (2.4 GB of score), the launch configuration the benchmark
    times: the FP64 sum equals the FP64 sum of the same FP32 values (taken on
    the device in float64 by torch, a plain restatement of the definition),
    and sampled gradient elements equal 2 g w U."""
    import torch
    shape = (8, 42, 96, 96, 96)
    gen = torch.Generator("cuda").manual_seed(5)
    U = torch.randn(shape, dtype=torch.complex64, device="cuda", generator=gen)
    w = torch.rand(shape, device="cuda", generator=gen)
    scratch = torch.empty(M.OS3D_ENERGY_SCRATCH_DOUBLES, dtype=torch.float64, device="cuda")
    M.os3d_weighted_energy(U, w, scratch=scratch)
    ref = float((w.double() * (U.real.double() ** 2 + U.imag.double() ** 2)).sum())
    assert abs(scratch[0].item() - ref) <= TOL_SUM * ref
    g = torch.tensor(0.3, device="cuda")
    G = M.os3d_weighted_energy_grad(U, w, g)
    idx = torch.randint(0, U.numel(), (4096,), device="cuda", generator=gen)
    Us = U.reshape(-1)[idx].cpu().numpy()
    ws = w.reshape(-1)[idx].cpu().numpy()
    Gs = G.reshape(-1)[idx].cpu().numpy()
    Go = O.weighted_energy_grad(Us, ws, 0.3)
    assert np.all(np.abs(Gs - Go) <= TOL_GRAD * np.abs(Go) * 2 + 1e-30)
    del U, w, G
    torch.cuda.empty_cache()


def test_fused_loss_autograd_matches_oracle(M):
    """f -> orientation_score -> weighted_energy -> backward on a 32^3 tube
    volume with 42 orientations: the loss equals the oracle's energy of the
    oracle's score and the gradient its Re W^*(2 w U) (relative L2 <= 1e-5)."""
    import torch
    from paper_1505_07690_gb300.autograd import orientation_score, weighted_energy
    dims = (32, 32, 32)
    f = synth.workload_volume("tubes32_no42")
    w = synth.score_weights((42,) + dims, seed=2)
    bank = M.os3d_make_wavelets(dims, M.os3d_icosa_orientations(1), M.os3d_default_params(L=12))
    ft = _cuda(f).requires_grad_(True)
    loss = weighted_energy(orientation_score(ft, bank), _cuda(w))
    loss.backward()
    ob = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    Uo = O.forward(f, ob)
    Lo = O.weighted_energy(Uo, w)
    go = O.adjoint(O.weighted_energy_grad(Uo, w), ob)
    g = ft.grad.cpu().numpy()
    assert abs(loss.item() - Lo) <= 2e-5 * Lo
    assert float(np.linalg.norm(g - go) / np.linalg.norm(go)) <= 1e-5
    with pytest.raises(ValueError):
        weighted_energy(orientation_score(ft, bank), _cuda(w).requires_grad_(True))


# ---------------------------------------------------------------------------
# weighted adjoint Re W^*(2 g w U): the gradient folded into the plane pass
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,L,nvol", [((32, 32, 32), 12, 2), ((16, 128, 160), 12, 2),
                                         ((16, 256, 256), 12, 1), ((48, 48, 48), 16, 2)])
def test_weighted_adjoint_against_oracle(M, dims, L, nvol):
    """Whole-plane, rectangular (128 x 160) and 8-CTA-cluster (256^2) plane
    passes; arbitrary scores (not ranges of W), g = 0.7."""
    import torch
    V = M.os3d_icosa_orientations(1)
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=L))
    shape = (nvol, len(V)) + dims
    U, w = _score(shape, seed=21)
    g = torch.tensor(0.7, device="cuda")
    Ut, wt = _cuda(U), _cuda(w)
    got = M.os3d_adjoint_weighted(bank, Ut, wt, g).cpu().numpy()
    two = M.os3d_adjoint(bank, M.os3d_weighted_energy_grad(Ut, wt, g)).cpu().numpy()
    ob = O.Bank(dims, O.icosa_orientations(1), O.Params(L=L))
    for v in range(nvol):
        ref = O.adjoint(O.weighted_energy_grad(U[v], w[v], 0.7), ob)
        assert float(np.linalg.norm(got[v] - ref) / np.linalg.norm(ref)) <= 1e-5, v
        assert np.abs(got[v] - ref).max() <= 2e-5 * np.abs(ref).max(), v
        assert float(np.linalg.norm(got[v] - two[v]) / np.linalg.norm(two[v])) <= 2e-6, v


def test_weighted_adjoint_unpaired_orientations(M):
    """21 orientations without their antipodes (each slot loads w_a U_a alone),
    blocks of 4 slots, two volumes."""
    import torch
    dims = (32, 32, 32)
    V = O.icosa_orientations(1)[:21].copy()
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=12, block_slots=4))
    U, w = _score((2, 21) + dims, seed=24)
    got = M.os3d_adjoint_weighted(bank, _cuda(U), _cuda(w), torch.tensor(1.3, device="cuda"))
    got = got.cpu().numpy()
    ob = O.Bank(dims, V, O.Params(L=12))
    for v in range(2):
        ref = O.adjoint(O.weighted_energy_grad(U[v], w[v], 1.3), ob)
        assert float(np.linalg.norm(got[v] - ref) / np.linalg.norm(ref)) <= 1e-5, v


def test_weighted_adjoint_unsupported_forms_and_score_energy_fallback(M):
    """BF16 scores and planes without a plane pass (32 x 48 x 64 runs pencil
    passes) answer EUNSUPPORTED; score_energy then stores G = 2 g w U and
    takes os3d_adjoint, with the same gradient as the oracle."""
    import torch
    from paper_1505_07690_gb300.autograd import score_energy
    dims = (32, 48, 64)
    V = M.os3d_icosa_orientations(1)
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=12))
    U, w = _score((1, len(V)) + dims, seed=22)
    with pytest.raises(M.OS3DError) as e:
        M.os3d_adjoint_weighted(bank, _cuda(U), _cuda(w))
    assert e.value.status == M.OS3D_EUNSUPPORTED
    bank32 = M.os3d_make_wavelets((32, 32, 32), V, M.os3d_default_params(L=12))
    Ub, _ = _bf16_pair(_score((1, len(V), 32, 32, 32), seed=23)[0])
    with pytest.raises(M.OS3DError) as e:
        M.os3d_adjoint_weighted(bank32, Ub, _cuda(np.ones((len(V), 32, 32, 32), np.float32)))
    assert e.value.status == M.OS3D_EUNSUPPORTED
    f = synth.workload_volume("splines96x8_no42")[:32, :48, :64].copy()
    wf = synth.score_weights((len(V),) + dims, seed=3)
    ft = _cuda(f).requires_grad_(True)
    loss = score_energy(ft, bank, _cuda(wf))
    loss.backward()
    ob = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    Uo = O.forward(f, ob)
    go = O.adjoint(O.weighted_energy_grad(Uo, wf), ob)
    g = ft.grad.cpu().numpy()
    assert float(np.linalg.norm(g - go) / np.linalg.norm(go)) <= 1e-5
    assert abs(loss.item() - O.weighted_energy(Uo, wf)) <= 2e-5 * O.weighted_energy(Uo, wf)


def test_score_energy_matches_the_composition_bit_for_bit_in_the_loss(M):
    """score_energy(f) and weighted_energy(orientation_score(f)) give the same
    loss bits (the same kernels) and gradients within FP32 rounding of each
    other (the weighting applied in the load instead of a stored G)."""
    import torch
    from paper_1505_07690_gb300.autograd import orientation_score, score_energy, weighted_energy
    dims = (64, 64, 64)
    V = M.os3d_icosa_orientations(1)
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=16))
    f = np.stack([synth.workload_volume("splines96x8_no42", batch_index=b)[16:80, 16:80, 16:80]
                  for b in range(2)]).copy()
    w = _cuda(synth.score_weights((2, len(V)) + dims, seed=4))
    ft = _cuda(f).requires_grad_(True)
    l1 = score_energy(ft, bank, w)
    l1.backward()
    g1 = ft.grad.clone()
    ft.grad = None
    l2 = weighted_energy(orientation_score(ft, bank), w)
    l2.backward()
    assert l1.item() == l2.item()
    rel = float(torch.linalg.vector_norm(g1 - ft.grad) / torch.linalg.vector_norm(ft.grad))
    assert rel <= 2e-6


# ---------------------------------------------------------------------------
# one sweep: L = sum w |W f|^2 and Re W^*(2 g w W f) without a stored score
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,subdiv,L,nvol,kw", [
    ((32, 32, 32), 1, 12, 2, {}),
    ((16, 128, 128), 1, 12, 1, {}),
    ((48, 48, 48), 1, 16, 1, {"block_slots": 3}),
    ((32, 32, 32), 1, 12, 2, {"block_slots": 8, "overlap": 0}),
    ((16, 16, 16), 2, 8, 1, {}),
    ((16, 256, 256), 1, 12, 1, {}),
    ((16, 128, 160), 1, 12, 2, {}),
])
def test_score_energy_sweep_against_oracle(M, dims, subdiv, L, nvol, kw):
    """Paired sets in several block sizes, with and without the two-stream
    overlap, 162 orientations on 16^3, batch 2, 256^2 planes on 8-CTA clusters
    and 128 x 160 planes; g = 0.8."""
    import torch
    V = M.os3d_icosa_orientations(subdiv)
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=L, **kw))
    f = np.stack([synth.spline_tubes(dims, 4, seed=70 + v) for v in range(nvol)])
    w = synth.score_weights((nvol, len(V)) + dims, seed=7)
    g = torch.tensor(0.8, device="cuda")
    loss, grad = M.os3d_score_energy_grad(bank, _cuda(f), _cuda(w), g)
    grad = grad.cpu().numpy()
    ob = O.Bank(dims, O.icosa_orientations(subdiv), O.Params(L=L))
    L_ref = 0.0
    for v in range(nvol):
        Uo = O.forward(f[v], ob)
        L_ref += O.weighted_energy(Uo, w[v])
        ref = O.adjoint(O.weighted_energy_grad(Uo, w[v], 0.8), ob)
        assert float(np.linalg.norm(grad[v] - ref) / np.linalg.norm(ref)) <= 1e-5, v
        assert np.abs(grad[v] - ref).max() <= 2e-5 * np.abs(ref).max(), v
    assert abs(loss.item() - L_ref) <= 2e-5 * L_ref


def test_score_energy_sweep_unpaired_orientations(M):
    """21 orientations without their antipodes: weight w_a alone per slot."""
    dims = (32, 32, 32)
    V = O.icosa_orientations(1)[:21].copy()
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=12, block_slots=4))
    f = synth.spline_tubes(dims, 4, seed=75)
    w = synth.score_weights((21,) + dims, seed=8)
    loss, grad = M.os3d_score_energy_grad(bank, _cuda(f), _cuda(w))
    ob = O.Bank(dims, V, O.Params(L=12))
    Uo = O.forward(f, ob)
    ref = O.adjoint(O.weighted_energy_grad(Uo, w), ob)
    g = grad.cpu().numpy()
    assert float(np.linalg.norm(g - ref) / np.linalg.norm(ref)) <= 1e-5
    Lo = O.weighted_energy(Uo, w)
    assert abs(loss.item() - Lo) <= 2e-5 * Lo


def test_score_energy_sweep_repeatable_and_autograd(M):
    """Bit-identical loss and gradient from call to call; the autograd Function
    on the sweep equals its stored-score form (sweep=False) within FP32
    rounding, the loss within the FP32 rounding of the two summation orders."""
    import torch
    from paper_1505_07690_gb300.autograd import score_energy
    dims = (64, 64, 64)
    V = M.os3d_icosa_orientations(1)
    bank = M.os3d_make_wavelets(dims, V, M.os3d_default_params(L=16))
    f = _cuda(np.stack([synth.spline_tubes(dims, 5, seed=80 + v) for v in range(2)]))
    w = _cuda(synth.score_weights((2, len(V)) + dims, seed=9))
    scratch = torch.empty(M.os3d_score_energy_scratch(bank, 2), dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(3):
        loss, grad = M.os3d_score_energy_grad(bank, f, w, scratch=scratch)
        outs.append((scratch[0].item(), grad.clone()))
    assert all(o[0] == outs[0][0] for o in outs)
    assert all(torch.equal(o[1], outs[0][1]) for o in outs)
    assert M.os3d_score_energy_scratch(bank, 2) == 1 + 2 * 21 * 64
    ft = f.clone().requires_grad_(True)
    l1 = score_energy(ft, bank, w)
    (3.0 * l1).backward()
    g1 = ft.grad.clone()
    ft.grad = None
    l2 = score_energy(ft, bank, w, sweep=False)
    (3.0 * l2).backward()
    assert abs(l1.item() - l2.item()) <= 1e-6 * abs(l2.item())
    assert float(torch.linalg.vector_norm(g1 - ft.grad) / torch.linalg.vector_norm(ft.grad)) <= 2e-6
    assert torch.allclose(g1, 3.0 * outs[0][1], rtol=1e-6, atol=0)
    with torch.no_grad():   # the loss alone takes the transform and the energy kernel
        assert score_energy(f, bank, w).item() == l2.item()


def test_score_energy_sweep_rejections(M):
    import torch
    V = M.os3d_icosa_orientations(1)
    bank = M.os3d_make_wavelets((32, 48, 64), V, M.os3d_default_params(L=12))
    f = torch.zeros((32, 48, 64), device="cuda")
    w = torch.zeros((42, 32, 48, 64), device="cuda")
    with pytest.raises(M.OS3DError) as e:
        M.os3d_score_energy_grad(bank, f, w)
    assert e.value.status == M.OS3D_EUNSUPPORTED
    bank = M.os3d_make_wavelets((32, 32, 32), V, M.os3d_default_params(L=12))
    f = torch.zeros((32, 32, 32), device="cuda")
    w = torch.zeros((42, 32, 32, 32), device="cuda")
    small = torch.empty(10, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    st = M.lib().os3d_score_energy_grad(bank.handle, vp(f.data_ptr()), vp(w.data_ptr()), vp(None),
                                        1, vp(None), vp(f.data_ptr()), vp(small.data_ptr()), 10,
                                        vp(None), vp(None))
    assert st == 1   # scratch smaller than os3d_score_energy_scratch
    x = torch.arange(7, dtype=torch.float32, device="cuda")
    y = M.os3d_scale_by(x, torch.tensor(-2.0, device="cuda"))
    assert torch.equal(y, -2.0 * x)
