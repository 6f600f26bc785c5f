"""GPU parity of the extensions through the C ABI against the FP64 oracle:
the plate-detector profile, the octahedral orientation sets, the approximate
reconstruction, the projection P_psi, the soft threshold, the fused
Upsilon = W^{*,ext} Phi W and the linear left-invariant diffusion. Tolerances as in test_gpu_parity.py: relative L2
error <= 1e-5 for FP32 results, 5e-3 where a score is stored in BF16."""
import numpy as np
import pytest

from oracle import os3d_oracle as O
from paper_1505_07690_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_BF16 = 5e-3


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_07690_gb300 import build, os3d
    build.build()
    return os3d


def _pair(M, dims, V, **kw):
    p = M.os3d_default_params(**kw)
    bank = M.os3d_make_wavelets(dims, V, p)
    ob = O.Bank(dims, V, O.Params(k=p.k, s_theta=p.s_theta, L=p.L, N=p.N, gamma=p.gamma,
                                  eps=p.eps, fit_mode=p.fit_mode, profile=p.profile))
    return bank, ob


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _c64(U):
    return _cuda(np.asarray(U).astype(np.complex64))


# ---------------------------------------------------------------------------
# wavelet variants (Sec. 3.1 plate detector, Sec. 2.1 octahedral sampling)
# ---------------------------------------------------------------------------
def test_plate_profile_fig3_parameters(M):
    """h = A with the parameters of Fig. 3 (L = 16, s_theta = 0.6, k = 2,
    N = 20, gamma = 0.8; the clamp binds near rho_N)."""
    dims = (32, 32, 32)
    V = O.icosa_orientations(1)
    bank, ob = _pair(M, dims, V, profile=1, L=16, s_theta=0.6, N=20, gamma=0.8)
    b, c = M.os3d_bank_coefficients(bank)
    assert np.abs(c - ob.c).max() <= 1e-10 * np.abs(ob.c).max()
    f = synth.straight_tubes(dims, 3, seed=21)
    U = M.os3d_forward(bank, _cuda(f))
    Uo = O.forward(f, ob)
    assert rel(_np(U)[0], Uo) <= TOL
    assert rel(_np(M.os3d_inverse(bank, U))[0], O.inverse(Uo, ob)) <= TOL


@pytest.mark.parametrize("dims,subdiv", [((32, 32, 32), 1), ((16, 16, 16), 2), ((32, 48, 64), 1)])
def test_octahedral_sets(M, dims, subdiv):
    V = O.octa_orientations(subdiv)
    assert np.abs(M.os3d_octa_orientations(subdiv) - V).max() < 1e-12
    bank, ob = _pair(M, dims, V, L=12, block_slots=4)
    f = synth.straight_tubes(dims, 2, seed=22, noise=0.1)
    U = M.os3d_forward(bank, _cuda(f))
    Uo = O.forward(f, ob)
    assert rel(_np(U)[0], Uo) <= TOL
    assert rel(_np(M.os3d_inverse(bank, U))[0], O.inverse(Uo, ob)) <= TOL


# ---------------------------------------------------------------------------
# approximate reconstruction and projection
# ---------------------------------------------------------------------------
def test_approximate_reconstruction(M):
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, O.icosa_orientations(1), L=12)
    rng = np.random.default_rng(23)
    G = (rng.standard_normal((2, 42) + dims) + 1j * rng.standard_normal((2, 42) + dims))
    fa = _np(M.os3d_approx_reconstruct(bank, _c64(G)))
    for v in range(2):
        assert rel(fa[v], O.approx_reconstruct(G[v].astype(np.complex64).astype(np.complex128), ob)) <= TOL
    # on a score of an image, and from BF16 storage
    f = synth.workload_volume("tubes32_no42")
    Uo = O.forward(f, ob)
    ref = O.approx_reconstruct(Uo, ob)
    Ub = M.os3d_forward(bank, _cuda(f), bf16=True)
    assert rel(_np(M.os3d_approx_reconstruct(bank, M.os3d_forward(bank, _cuda(f))))[0], ref) <= TOL
    assert rel(_np(M.os3d_approx_reconstruct(bank, Ub))[0], ref) <= TOL_BF16


def test_approximate_reconstruction_162_orientations(M):
    dims = (64, 64, 64)
    bank, ob = _pair(M, dims, O.icosa_orientations(2), L=16)
    f = synth.spline_tubes(dims, 6, seed=24)
    U = M.os3d_forward(bank, _cuda(f))
    Uo = O.forward(f, ob)
    assert rel(_np(M.os3d_approx_reconstruct(bank, U))[0], O.approx_reconstruct(Uo, ob)) <= TOL


@pytest.mark.parametrize("dims", [(32, 32, 32), (32, 48, 64)])
def test_projection(M, dims):
    bank, ob = _pair(M, dims, O.icosa_orientations(1), L=12, block_slots=4)
    rng = np.random.default_rng(25)
    G = (rng.standard_normal((1, 42) + dims) + 1j * rng.standard_normal((1, 42) + dims))
    G = G.astype(np.complex64)
    Gd = _cuda(G)
    P = _np(M.os3d_project(bank, Gd))[0]
    Po = O.project(G[0].astype(np.complex128), ob)
    assert rel(P, Po) <= TOL
    # in place
    M.os3d_project(bank, Gd, U_out=Gd)
    assert rel(_np(Gd)[0], Po) <= TOL


# ---------------------------------------------------------------------------
# soft threshold and Upsilon (Sec. 4.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("power", [1.5, 2.0, 0.7])
def test_soft_threshold(M, power):
    import torch
    rng = np.random.default_rng(26)
    U = (rng.standard_normal((3, 7, 16)) + 1j * rng.standard_normal((3, 7, 16))).astype(np.complex64)
    out = _np(M.os3d_soft_threshold(_cuda(U), power))
    ref = O.soft_threshold(U.astype(np.complex128), power)
    assert rel(out, ref) <= 1e-6
    # bf16 storage, in place
    Ub = torch.view_as_real(_cuda(U)).to(torch.bfloat16).contiguous()
    Ur = Ub.float().cpu().numpy()
    M.os3d_soft_threshold(Ub, power, out=Ub)
    got = Ub.float().cpu().numpy()
    exp = O.soft_threshold(Ur[..., 0] + 1j * Ur[..., 1], power)
    assert rel(got[..., 0] + 1j * got[..., 1], exp) <= TOL_BF16


def _upsilon_check(M, dims, V, f, power=1.5, **kw):
    bank, ob = _pair(M, dims, V, **kw)
    fu = _np(M.os3d_upsilon(bank, _cuda(f), power))
    fb = f if f.ndim == 4 else f[None]
    for v in range(fb.shape[0]):
        assert rel(fu[v] if fu.ndim == 4 else fu, O.upsilon(fb[v], ob, power)) <= TOL
    return bank, ob, fu


def test_upsilon_cluster_path(M):
    dims = (32, 32, 32)
    f = synth.workload_volume("tubes32_no42")
    _upsilon_check(M, dims, O.icosa_orientations(1), f, L=12)


@pytest.mark.parametrize("bs,overlap", [(3, 1), (8, 0)])
def test_upsilon_blocks_and_batch(M, bs, overlap):
    dims = (32, 32, 32)
    f = np.stack([synth.straight_tubes(dims, 3, seed=s) for s in (27, 28)])
    _upsilon_check(M, dims, O.icosa_orientations(1), f, L=12, block_slots=bs, overlap=overlap)


def test_upsilon_unpaired_and_pencil_grid(M):
    """Orientations without antipodes (scale 1) on a grid that takes the
    pencil passes and the separate soft-threshold kernel."""
    dims = (32, 48, 64)
    V = O.icosa_orientations(1)[:21].copy()
    f = synth.straight_tubes(dims, 3, seed=29)
    _upsilon_check(M, dims, V, f, L=12, block_slots=4)


@pytest.mark.parametrize("dims", [(16, 256, 256), (16, 128, 160)])
def test_upsilon_cluster_and_rectangular_planes(M, dims):
    """The fused score-domain plane kernel on 8-CTA clusters (256^2 planes,
    exchanges through distributed shared memory) and on 128 x 160 planes (the
    y direction's last pass of columns partial), against the oracle, p = 1.5."""
    f = synth.straight_tubes(dims, 3, seed=31)
    _upsilon_check(M, dims, O.icosa_orientations(1), f, L=12)


def test_upsilon_equals_the_composition(M):
    """Fused Upsilon = os3d_forward, os3d_soft_threshold, os3d_inverse."""
    dims = (64, 64, 64)
    bank, ob = _pair(M, dims, O.icosa_orientations(2), L=16)
    f = _cuda(synth.spline_tubes(dims, 6, seed=30))
    fu = _np(M.os3d_upsilon(bank, f, 1.5))
    U = M.os3d_forward(bank, f)
    M.os3d_soft_threshold(U, 1.5, out=U)
    fc = _np(M.os3d_inverse(bank, U))
    assert rel(fu, fc) <= TOL


def test_upsilon_64_cubed_162_orientations_p15(M):
    """The fused Upsilon with p = 1.5 on the whole 64^3 x 162 grid (the
    162-orientation set, 81 pairs in blocks of 11) against the oracle's
    W^{*,ext} Phi W f, element by element."""
    dims = (64, 64, 64)
    f = synth.spline_tubes(dims, 6, seed=62, noise=0.2)
    bank, _ = _pair(M, dims, M.os3d_icosa_orientations(2), L=16)
    fu = _np(M.os3d_upsilon(bank, _cuda(f), 1.5))
    from _oracle_pool import oracle_map, upsilon_of
    ref = oracle_map(upsilon_of, [(f, dims, 2, 16, 1.5)])[0]
    assert rel(fu, ref) <= TOL
    assert np.abs(fu - ref).max() <= 2e-5 * np.abs(ref).max()


def test_upsilon_headline_size_properties(M):
    """128^3 spline tubes, 162 orientations, L = 16 (the benchmark's grid):
    with p = 1 Upsilon is exactly the ball projection IDFT[1_ball f_hat];
    with p = 1.5 it is positively homogeneous of degree 1.5 and odd."""
    dims = (128, 128, 128)
    f = synth.workload_volume("splines128_no162")
    bank, ob = _pair(M, dims, O.icosa_orientations(2), L=16)
    fd = _cuda(f)
    wz, wy, wx = O.freq_grid(dims)
    ball = np.sqrt(wz ** 2 + wy ** 2 + wx ** 2) < np.pi
    fb = np.fft.ifftn(np.fft.fftn(f.astype(np.float64)) * ball).real
    assert rel(_np(M.os3d_upsilon(bank, fd, 1.0)), fb) <= TOL
    u = _np(M.os3d_upsilon(bank, fd, 1.5))
    assert rel(_np(M.os3d_upsilon(bank, 4.0 * fd, 1.5)), 8.0 * u) <= TOL
    assert rel(_np(M.os3d_upsilon(bank, -fd, 1.5)), -u) <= TOL


# ---------------------------------------------------------------------------
# linear left-invariant diffusion (Sec. 4.1)
# ---------------------------------------------------------------------------
def _diff(M, **kw):
    d = M.os3d_default_diffusion(**kw)
    return d, O.Diffusion(t=d.t, steps=d.steps, D11=d.D11, D33=d.D33, D44=d.D44,
                          sh_degree=d.sh_degree)


def _icosa42_plus_two_pairs(seed):
    """The 42 set and two seeded random directions with their antipodes (46)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((2, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return np.vstack([O.icosa_orientations(1), u, -u])


# the orientation counts 6, 12, 18, 42, 46 and 66 reach every row layout of the
# diffusion kernel (8, 12, 24, 42, 48 and 72 propagator rows)
@pytest.mark.parametrize("make,sub,dims,kw", [
    (O.icosa_orientations, 1, (32, 32, 32), {}),
    (O.octa_orientations, 0, (16, 16, 16), dict(t=2.0, steps=2, D44=0.1)),
    (_icosa42_plus_two_pairs, 5, (16, 16, 16), dict(t=3.0, steps=3, D44=0.05)),
    (O.icosa_orientations, 1, (32, 32, 32), dict(t=2.0, steps=3, D11=0.2, D33=1.0, D44=0.1)),
    (O.octa_orientations, 1, (32, 32, 32), dict(t=4.0, steps=5, D11=0.05, D33=0.5, D44=0.2)),
    (O.icosa_orientations, 0, (16, 16, 16), dict(D44=0.3)),
    (O.octa_orientations, 2, (16, 16, 16), dict(t=3.0, steps=4, D44=0.05)),
    (O.icosa_orientations, 1, (32, 48, 64), dict(t=5.0, steps=6, D11=0.1)),
])
def test_enhance_linear_against_oracle(M, make, sub, dims, kw):
    V = make(sub)
    bank, ob = _pair(M, dims, V, L=12)
    d, od = _diff(M, **kw)
    f = synth.straight_tubes(dims, 3, seed=40, noise=0.1)
    g = _np(M.os3d_enhance_linear(bank, _cuda(f), d))
    assert rel(g, O.enhance_linear(f, ob, od)) <= TOL


def test_enhance_linear_batch_and_identity(M):
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, O.icosa_orientations(1), L=12)
    f = np.stack([synth.straight_tubes(dims, 3, seed=s) for s in (41, 42)])
    d, od = _diff(M, t=3.0, steps=4, D11=0.1, D44=0.05)
    g = _np(M.os3d_enhance_linear(bank, _cuda(f), d))
    for v in range(2):
        assert rel(g[v], O.enhance_linear(f[v], ob, od)) <= TOL
    # t = 0: the ball projection IDFT[1_ball f_hat]
    d0, _ = _diff(M, t=0.0, steps=1)
    wz, wy, wx = O.freq_grid(dims)
    ball = np.sqrt(wz ** 2 + wy ** 2 + wx ** 2) < np.pi
    fb = np.fft.ifftn(np.fft.fftn(f[0]) * ball).real
    assert rel(_np(M.os3d_enhance_linear(bank, _cuda(f[0]), d0)), fb) <= TOL


def _icosa162_minus(k):
    """The 162 set without its last k antipodal pairs (162 - 2k orientations)."""
    V = O.icosa_orientations(2)
    return np.vstack([V[:81 - k], V[81:162 - k]])


# more than 68 orientations: the propagator product on the tensor cores, every
# padded size of that kernel (96, 128, 176 rows) and both wavelet forms
@pytest.mark.parametrize("make,sub,dims,kw", [
    (O.icosa_orientations, 2, (32, 32, 32), {}),
    (O.icosa_orientations, 2, (32, 32, 32), dict(t=2.0, steps=3, D11=0.2, D33=1.0, D44=0.1)),
    (O.icosa_orientations, 2, (16, 32, 48), dict(t=5.0, steps=6, D11=0.1, D44=0.02)),
    (lambda k: _icosa162_minus(k), 20, (16, 16, 16), dict(t=2.0, steps=2, D44=0.2)),
    (lambda k: _icosa162_minus(k), 46, (16, 16, 16), dict(t=1.0, steps=5, D11=0.3, D33=0.6)),
])
def test_enhance_linear_tensor_cores_against_oracle(M, make, sub, dims, kw):
    V = make(sub)
    assert len(V) > 68
    bank, ob = _pair(M, dims, V, L=12)
    d, od = _diff(M, **kw)
    f = synth.straight_tubes(dims, 3, seed=43, noise=0.1)
    g = _np(M.os3d_enhance_linear(bank, _cuda(f), d))
    ref = O.enhance_linear(f, ob, od)
    assert rel(g, ref) <= TOL
    assert np.abs(g - ref).max() <= 2e-5 * np.abs(ref).max()
    assert bank.wait_errors() == 0


def test_enhance_linear_tensor_cores_batch_and_repeat(M):
    """Two volumes per call, two calls: bit-identical repeats (fixed
    accumulation order on the tensor cores) and parity for both volumes."""
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, O.icosa_orientations(2), L=16)
    f = np.stack([synth.spline_tubes(dims, 4, seed=s) for s in (44, 45)])
    d, od = _diff(M, t=3.0, steps=4, D11=0.1, D44=0.05)
    g1 = _np(M.os3d_enhance_linear(bank, _cuda(f), d))
    g2 = _np(M.os3d_enhance_linear(bank, _cuda(f), d))
    assert np.array_equal(g1, g2)
    for v in range(2):
        assert rel(g1[v], O.enhance_linear(f[v], ob, od)) <= TOL
    assert bank.wait_errors() == 0


def test_enhance_linear_rejects_large_orientation_sets(M):
    """Sets above 176 orientations (the 258-vector octahedral set) are not
    supported by either kernel."""
    bank, _ = _pair(M, (16, 16, 16), O.octa_orientations(3), L=8)
    with pytest.raises(M.OS3DError) as e:
        M.os3d_enhance_linear(bank, _cuda(np.zeros((16, 16, 16), np.float32)))
    assert e.value.status == 5
