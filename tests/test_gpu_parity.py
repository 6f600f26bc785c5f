"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs. Tolerance: relative L2 error <= 1e-5 for FP32 results
(complex64 scores, reconstructions, adjoints); BF16-stored scores <= 5e-3.
Beside the global norm, an element-wise bound: max |x_gpu - x_oracle| over
the array, relative to max |x_oracle|, <= 2e-5 for FP32 results (a few wrong
columns or one wrong plane would show as an O(1) value here while moving the
global norm little) and <= 1e-2 for BF16 storage (8-bit mantissa)."""
import numpy as np
import pytest

from oracle import os3d_oracle as O
from paper_1505_07690_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
TOL_BF16 = 5e-3
MAXTOL = 2e-5
MAXTOL_BF16 = 1e-2


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def maxrel(a, b):
    """max |a - b| relative to max |b| (element-wise)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def close(a, b, bf16=False):
    return (rel(a, b) <= (TOL_BF16 if bf16 else TOL)
            and maxrel(a, b) <= (MAXTOL_BF16 if bf16 else MAXTOL))


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_07690_gb300 import build, os3d
    build.build()
    return os3d


def _params(M, **kw):
    p = M.os3d_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _oracle_params(p):
    return O.Params(k=p.k, s_theta=p.s_theta, L=p.L, N=p.N, gamma=p.gamma, eps=p.eps,
                    fit_mode=p.fit_mode)


def _pair(M, dims, subdiv=1, orient=None, **kw):
    p = _params(M, **kw)
    Vg = M.os3d_icosa_orientations(subdiv) if orient is None else orient
    Vo = O.icosa_orientations(subdiv) if orient is None else orient
    bank = M.os3d_make_wavelets(dims, Vg, p)
    ob = O.Bank(dims, Vo, _oracle_params(p))
    return bank, ob


def _to_np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("fit_mode,L", [(1, 12), (0, 16), (1, 20)])
def test_coefficients_fp64(M, fit_mode, L):
    bank, ob = _pair(M, (16, 16, 16), fit_mode=fit_mode, L=L)
    b, c = M.os3d_bank_coefficients(bank)
    bo = O.fit_coefficients(ob.p)
    assert np.abs(b - bo).max() <= 1e-10 * np.abs(bo).max()
    assert np.abs(c - ob.c).max() <= 1e-10 * np.abs(ob.c).max()


def test_minv_fp64(M):
    bank, ob = _pair(M, (32, 32, 32), L=12)
    mi = _to_np(M.os3d_bank_minv(bank))
    assert rel(mi, ob.M_inv()) < 1e-6


@pytest.mark.parametrize("dims,paired", [((32, 48, 64), True), ((16, 16, 16), False),
                                         ((16, 32, 48), True)])
def test_minv_mirror_and_unpaired_sets(M, dims, paired):
    """For an antipodally closed set the bank computes M on half of the grid
    and writes it at w and -w: the table equals the oracle's and is symmetric
    bit for bit; a set without antipodes takes every frequency itself."""
    V = O.icosa_orientations(1)
    if not paired:
        V = V[:21].copy()
    bank, ob = _pair(M, dims, orient=V, L=12)
    mi = _to_np(M.os3d_bank_minv(bank))
    assert rel(mi, ob.M_inv()) < 1e-6 and maxrel(mi, ob.M_inv()) < 2e-6
    if paired:
        mirror = mi[(-np.arange(dims[0])) % dims[0]][:, (-np.arange(dims[1])) % dims[1]][
            :, :, (-np.arange(dims[2])) % dims[2]]
        assert np.array_equal(mi.view(np.uint32), mirror.view(np.uint32))


def _check_forward_inverse(M, dims, f, subdiv=1, orient=None, batch_oracle=True, **kw):
    bank, ob = _pair(M, dims, subdiv, orient, **kw)
    U = M.os3d_forward(bank, _cuda(f))
    Ug = _to_np(U)[0]
    Uo = O.forward(f, ob)
    assert rel(Ug, Uo) <= TOL and maxrel(Ug, Uo) <= MAXTOL
    fr = _to_np(M.os3d_inverse(bank, U))[0]
    fro = O.inverse(Uo, ob)
    assert rel(fr, fro) <= TOL and maxrel(fr, fro) <= MAXTOL
    return bank, ob, Uo


def test_forward_inverse_tubes32_no42(M):
    """32^3 straight-tube volume, 42 orientations, L = 12 (the parity workload)."""
    f = synth.workload_volume("tubes32_no42")
    _check_forward_inverse(M, (32, 32, 32), f, L=12)


@pytest.mark.parametrize("dims,subdiv,L,bs", [((16, 16, 16), 0, 8, 0), ((16, 16, 16), 1, 16, 4),
                                              ((48, 48, 48), 1, 16, 0), ((32, 32, 32), 2, 16, 3),
                                              ((64, 64, 64), 0, 16, 0)])
def test_forward_inverse_sizes(M, dims, subdiv, L, bs):
    f = synth.straight_tubes(dims, 2, seed=3, noise=0.1)
    _check_forward_inverse(M, dims, f, subdiv=subdiv, L=L, block_slots=bs)


@pytest.mark.parametrize("bs,subdiv", [(11, 1), (12, 1), (11, 2), (12, 2)])
def test_long_blocks(M, bs, subdiv):
    """Blocks of 11 (the automatic size) and 12 pairs (the limit): 21 pairs
    split 11 + 10 and 12 + 9, 81 pairs 7 x 11 + 4 and 6 x 12 + 9."""
    f = synth.straight_tubes((32, 32, 32), 3, seed=6, noise=0.1)
    _check_forward_inverse(M, (32, 32, 32), f, subdiv=subdiv, L=12, block_slots=bs)


def test_unpaired_orientations_and_ragged_blocks(M):
    """Orientations without antipodes take the single-orientation path; 21
    slots in blocks of 4 leave a ragged last block."""
    V = O.icosa_orientations(1)[:21].copy()
    f = synth.straight_tubes((32, 32, 32), 3, seed=4)
    _check_forward_inverse(M, (32, 32, 32), f, orient=V, L=12, block_slots=4)


def test_inverse_and_adjoint_of_arbitrary_scores(M):
    """Inputs that are not scores of any image: exercises the pair folding
    U_a + conj(U_b) for general U."""
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, L=12)
    rng = np.random.default_rng(7)
    G = (rng.standard_normal((1, 42) + dims) + 1j * rng.standard_normal((1, 42) + dims)).astype(np.complex64)
    Gd = _cuda(G)
    fr = _to_np(M.os3d_inverse(bank, Gd))[0]
    assert rel(fr, O.inverse(G[0].astype(np.complex128), ob)) <= TOL
    ga = _to_np(M.os3d_adjoint(bank, Gd))[0]
    assert rel(ga, O.adjoint(G[0].astype(np.complex128), ob)) <= TOL


@pytest.mark.parametrize("bs", [0, 1, 3])
def test_batch_of_two_repeated(M, bs):
    """Two volumes per call, three calls in a row on one bank (consecutive
    blocks run on two streams; a missing dependency shows up here)."""
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, L=12, block_slots=bs)
    f = np.stack([synth.straight_tubes(dims, 3, seed=s) for s in (11, 12)])
    Uo = [O.forward(f[b], ob) for b in range(2)]
    fo = [O.inverse(Uo[b], ob) for b in range(2)]
    fd = _cuda(f)
    for _ in range(3):
        U = M.os3d_forward(bank, fd)
        fr = M.os3d_inverse(bank, U)
        Ug, frg = _to_np(U), _to_np(fr)
        for b in range(2):
            assert rel(Ug[b], Uo[b]) <= TOL
            assert rel(frg[b], fo[b]) <= TOL


def test_bf16_storage(M):
    import torch
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, L=12)
    f = synth.workload_volume("tubes32_no42")
    Ub = M.os3d_forward(bank, _cuda(f), bf16=True)
    assert Ub.dtype == torch.bfloat16 and Ub.shape[-1] == 2
    Ug = _to_np(Ub.float())[0]
    Ug = Ug[..., 0] + 1j * Ug[..., 1]
    Uo = O.forward(f, ob)
    assert close(Ug, Uo, bf16=True)
    fr = _to_np(M.os3d_inverse(bank, Ub))[0]
    assert close(fr, O.inverse(Uo, ob), bf16=True)


def test_clamp_and_edge_parameters(M):
    """N = 20 (the figures' radial order): the eps clamp binds near rho_N."""
    dims = (32, 32, 32)
    f = synth.straight_tubes(dims, 3, seed=5)
    _check_forward_inverse(M, dims, f, L=16, N=20, gamma=0.85, s_theta=0.7)
    # eps above max M: the inverse equals the adjoint / eps
    bank, ob = _pair(M, dims, L=12, eps=50.0)
    U = M.os3d_forward(bank, _cuda(f))
    fi = _to_np(M.os3d_inverse(bank, U))[0]
    fa = _to_np(M.os3d_adjoint(bank, U))[0]
    assert rel(fi, fa / 50.0) <= TOL


def test_workspace_argument(M):
    import torch
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, L=12)
    f = synth.straight_tubes(dims, 3, seed=6)
    ws = torch.empty(bank.workspace_bytes, dtype=torch.uint8, device="cuda")
    U = M.os3d_forward(bank, _cuda(f), workspace=ws)
    Uo = O.forward(f, ob)
    assert rel(_to_np(U)[0], Uo) <= TOL
    fr = _to_np(M.os3d_inverse(bank, U, workspace=ws))[0]
    assert rel(fr, O.inverse(Uo, ob)) <= TOL


@pytest.mark.parametrize("bf16,bs,subdiv", [(False, 0, 1), (True, 0, 1), (False, 4, 2), (True, 3, 1)])
def test_plane_pass_128_squared(M, bf16, bs, subdiv):
    """128^2 planes take the whole-plane pass (one CTA holds a plane, no
    cluster): 32 x 128 x 128 against the oracle element by element, c64 and
    BF16 scores, full and ragged blocks, two calls in a row."""
    dims = (32, 128, 128)
    f = synth.spline_tubes(dims, 5, seed=63, noise=0.2)
    bank, ob = _pair(M, dims, subdiv, L=12, block_slots=bs)
    Uo = O.forward(f, ob)
    fo = O.inverse(Uo, ob)
    fd = _cuda(f)
    for _ in range(2):
        U = M.os3d_forward(bank, fd, bf16=bf16)
        Ug = _to_np(U.float())[0] if bf16 else _to_np(U)[0]
        if bf16:
            Ug = Ug[..., 0] + 1j * Ug[..., 1]
        assert close(Ug, Uo, bf16)
        assert close(_to_np(M.os3d_inverse(bank, U))[0], fo, bf16)


def test_headline_size_sampled(M):
    """128^3 spline tubes, 162 orientations, L = 16, in the benchmark's
    configuration: sampled orientations against the oracle one by one, and
    the reconstruction against the exactly known W^-1 W f = IDFT[1_ball f_hat]."""
    dims = (128, 128, 128)
    f = synth.workload_volume("splines128_no162")
    bank, ob = _pair(M, dims, subdiv=2, L=16)
    U = M.os3d_forward(bank, _cuda(f))
    fhat = np.fft.fftn(f.astype(np.float64))
    for i in (0, 37, 80, 81, 161):
        Ui = _to_np(U[0, i])
        assert close(Ui, O.forward_one(fhat, ob, i)), i
    fr = _to_np(M.os3d_inverse(bank, U))[0]
    wz, wy, wx = O.freq_grid(dims)
    ball = np.sqrt(wz ** 2 + wy ** 2 + wx ** 2) < np.pi
    fb = np.fft.ifftn(fhat * ball).real
    assert close(fr, fb)


@pytest.mark.parametrize("dims,subdiv", [((32, 48, 64), 1), ((32, 256, 16), 0), ((16, 160, 32), 1),
                                         ((256, 32, 32), 0)])
def test_pencil_path_grids(M, dims, subdiv):
    """Grids whose z-planes are not square planes of side <= 128 run the x and
    y directions as separate pencil passes (and 256 along any axis)."""
    f = synth.straight_tubes(dims, 2, seed=8, noise=0.1)
    _check_forward_inverse(M, dims, f, subdiv=subdiv, L=12, block_slots=4)


@pytest.mark.parametrize("bf16", [False, True])
def test_plane_pass_rectangular_128x160(M, bf16):
    """128 x 160 planes (the serving mix's 96 x 128 x 160 grid) take the
    whole-plane pass with a partial last pass of columns in the y direction;
    16 x 128 x 160 against the oracle element by element, ragged blocks."""
    dims = (16, 128, 160)
    f = synth.spline_tubes(dims, 4, seed=64, noise=0.2)
    bank, ob = _pair(M, dims, 1, L=12, block_slots=4)
    U = M.os3d_forward(bank, _cuda(f), bf16=bf16)
    Ug = _to_np(U.float())[0] if bf16 else _to_np(U)[0]
    if bf16:
        Ug = Ug[..., 0] + 1j * Ug[..., 1]
    Uo = O.forward(f, ob)
    assert close(Ug, Uo, bf16)
    assert close(_to_np(M.os3d_inverse(bank, U))[0], O.inverse(Uo, ob), bf16)


def test_precision_workload_sampled_c64_and_bf16(M):
    """256^3, 40 spline tubes, 42 orientations, L = 20: complex64 scores match
    the oracle on sampled orientations; both storage formats reconstruct
    W^-1 W f = IDFT[1_ball f_hat] (complex64 within 1e-5, bf16 within 5e-3)."""
    import torch
    dims = (256, 256, 256)
    f = synth.workload_volume("splines256_no42")
    bank, ob = _pair(M, dims, subdiv=1, L=20)
    fd = _cuda(f)
    fhat = np.fft.fftn(f.astype(np.float64))
    wz, wy, wx = O.freq_grid(dims)
    fb = np.fft.ifftn(fhat * (np.sqrt(wz ** 2 + wy ** 2 + wx ** 2) < np.pi)).real
    U = M.os3d_forward(bank, fd)
    for i in (0, 29):
        assert close(_to_np(U[0, i]), O.forward_one(fhat, ob, i)), i
    assert close(_to_np(M.os3d_inverse(bank, U))[0], fb)
    del U
    torch.cuda.empty_cache()
    Ub = M.os3d_forward(bank, fd, bf16=True)
    assert close(_to_np(M.os3d_inverse(bank, Ub))[0], fb, bf16=True)


def test_degenerate_orientation_sets(M):
    """One orientation (unpaired), and a single antipodal pair."""
    dims = (32, 32, 32)
    f = synth.straight_tubes(dims, 2, seed=51)
    V = O.icosa_orientations(1)
    _check_forward_inverse(M, dims, f, orient=V[:1].copy(), L=12)
    _check_forward_inverse(M, dims, f, orient=np.stack([V[0], V[21]]), L=12)


def test_degenerate_inputs(M):
    """A constant volume (only w = 0, where every psi_hat_i = c_0): every U_i
    is the constant c_0 f and the inverse returns f; the Nyquist checkerboard
    (-1)^(x+y+z) (only the corner |w| = sqrt(3) pi, outside the ball): U = 0
    and the inverse 0; the zero volume; a unit impulse against the oracle."""
    import torch
    dims = (32, 32, 32)
    V = M.os3d_icosa_orientations(1)
    bank = M.os3d_make_wavelets(dims, V, _params(M, L=12))
    _, c = M.os3d_bank_coefficients(bank)
    const = np.full(dims, 0.75, dtype=np.float32)
    U = _to_np(M.os3d_forward(bank, _cuda(const)))[0]
    assert np.abs(U - c[0] * 0.75).max() <= 2e-6 * abs(c[0] * 0.75)
    fr = _to_np(M.os3d_inverse(bank, _cuda(U[None])))[0]
    assert np.abs(fr - 0.75).max() <= 2e-6
    z, y, x = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    cb = ((-1.0) ** (z + y + x)).astype(np.float32)
    U = _to_np(M.os3d_forward(bank, _cuda(cb)))[0]
    assert np.abs(U).max() <= 1e-6
    assert np.abs(_to_np(M.os3d_inverse(bank, _cuda(U[None])))[0]).max() <= 1e-6
    zero = np.zeros(dims, dtype=np.float32)
    U = _to_np(M.os3d_forward(bank, _cuda(zero)))[0]
    assert not U.any()
    imp = np.zeros(dims, dtype=np.float32)
    imp[5, 17, 30] = 1.0
    _check_forward_inverse(M, dims, imp, L=12)
    torch.cuda.synchronize()


def test_isotropic_wavelet_closed_form(M):
    """L = 0: h is the constant c_0, so every psi_hat_i = c_0 G and
    U_i = IDFT[c_0 G f_hat] for all i, with c_0 = 1/sqrt(N_o) (the
    normalisation); the inverse returns IDFT[1_ball f_hat]. Checked against
    these closed forms, not the oracle."""
    dims = (32, 32, 32)
    f = synth.straight_tubes(dims, 3, seed=52)
    V = O.icosa_orientations(1)
    bank = M.os3d_make_wavelets(dims, V, _params(M, L=0))
    b, c = M.os3d_bank_coefficients(bank)
    assert abs(c[0] - 1.0 / np.sqrt(42.0)) < 1e-12
    U = _to_np(M.os3d_forward(bank, _cuda(f)))[0]
    fh = np.fft.fftn(f.astype(np.float64))
    G = O.radial_ball(dims, 8, 0.8)
    u0 = np.fft.ifftn(fh * G * c[0])
    for i in (0, 7, 41):
        assert rel(U[i], u0) <= TOL
    wz, wy, wx = O.freq_grid(dims)
    ball = np.sqrt(wz ** 2 + wy ** 2 + wx ** 2) < np.pi
    fr = _to_np(M.os3d_inverse(bank, _cuda(U[None])))[0]
    assert rel(fr, np.fft.ifftn(fh * ball).real) <= TOL


@pytest.mark.parametrize("kw", [dict(N=0, L=12), dict(L=32, fit_mode=0), dict(L=28, k=3, s_theta=0.5)])
def test_parameter_extremes(M, kw):
    """N = 0 (plain Gaussian window), L = 32 and L = 28 (Chebyshev evaluation
    of h), cubic B-spline profile."""
    dims = (32, 32, 32)
    f = synth.straight_tubes(dims, 3, seed=53)
    _check_forward_inverse(M, dims, f, **kw)


def test_batch_zero_is_rejected(M):
    dims = (16, 16, 16)
    bank, _ = _pair(M, dims, L=8)
    import ctypes
    L = M.lib()
    assert L.os3d_forward(bank.handle, ctypes.c_void_p(1), 0, ctypes.c_void_p(1), 0, None, None) == 1
    assert L.os3d_inverse(bank.handle, ctypes.c_void_p(1), 0, 0, ctypes.c_void_p(1), None, None) == 1


def test_plane_pass_256_squared(M):
    """256^2 planes: the forward score pass on four quarter-plane CTAs per
    plane (output rows folded modulo 4), the inverse on 8-CTA clusters (an
    eighth of a plane per CTA); 32 x 256 x 256 keeps the oracle fast."""
    dims = (32, 256, 256)
    f = synth.straight_tubes(dims, 3, seed=54, noise=0.1)
    _check_forward_inverse(M, dims, f, subdiv=0, L=12, block_slots=4)
    # Upsilon on this grid: the score-domain step takes the pencil passes
    bank, ob = _pair(M, dims, subdiv=0, L=12, block_slots=4)
    fu = _to_np(M.os3d_upsilon(bank, _cuda(f), 1.5))
    assert rel(fu, O.upsilon(f, ob, 1.5)) <= TOL


def test_quarter_plane_forward_unpaired_batch_and_bf16(M):
    """The quarter-plane forward pass of 256^2 planes with orientations that
    have no antipode (U_a only), a batch of two volumes and ragged blocks of 4
    slots, against the oracle; and with BF16 scores, against the oracle and
    against the complex64 scores of the same call."""
    import torch
    dims = (16, 256, 256)
    fs = [synth.straight_tubes(dims, 3, seed=s, noise=0.1) for s in (71, 72)]
    V = O.icosa_orientations(1)[:21].copy()
    bank, ob = _pair(M, dims, orient=V, L=12, block_slots=4)
    U = _to_np(M.os3d_forward(bank, torch.from_numpy(np.stack(fs)).cuda()))
    for v in range(2):
        assert close(U[v], O.forward(fs[v], ob)), v
    bank2, ob2 = _pair(M, dims, subdiv=0, L=12)
    fd = _cuda(fs[0])
    Uc = _to_np(M.os3d_forward(bank2, fd))[0]
    Ub = M.os3d_forward(bank2, fd, bf16=True).float().cpu().numpy()[0]
    Ub = Ub[..., 0] + 1j * Ub[..., 1]
    assert close(Uc, O.forward(fs[0], ob2))
    assert close(Ub, O.forward(fs[0], ob2), bf16=True)
    assert rel(Ub, Uc) <= 4e-3


def test_default_workspace_is_allocated_on_first_use(M):
    """A bank holds only its tables until a call passes no workspace; calls
    with a caller's workspace never allocate the bank's own. The allocation
    failing (injected on the host) is reported as ENOMEM."""
    import os
    import torch
    dims = (32, 32, 32)
    bank, ob = _pair(M, dims, L=12)
    tables = bank.resident_bytes()
    assert tables < bank.workspace_bytes
    f = synth.straight_tubes(dims, 3, seed=61)
    ws = torch.empty(bank.workspace_bytes, dtype=torch.uint8, device="cuda")
    U = M.os3d_forward(bank, _cuda(f), workspace=ws)
    M.os3d_inverse(bank, U, workspace=ws)
    torch.cuda.synchronize()
    assert bank.resident_bytes() == tables
    os.environ["OS3D_FAULT"] = "alloc_ws"
    try:
        with pytest.raises(M.OS3DError) as e:
            M.os3d_forward(bank, _cuda(f))
        assert e.value.status == 2
    finally:
        del os.environ["OS3D_FAULT"]
    assert bank.resident_bytes() == tables
    U2 = M.os3d_forward(bank, _cuda(f))
    assert bank.resident_bytes() == tables + bank.workspace_bytes
    assert close(_to_np(U2)[0], O.forward(f, ob))
    _, fp = bank.workspace_bytes, bank.footprint_bytes_per_volume
    assert fp == 8 * 42 * 32 ** 3 + 2 * 4 * 32 ** 3
