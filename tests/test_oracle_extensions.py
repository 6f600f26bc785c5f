"""Pins of the oracle's extensions: the octahedral orientation sets, the plate
detector profile, the approximate reconstruction, the projection P_psi, the
soft-threshold processing Upsilon and the linear left-invariant diffusion.
As in test_oracle_pins.py, each test checks the oracle against something
other than itself: a spherical design identity, grid rotations, the detector
semantics the paper states, harmonic polynomials, the heat kernel, the order
of the splitting and algebraic properties (fixed points, idempotence,
homogeneity)."""
import math

import numpy as np
import pytest

from oracle import os3d_oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------------------
# octahedral orientation sets (Sec. 2.1: platonic solids and tessellations)
# ---------------------------------------------------------------------------
def _rot_z90():
    return np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])


def _rot_x90():
    return np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def _act(R, f):
    """g(r) = f(R^T r) on a periodic cubic grid, array axes (z, y, x)."""
    n = f.shape[0]
    r = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    xyz = r[..., ::-1]                                  # (x, y, z) of every voxel
    src = np.einsum("ji,abcj->abci", R, xyz).round().astype(int) % n   # R^T r
    return f[src[..., 2], src[..., 1], src[..., 0]]


@pytest.mark.parametrize("subdiv,count", [(0, 6), (1, 18), (2, 66), (3, 258)])
def test_octahedral_sets(subdiv, count):
    V = O.octa_orientations(subdiv)
    assert V.shape == (count, 3)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    h = count // 2
    assert np.allclose(V[h:], -V[:h], atol=0)
    # closed under the 90-degree rotations about the axes (as sets)
    for R in (_rot_z90(), _rot_x90()):
        RV = V @ R.T
        d = np.abs(RV[:, None, :] - V[None, :, :]).max(-1)
        assert np.all(d.min(1) < 1e-12)
        assert len(set(np.argmin(d, 1))) == count


def test_channel_permutation_under_90_degree_rotations():
    """W[f o R^-1](x, R n) = W[f](R^-1 x, n): rotating the image by 90 degrees
    about an axis permutes the channels of the octahedral set and rotates
    each channel (exact on a cubic periodic grid with the ball limit)."""
    n = 12
    dims = (n, n, n)
    f = np.random.default_rng(31).standard_normal(dims)
    bank = O.Bank(dims, O.octa_orientations(1), O.Params(L=12))
    U = O.forward(f, bank)
    V = bank.orients
    for R in (_rot_z90(), _rot_x90()):
        g = _act(R, f)
        r = np.array([3, 1, 2])
        src = (R.T @ r).round().astype(int) % n
        assert g[r[2], r[1], r[0]] == f[src[2], src[1], src[0]]
        perm = [int(np.argmin(np.abs(V - rv).sum(1))) for rv in V @ R.T]
        U2 = O.forward(g, bank)
        for i in range(bank.n_o):
            assert np.allclose(U2[perm[i]], _act(R, U[i]), atol=1e-12)


# ---------------------------------------------------------------------------
# plate detector h = A versus the cake wavelet (Sec. 3.1, Fig. 3 and Fig. 4)
# ---------------------------------------------------------------------------
def _center_real_responses(f, bank):
    U = O.forward(f, bank)
    c = tuple(d // 2 for d in f.shape)
    return np.array([U[i][c].real for i in range(bank.n_o)])


def test_plate_and_line_detectors():
    """With h = A the real part detects plates perpendicular to n; after the
    Funk transform it detects lines along n."""
    n = 24
    dims = (n, n, n)
    z, y, x = np.meshgrid(*(np.arange(n) - n // 2,) * 3, indexing="ij")
    line_z = np.exp(-(x ** 2 + y ** 2) / (2 * 1.5 ** 2))
    plate_z = np.exp(-(z ** 2) / (2 * 1.5 ** 2))
    V = O.octa_orientations(1)
    ez = {0, len(V) // 2}                 # +e_z and -e_z in canonical order
    assert np.allclose(V[0], [0, 0, 1])
    cake = O.Bank(dims, V, O.Params(L=16, profile=0))
    plate = O.Bank(dims, V, O.Params(L=16, profile=1))
    assert int(np.argmax(_center_real_responses(line_z, cake))) in ez
    assert int(np.argmax(_center_real_responses(plate_z, plate))) in ez
    assert int(np.argmax(_center_real_responses(plate_z, cake))) not in ez
    assert int(np.argmax(_center_real_responses(line_z, plate))) not in ez


def test_plate_profile_coefficients_are_the_normalised_fit():
    p = O.Params(L=12, profile=1, fit_mode=0)
    b = O.fit_coefficients(p)
    c = O.wavelet_coefficients(p, 42)
    ratio = c / b
    assert np.allclose(ratio, ratio[0], rtol=1e-13)
    l = np.arange(13)
    assert abs(42 * np.sum(c * c / (2 * l + 1)) - 1.0) < 1e-13


# ---------------------------------------------------------------------------
# approximate reconstruction (Eq. Reconstruction2Approximation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L,exact", [(4, True), (5, True), (6, False)])
def test_approximate_reconstruction_on_a_spherical_5_design(L, exact):
    """The 12 icosahedron vertices form a spherical 5-design, so for L <= 5
    sum_i h(w.n_i) = N_o c_0 for every direction and the approximate
    reconstruction equals IDFT[ f_hat g 1_ball ] exactly; at L = 6 it does not."""
    dims = (10, 12, 8)
    f = np.random.default_rng(32).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(0), O.Params(L=L, fit_mode=0))
    U = O.forward(f, bank)
    fa = O.approx_reconstruct(U, bank)
    ref = np.fft.ifftn(np.fft.fftn(f) * O.radial_ball(dims, 8, 0.8)).real
    err = np.abs(fa - ref).max() / np.abs(ref).max()
    assert (err < 1e-13) == exact
    # the odd (edge) parts cancel over antipodal pairs: the sum is real
    assert np.abs(U.sum(0).imag).max() < 1e-13 * np.abs(U).max()


def test_approximate_reconstruction_keeps_the_mean():
    dims = (8, 8, 8)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=16))
    f = np.full(dims, 3.25)
    assert np.allclose(O.approx_reconstruct(O.forward(f, bank), bank), 3.25, atol=1e-13)


# ---------------------------------------------------------------------------
# projection P_psi = W W^{*,ext} (App. A, corollary)
# ---------------------------------------------------------------------------
def test_projection_fixes_scores_and_is_idempotent():
    dims = (10, 12, 8)
    rng = np.random.default_rng(33)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    f = rng.standard_normal(dims)
    U = O.forward(f, bank)
    assert np.abs(O.project(U, bank) - U).max() < 1e-13 * np.abs(U).max()
    G = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    P1 = O.project(G, bank)
    assert np.abs(O.project(P1, bank) - P1).max() < 1e-13 * np.abs(P1).max()
    # the projection of anything is the score of a real image: antipodes conjugate
    h = bank.n_o // 2
    assert np.abs(P1[h:] - np.conj(P1[:h])).max() < 1e-13 * np.abs(P1).max()
    assert np.abs(P1 - G).max() > 0.1 * np.abs(G).max()


# ---------------------------------------------------------------------------
# soft thresholding and Upsilon (Sec. 4.1, Fig. 6)
# ---------------------------------------------------------------------------
def test_soft_threshold_values():
    U = np.array([-2.0 + 3.0j, 0.5 - 0.25j, 0.0 + 0.0j])
    assert np.allclose(O.soft_threshold(U, 2.0), [-4.0 + 9.0j, 0.25 - 0.0625j, 0.0])
    assert np.allclose(O.soft_threshold(U, 1.5),
                       [-2.0 ** 1.5 + 3.0 ** 1.5 * 1j, 0.5 ** 1.5 - 0.25 ** 1.5 * 1j, 0.0])
    assert np.array_equal(O.soft_threshold(U, 1.0), U)


def test_upsilon_identities():
    dims = (8, 10, 12)
    rng = np.random.default_rng(34)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    f = rng.standard_normal(dims)
    # p = 1: Phi is the identity and Upsilon the ball projection
    ref = np.fft.ifftn(np.fft.fftn(f) * (bank.G > 0)).real
    assert np.abs(O.upsilon(f, bank, 1.0) - ref).max() < 1e-12
    u = O.upsilon(f, bank, 1.5)
    # odd and positively homogeneous of degree p
    assert np.abs(O.upsilon(-f, bank, 1.5) + u).max() < 1e-12 * np.abs(u).max()
    assert np.abs(O.upsilon(4.0 * f, bank, 1.5) - 8.0 * u).max() < 1e-12 * np.abs(u).max()
    assert np.abs(u - ref).max() > 0.01 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# linear left-invariant diffusion (Sec. 4.1 with a constant diagonal D_ij)
# ---------------------------------------------------------------------------
def test_discrete_laplace_beltrami_on_harmonic_polynomials():
    """Restrictions of harmonic polynomials of degree l to S^2 are
    eigenfunctions of the Laplace-Beltrami operator with eigenvalue -l(l+1)."""
    V = O.icosa_orientations(1)
    L = O.angular_laplacian(V, O.sh_degree_for(V))
    x, y, z = V.T
    for u, ev in ((np.ones_like(z), 0), (z, -2), (x * y, -6), (z * z - 1.0 / 3.0, -6),
                  (x * y * z, -12), (x ** 3 - 3 * x * y * y, -12)):
        assert np.abs(L @ u - ev * u).max() < 1e-10
    import scipy.linalg
    E = scipy.linalg.expm(0.3 * L)
    assert np.abs(E @ z - np.exp(-0.6) * z).max() < 1e-10


@pytest.mark.parametrize("make,n,deg", [(O.icosa_orientations, 1, 5), (O.octa_orientations, 1, 2),
                                        (O.octa_orientations, 2, 6), (O.icosa_orientations, 2, 11)])
def test_laplacian_degree_choice(make, n, deg):
    """The largest degree with (l+1)^2 <= N_o, lowered while a harmonic of the
    top degree vanishes on the set: every vector of the 18-point octahedral set
    has a zero coordinate, so the degree-3 harmonic xyz vanishes there."""
    V = make(n)
    if len(V) == 18:
        assert np.abs(V[:, 0] * V[:, 1] * V[:, 2]).max() < 1e-15
    assert O.sh_degree_for(V) == deg


def test_isotropic_spatial_diffusion_is_the_heat_kernel():
    """With D44 = 0 and D11 = D33 = D the evolution multiplies every
    orientation by exp(-t D |w|^2), which commutes with W: the enhancement is
    the ball-limited heat kernel, for any number of Strang steps."""
    dims = (12, 16, 10)
    f = np.random.default_rng(35).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    wz, wy, wx = O.freq_grid(dims)
    r2 = wz ** 2 + wy ** 2 + wx ** 2
    ref = np.fft.ifftn(np.fft.fftn(f) * (r2 < np.pi ** 2) * np.exp(-1.5 * 0.4 * r2)).real
    for K in (1, 3):
        g = O.enhance_linear(f, bank, O.Diffusion(t=1.5, steps=K, D11=0.4, D33=0.4, D44=0.0))
        assert np.abs(g - ref).max() < 1e-12 * np.abs(ref).max()
    g0 = O.enhance_linear(f, bank, O.Diffusion(t=0.0, steps=2))
    ref0 = np.fft.ifftn(np.fft.fftn(f) * (r2 < np.pi ** 2)).real
    assert np.abs(g0 - ref0).max() < 1e-12


def test_angular_diffusion_keeps_orientation_constant_scores():
    dims = (8, 8, 8)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    g = np.random.default_rng(36).standard_normal(dims)
    U = np.broadcast_to(g, (bank.n_o,) + dims).astype(np.complex128)
    out = O.diffuse(U, bank, O.Diffusion(t=3.0, steps=4, D11=0.0, D33=0.0, D44=0.5))
    assert np.abs(out - U).max() < 1e-12


def test_strang_splitting_is_second_order():
    dims = (12, 12, 12)
    f = np.random.default_rng(37).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    D = dict(t=2.0, D11=0.1, D33=1.0, D44=0.05)
    ref = O.enhance_linear(f, bank, O.Diffusion(steps=256, **D))
    err = [np.abs(O.enhance_linear(f, bank, O.Diffusion(steps=K, **D)) - ref).max()
           for K in (4, 8, 16)]
    for a, b in zip(err[:-1], err[1:]):
        assert 3.5 < a / b < 4.5


def test_diffused_score_of_a_real_image_keeps_antipodal_conjugacy():
    dims = (10, 12, 8)
    f = np.random.default_rng(38).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    W = O.diffuse(O.forward(f, bank), bank, O.Diffusion(t=2.0, steps=3, D11=0.2, D33=1.0, D44=0.1))
    h = bank.n_o // 2
    assert np.abs(W[h:] - np.conj(W[:h])).max() < 1e-13 * np.abs(W).max()


# ---------------------------------------------------------------------------
# pins of the individual diffusion rates (Sec. 4.1): the spatial generator
# D11 (A1^2 + A2^2) + D33 A3^2 acts on a plane wave exp(i w.x) in channel n as
# multiplication by -[D11 (|w|^2 - (w.n)^2) + D33 (w.n)^2], so a plane wave
# along n feels only D33 and one across n only D11; the angular generator
# D44 (A4^2 + A5^2) multiplies a degree-l harmonic of n by -D44 l (l + 1).
# ---------------------------------------------------------------------------
def _plane_wave_decay(D11, D33, t=0.7, steps=3):
    """Per channel, the factor by which ``diffuse`` scales a plane wave along
    z (D44 = 0, so every Strang step is exact); the wave number and the
    channel orientations."""
    dims = (16, 8, 8)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    kz = 3
    z = np.arange(dims[0]).reshape(-1, 1, 1)
    wave = np.broadcast_to(np.exp(2j * np.pi * kz * z / dims[0]), dims)
    U = np.broadcast_to(wave, (bank.n_o,) + dims).astype(np.complex128)
    out = O.diffuse(U, bank, O.Diffusion(t=t, steps=steps, D11=D11, D33=D33, D44=0.0))
    ratio = (out / U).reshape(bank.n_o, -1)
    assert np.abs(ratio - ratio[:, :1]).max() < 1e-12   # a pure multiplier per channel
    assert np.abs(ratio.imag).max() < 1e-12
    return ratio[:, 0].real, 2.0 * np.pi * kz / dims[0], bank.orients


def _check_anisotropy(D=0.35, t=0.7):
    """Diffusion only along n (D33 = D): the channel with n = +-e_z decays by
    exp(-t D |w|^2) for the wave w along z; the channels with n in the xy-plane
    (n.w = 0) keep it. Only across n (D11 = D): the reverse."""
    along, w, V = _plane_wave_decay(0.0, D, t)
    across, _, _ = _plane_wave_decay(D, 0.0, t)
    par = np.abs(np.abs(V[:, 2]) - 1.0) < 1e-12
    perp = np.abs(V[:, 2]) < 1e-12
    assert par.sum() == 2 and perp.sum() >= 4
    full = math.exp(-t * D * w * w)
    err = max(np.abs(along[par] - full).max(), np.abs(along[perp] - 1.0).max(),
              np.abs(across[par] - 1.0).max(), np.abs(across[perp] - full).max())
    return err


def test_spatial_diffusion_along_and_across_the_orientation():
    assert _check_anisotropy() < 1e-12


def _check_angular_rate(D44=0.3, t=1.1, steps=5):
    """U_i(x) = Y(n_i) g(x) with Y a harmonic polynomial of degree l <= the
    operator's degree decays as exp(-t D44 l (l + 1)) for any number of Strang
    steps (D11 = D33 = 0)."""
    dims = (6, 6, 6)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    g = np.random.default_rng(40).standard_normal(dims)
    x, y, z = bank.orients.T
    err = 0.0
    for Y, l in ((z, 1), (x * y, 2), (x * x - y * y, 2), (x * y * z, 3), (x ** 3 - 3 * x * y * y, 3)):
        U = Y[:, None, None, None] * g[None]
        out = O.diffuse(U.astype(np.complex128), bank,
                        O.Diffusion(t=t, steps=steps, D11=0.0, D33=0.0, D44=D44))
        err = max(err, np.abs(out - math.exp(-t * D44 * l * (l + 1)) * U).max() / np.abs(U).max())
    return err


def test_angular_diffusion_rate_of_harmonics():
    assert _check_angular_rate() < 1e-12


def test_rate_pins_fail_on_planted_mistakes(monkeypatch):
    """The two pins above reject the mistakes a shared reading could make: the
    rates D11 and D33 swapped, and a wrong step factor on dt D44."""
    real_rates = O.spatial_rates

    def swapped(bank, D):
        return real_rates(bank, O.Diffusion(t=D.t, steps=D.steps, D11=D.D33, D33=D.D11,
                                            D44=D.D44, sh_degree=D.sh_degree))

    with monkeypatch.context() as m:
        m.setattr(O, "spatial_rates", swapped)
        assert _check_anisotropy() > 1e-2
    real_expm = O.scipy.linalg.expm
    with monkeypatch.context() as m:
        m.setattr(O.scipy.linalg, "expm", lambda A: real_expm(0.5 * A))   # dt/2 instead of dt
        assert _check_angular_rate() > 1e-2
    with monkeypatch.context() as m:
        m.setattr(O.scipy.linalg, "expm", lambda A: real_expm(2.0 * A))
        assert _check_angular_rate() > 1e-2


# ---------------------------------------------------------------------------
# radial window g = M_N(rho^2 / t) (Sec. 3.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,gamma", [(8, 0.8), (20, 0.8), (20, 0.85), (3, 0.5)])
def test_radial_window_is_the_regularised_upper_gamma_with_its_inflection_at_gamma_rho_n(N, gamma):
    """exp(-x) sum_{k<=N} x^k / k! is the regularised upper incomplete gamma
    function Q(N + 1, x) (a library routine); as a function of rho its second
    derivative changes sign at gamma rho_N, the inflection point Sec. 3.1
    places there by the choice of t."""
    import scipy.special
    rho = np.linspace(0.0, 1.8 * np.pi, 301)
    t = O.radial_t(N, gamma)
    assert np.abs(O.radial_window(rho, N, gamma) - scipy.special.gammaincc(N + 1, rho ** 2 / t)).max() < 1e-13
    r0, h = gamma * np.pi, 1e-3
    d2 = lambda r: (O.radial_window(r + h, N, gamma) - 2 * O.radial_window(r, N, gamma)
                    + O.radial_window(r - h, N, gamma)) / h ** 2
    assert d2(r0 - 0.02) < 0.0 < d2(r0 + 0.02)
    assert abs(d2(r0)) < 1e-3 * abs(d2(r0 - 0.3))


# ---------------------------------------------------------------------------
# weighted energy sum w |U|^2 of a score (Sec. 2, norm preservation)
# ---------------------------------------------------------------------------
def test_weighted_energy_of_a_score_is_parseval_with_M():
    # sum_i sum_x |U_i|^2 = (1/n^3) sum_w M(w) |f_hat(w)|^2: with M = 1 this is
    # the norm preservation ||W f||^2 = ||f||^2 of Sec. 2
    dims = (12, 10, 16)
    rng = np.random.default_rng(31)
    f = rng.standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    U = O.forward(f, bank)
    rhs = np.sum(bank.M() * np.abs(np.fft.fftn(f)) ** 2) / np.prod(dims)
    assert abs(O.weighted_energy(U) - rhs) <= 1e-12 * rhs
    # a plane wave inside the pass band, where M ~ 1: the energy is ||f||^2
    z, y, x = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    k = (1, 1, 2)
    pw = np.cos(2 * np.pi * (k[0] * z / dims[0] + k[1] * y / dims[1] + k[2] * x / dims[2]))
    e = O.weighted_energy(O.forward(pw, bank))
    m = bank.M()[k]
    assert abs(e - m * np.sum(pw ** 2)) <= 1e-12 * e
    assert abs(m - 1.0) < 0.05


def test_weighted_energy_is_the_loop_sum():
    rng = np.random.default_rng(32)
    U = rng.standard_normal((3, 2, 4)) + 1j * rng.standard_normal((3, 2, 4))
    w = rng.uniform(0, 1, U.shape)
    s = 0.0
    for idx in np.ndindex(U.shape):
        s += w[idx] * (U[idx].real ** 2 + U[idx].imag ** 2)
    assert abs(O.weighted_energy(U, w) - s) <= 1e-14 * s
    assert O.weighted_energy(np.zeros((0, 4), complex)) == 0.0
    assert abs(O.weighted_energy(U) - sum(abs(u) ** 2 for u in U.ravel())) <= 1e-13


def _energy_grad_mismatch(grad_fn, seed=33):
    """max relative gap between central differences of L(U + t D) and the
    directional derivative Re sum conj(G) D that PyTorch's convention assigns
    to the gradient G (L is quadratic, so the difference quotient is exact up
    to rounding)."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((4, 5, 6)) + 1j * rng.standard_normal((4, 5, 6))
    w = rng.uniform(0, 1, U.shape)
    g = 0.75
    worst = 0.0
    for _ in range(4):
        D = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
        h = 1e-3
        fd = g * (O.weighted_energy(U + h * D, w) - O.weighted_energy(U - h * D, w)) / (2 * h)
        dd = float(np.real(np.vdot(grad_fn(U, w, g), D)))
        worst = max(worst, abs(fd - dd) / abs(fd))
    return worst


def test_weighted_energy_gradient_by_central_differences():
    assert _energy_grad_mismatch(O.weighted_energy_grad) < 1e-10


def test_energy_gradient_pin_fails_on_planted_mistakes():
    planted = [lambda U, w, g: g * w * U,                 # factor 2 dropped
               lambda U, w, g: 2 * g * w * np.conj(U),    # conjugate taken
               lambda U, w, g: 2 * g * U,                 # weight dropped
               lambda U, w, g: 2 * w * U]                 # upstream scalar dropped
    for bad in planted:
        assert _energy_grad_mismatch(bad) > 1e-2
