"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute-force
sums, textbook closed forms, library routines the oracle does not use,
quadrature, identities of Sec. 2 and App. A, and symmetries of the grid.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sps

from oracle import os3d_oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _dft_matrix(n, sign):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


def _idft3_bruteforce(X):
    """x(r) = 1/n^3 sum_k X(k) exp(+2 pi i k.r/n), by explicit matrices."""
    nz, ny, nx = X.shape
    Z, Y, XX = _dft_matrix(nz, +1), _dft_matrix(ny, +1), _dft_matrix(nx, +1)
    return np.einsum("az,by,cx,zyx->abc", Z, Y, XX, X) / (nz * ny * nx)


def _small_bank(dims, subdiv=0, L=6, **kw):
    p = O.Params(L=L, fit_mode=kw.pop("fit_mode", 0), **kw)
    return O.Bank(dims, O.icosa_orientations(subdiv), p)


# ---------------------------------------------------------------------------
# the transform against the correlation definition (Eq. construction1Discrete)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(8, 8, 8), (6, 8, 10)])
def test_forward_is_bruteforce_correlation(dims):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(dims)
    bank = _small_bank(dims)
    U = O.forward(f, bank, orients_idx=[0, 3, 7])
    nz, ny, nx = dims
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for j, i in enumerate([0, 3, 7]):
        psi = _idft3_bruteforce(bank.psi_hat(i))       # spatial wavelet psi_i
        ref = np.empty(dims, dtype=np.complex128)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    # U(x) = sum_x' conj(psi(x' - x)) f(x'), periodic
                    sh = psi[(zz - z) % nz, (yy - y) % ny, (xx - x) % nx]
                    ref[z, y, x] = np.sum(np.conj(sh) * f)
        assert np.abs(U[j] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_spatial_wavelet_parts():
    """Re psi comes from the even (line) part, Im psi from the odd (edge) part."""
    bank = _small_bank((8, 8, 8), L=8)
    ce, co = O.funk_antisym(O.fit_coefficients(bank.p))
    kap = bank.c[0] / ce[0]
    he = O.Bank.__new__(O.Bank)
    he.__dict__.update(bank.__dict__)
    he.c = kap * ce
    psi_e = _idft3_bruteforce(he.psi_hat(2))
    ho = O.Bank.__new__(O.Bank)
    ho.__dict__.update(bank.__dict__)
    ho.c = kap * co
    psi_o = _idft3_bruteforce(ho.psi_hat(2))
    psi = _idft3_bruteforce(bank.psi_hat(2))
    assert np.abs(psi_e.imag).max() < 1e-14
    assert np.abs(psi_o.real).max() < 1e-14
    assert np.allclose(psi, psi_e + psi_o, atol=1e-14)


# ---------------------------------------------------------------------------
# Legendre polynomials, B-splines
# ---------------------------------------------------------------------------
def test_legendre_against_scipy_and_closed_form():
    t = np.linspace(-1, 1, 41)
    P = O.legendre_table(24, t)
    for l in range(25):
        assert np.allclose(P[l], sps.eval_legendre(l, t), atol=1e-13)
    P0 = O.legendre_table(24, np.array(0.0))
    for l in range(25):
        if l % 2:
            exact = Fraction(0)
        else:
            num = math.prod(range(l - 1, 0, -2)) if l > 0 else 1
            den = math.prod(range(l, 0, -2)) if l > 0 else 1
            exact = Fraction((-1) ** (l // 2) * num, den)
        assert abs(P0[l] - float(exact)) < 1e-15


def test_bspline_closed_forms_and_convolution():
    x = np.linspace(-3, 3, 1201)
    B1 = np.where(np.abs(x) < 1, 1 - np.abs(x), 0)
    assert np.allclose(O.bspline(x, 1), B1, atol=1e-14)
    ax = np.abs(x)
    B2 = np.where(ax <= 0.5, 0.75 - ax ** 2, np.where(ax <= 1.5, 0.5 * (1.5 - ax) ** 2, 0))
    assert np.allclose(O.bspline(x, 2), B2, atol=1e-14)
    # B^k = B^{k-1} * B^0, by numerical convolution on a fine grid
    h = 1e-3
    g = np.arange(-4, 4 + h / 2, h)
    box = np.where(np.abs(g) < 0.5, 1.0, 0.0)
    for k in (1, 2, 3):
        conv = np.convolve(O.bspline(g, k - 1), box, mode="same") * h
        assert np.abs(conv - O.bspline(g, k)).max() < 3e-3
    # partition of unity and unit integral
    for k in (0, 1, 2, 3, 4):
        s = sum(O.bspline(x + j, k) for j in range(-8, 9))
        assert np.allclose(s[(x > -2) & (x < 2)], 1.0, atol=1e-12) or k == 0
        assert abs(np.sum(O.bspline(g, k)) * h - 1.0) < 2e-3


# ---------------------------------------------------------------------------
# Zonal SH fit (Sec. 3.2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
def test_fit_recovers_polynomial_profiles(mode):
    rng = np.random.default_rng(3)
    L = 12
    beta = rng.standard_normal(L + 1)

    def prof(th):
        return O.legendre_series(beta, np.cos(th))

    if mode == 0:
        b = O.fit_legendre_projection(prof, L)
    else:
        b = O.fit_legendre_lsq(prof, L)
    assert np.allclose(b, beta, atol=1e-10)


def test_fit_modes_approximate_the_bspline():
    for p in (O.Params(L=16, fit_mode=0), O.Params(L=16, fit_mode=1)):
        b = O.fit_coefficients(p)
        th = np.linspace(0, np.pi, 2001)
        A = O.orientation_distribution(th, p.k, p.s_theta)
        Af = O.legendre_series(b, np.cos(th))
        assert np.sqrt(np.mean((A - Af) ** 2)) < 0.02
    b0 = O.fit_coefficients(O.Params(L=16, fit_mode=0))
    b1 = O.fit_coefficients(O.Params(L=16, fit_mode=1))
    assert np.abs(b0 - b1).max() < 2e-3


def test_tessellation_counts():
    for nu in (1, 2, 3, 15):
        pts = O.icosa_tessellation(nu)
        assert pts.shape == (10 * nu * nu + 2, 3)
        assert np.allclose(np.linalg.norm(pts, axis=1), 1)
    a = np.round(O.icosa_tessellation(2), 9)
    b = np.round(O.icosa_orientations(1), 9)
    assert {tuple(r) for r in a} == {tuple(r) for r in b}


# ---------------------------------------------------------------------------
# Funk transform and anti-symmetrisation (Sec. 3.2)
# ---------------------------------------------------------------------------
def _great_circle_integral(func, n, m=4096):
    n = n / np.linalg.norm(n)
    a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.9 else np.array([0, 1.0, 0])
    u = np.cross(n, a)
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    ph = np.arange(m) * 2 * np.pi / m
    pts = np.cos(ph)[:, None] * u + np.sin(ph)[:, None] * v
    return np.sum(func(pts)) * 2 * np.pi / m


def test_funk_eigenvalue_by_quadrature():
    rng = np.random.default_rng(4)
    for _ in range(4):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        for l in range(9):
            lhs = _great_circle_integral(lambda p: sps.eval_legendre(l, p[:, 2]), n)
            rhs = 2 * np.pi * sps.eval_legendre(l, 0.0) * sps.eval_legendre(l, n[2])
            assert abs(lhs - rhs) < 1e-10


def test_line_part_is_funk_of_fitted_profile():
    p = O.Params(L=16, fit_mode=0)
    b = O.fit_coefficients(p)
    ce, co = O.funk_antisym(b)
    rng = np.random.default_rng(5)
    for _ in range(5):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        quad = _great_circle_integral(lambda q: O.legendre_series(b, q[:, 2]), n)
        assert abs(O.legendre_series(ce, n[2]) - quad) < 1e-10
        # and close to the Funk transform of the exact B-spline profile
        quadA = _great_circle_integral(
            lambda q: O.orientation_distribution(np.arccos(np.clip(q[:, 2], -1, 1)), p.k, p.s_theta), n)
        assert abs(O.legendre_series(ce, n[2]) - quadA) < 0.05 * abs(quadA) + 0.02


def test_edge_part_is_antisymmetrised_profile():
    b = O.fit_coefficients(O.Params(L=16))
    ce, co = O.funk_antisym(b)
    t = np.linspace(-1, 1, 101)
    ho = O.legendre_series(co, t)
    assert np.allclose(ho, O.legendre_series(b, t) - O.legendre_series(b, -t), atol=1e-14)
    assert np.allclose(ho, -O.legendre_series(co, -t), atol=1e-14)
    he = O.legendre_series(ce, t)
    assert np.allclose(he, O.legendre_series(ce, -t), atol=1e-14)


# ---------------------------------------------------------------------------
# steering (Eq. Rotationh): zonal form = SH addition theorem
# ---------------------------------------------------------------------------
def test_zonal_steering_matches_spherical_harmonics():
    L = 6
    b = np.random.default_rng(6).standard_normal(L + 1)
    rng = np.random.default_rng(7)
    for _ in range(6):
        n = rng.standard_normal(3); n /= np.linalg.norm(n)
        w = rng.standard_normal(3); w /= np.linalg.norm(w)
        tn, pn = np.arccos(n[2]), np.arctan2(n[1], n[0])
        tw, pw = np.arccos(w[2]), np.arctan2(w[1], w[0])
        sh = 0.0
        for l in range(L + 1):
            s = sum(sps.sph_harm_y(l, m, tw, pw) * np.conj(sps.sph_harm_y(l, m, tn, pn))
                    for m in range(-l, l + 1))
            sh += b[l] * 4 * np.pi / (2 * l + 1) * s
        assert abs(O.legendre_series(b, w @ n) - sh) < 1e-12


# ---------------------------------------------------------------------------
# orientation sets (Sec. 2.1)
# ---------------------------------------------------------------------------
def test_orientation_sets():
    V0 = O.icosa_orientations(0)
    d = V0 @ V0.T
    # every icosahedron vertex has exactly 5 nearest neighbours at cos = 1/sqrt(5)
    assert np.all(np.sum(np.abs(d - 1 / np.sqrt(5)) < 1e-12, axis=1) == 5)
    for s, n in ((0, 12), (1, 42), (2, 162)):
        V = O.icosa_orientations(s)
        assert V.shape == (n, 3)
        assert np.allclose(np.linalg.norm(V, axis=1), 1)
        h = n // 2
        assert np.allclose(V[h:], -V[:h], atol=0)
        assert np.all((V[:h, 2] > 1e-9) | ((np.abs(V[:h, 2]) <= 1e-9) & (V[:h, 1] > 1e-9))
                      | ((np.abs(V[:h, 2]) <= 1e-9) & (np.abs(V[:h, 1]) <= 1e-9) & (V[:h, 0] > 0)))
        assert np.all(np.diff(V[:h, 2]) <= 1e-9)
        assert len({tuple(np.round(v, 9)) for v in V}) == n
        pairs = O.orientation_pairs(V)
        assert np.all(pairs == np.concatenate([np.arange(h, n), np.arange(h)]))


# ---------------------------------------------------------------------------
# M_psi, Parseval, symmetry, reconstruction (Sec. 2, 2.1, App. A)
# ---------------------------------------------------------------------------
def _rho(dims):
    wz, wy, wx = O.freq_grid(dims)
    return np.sqrt(wz ** 2 + wy ** 2 + wx ** 2)


@pytest.mark.parametrize("subdiv,L,tol", [(1, 12, 0.03), (2, 16, 0.02)])
def test_M_close_to_one_in_pass_band(subdiv, L, tol):
    dims = (24, 24, 24)
    bank = O.Bank(dims, O.icosa_orientations(subdiv), O.Params(L=L))
    M = bank.M()
    rho = _rho(dims)
    band = (rho > 0) & (rho <= 0.5 * np.pi)
    assert np.abs(M[band] - 1).max() <= tol
    ball = (rho > 0) & (rho < np.pi)
    assert np.all(M[ball] >= 0.99 * bank.G[ball] ** 2)
    assert np.all(M[rho >= np.pi] == 0)


def test_spherical_mean_of_angular_M_is_one():
    bank = O.Bank((4, 4, 4), O.icosa_orientations(1), O.Params(L=12))
    m = 20000   # Fibonacci sphere
    i = np.arange(m) + 0.5
    z = 1 - 2 * i / m
    r = np.sqrt(1 - z * z)
    ph = np.pi * (1 + 5 ** 0.5) * i
    w = np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)
    s = sum(O.legendre_series(bank.c, w @ n) ** 2 for n in bank.orients)
    assert abs(np.mean(s) - 1.0) < 1e-4


def test_parseval_identity():
    dims = (16, 12, 10)
    rng = np.random.default_rng(8)
    f = rng.standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    U = O.forward(f, bank)
    lhs = np.sum(np.abs(U) ** 2)
    fh = np.fft.fftn(f)
    rhs = np.sum(bank.M() * np.abs(fh) ** 2) / np.prod(dims)
    assert abs(lhs - rhs) <= 1e-12 * rhs


def test_hermitian_and_antipodal_symmetry():
    dims = (12, 12, 12)
    f = np.random.default_rng(9).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    U = O.forward(f, bank)
    h = bank.n_o // 2
    assert np.abs(U[h:] - np.conj(U[:h])).max() < 1e-13 * np.abs(U).max()
    # Re U_i = line response IDFT(f_hat G h_e), Im U_i from the edge part
    ce, co = O.funk_antisym(O.fit_coefficients(bank.p))
    kap = bank.c[0] / ce[0]
    fh = np.fft.fftn(f)
    for i in (0, 5):
        t = sum(bank.what[a] * bank.orients[i][2 - a] for a in range(3))
        he = np.where(bank.zero, kap * ce[0], O.legendre_series(kap * ce, t))
        ho = np.where(bank.zero, 0.0, O.legendre_series(kap * co, t))
        re = np.fft.ifftn(fh * bank.G * he)
        im = np.fft.ifftn(fh * bank.G * ho)
        assert np.abs(re.imag).max() < 1e-13 and np.abs(im.real).max() < 1e-13
        assert np.allclose(U[i].real, re.real, atol=1e-13)
        assert np.allclose(U[i].imag, im.imag, atol=1e-13)


def test_exact_reconstruction():
    dims = (16, 16, 16)
    f = np.random.default_rng(10).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    fr = O.inverse(O.forward(f, bank), bank)
    ball = _rho(dims) < np.pi
    fb = np.fft.ifftn(np.fft.fftn(f) * ball).real
    assert np.abs(fr - fb).max() < 1e-12
    # a ball-limited image is reproduced exactly
    fr2 = O.inverse(O.forward(fb, bank), bank)
    assert np.abs(fr2 - fb).max() < 1e-12


def test_clamp_limits():
    """eps above max M turns the exact inverse into the adjoint / eps."""
    dims = (12, 12, 12)
    f = np.random.default_rng(11).standard_normal(dims)
    p = O.Params(L=12, eps=50.0)
    bank = O.Bank(dims, O.icosa_orientations(1), p)
    assert bank.M().max() < p.eps
    U = O.forward(f, bank)
    assert np.allclose(O.inverse(U, bank), O.adjoint(U, bank) / p.eps, atol=1e-14)


def test_figure_parameter_sets_are_admissible():
    path = os.path.join(os.path.dirname(__file__), "golden", "figure_params.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for name, L, s, k, N, g, grid, no, *_ in rows:
        p = O.Params(L=int(L), s_theta=float(s), k=int(k), N=int(N), gamma=float(g))
        n = min(int(grid), 16)
        bank = O.Bank((n, n, n), O.icosa_orientations(1), p)
        M = bank.M()
        inner = (_rho(bank.dims) > 0) & (_rho(bank.dims) < 0.6 * np.pi)
        assert M[inner].min() > 0.5            # admissibility (Eq. AdmissibilityRequirement)
        assert np.isfinite(M).all()
    # N = 20: g(rho_N)^2 ~ 2.5e-4, so the clamp eps = 1e-4 is close to binding there
    assert O.radial_window(np.pi, 20, 0.8) ** 2 < 1e-3


# ---------------------------------------------------------------------------
# grid symmetries that map the icosahedral sets onto themselves
# ---------------------------------------------------------------------------
def _grid_maps():
    """(R acting on (x,y,z) vectors, index map of an array f(z,y,x) -> f(R^T r))."""
    def flip(a, axes):
        return np.roll(np.flip(a, axis=axes), 1, axis=axes)
    maps = []
    # 180 deg about z: (x,y,z) -> (-x,-y,z)
    maps.append((np.diag([-1, -1, 1.0]), lambda a: flip(a, (-1, -2))))
    # 180 deg about x: (x,y,z) -> (x,-y,-z)
    maps.append((np.diag([1, -1, -1.0]), lambda a: flip(a, (-2, -3))))
    # inversion
    maps.append((-np.eye(3), lambda a: flip(a, (-1, -2, -3))))
    # cyclic permutation (x,y,z) -> (y,z,x), i.e. R e_x = e_z, R e_y = e_x, R e_z = e_y
    R = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0.0]])
    # g(r) = f(R^T r): array axes are (z,y,x) and R^T (x,y,z) = (z,x,y), so
    # g[z,y,x] = f[y,x,z], i.e. g[a,b,c] = f[b,c,a]
    maps.append((R, lambda a: np.transpose(a, (2, 0, 1))))
    return maps


def test_equivariance_under_grid_symmetries():
    dims = (12, 12, 12)
    f = np.random.default_rng(12).standard_normal(dims)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    U = O.forward(f, bank)
    V = bank.orients
    for R, act in _grid_maps():
        RV = V @ R.T
        perm = [int(np.argmin(np.abs(V - rv).sum(axis=1))) for rv in RV]
        assert np.allclose(V[perm], RV, atol=1e-12)
        # check the index map realises f(R^T r) on a test vector
        r = np.array([3, 1, 2])    # (x,y,z)
        g = act(f)
        src = (R.T @ r).astype(int) % 12
        assert g[r[2], r[1], r[0]] == f[src[2], src[1], src[0]]
        U2 = O.forward(g, bank)
        for i in range(bank.n_o):
            assert np.allclose(U2[perm[i]], act(U[i]), atol=1e-12)


# ---------------------------------------------------------------------------
# adjoint (Sec. 4.1, App. A)
# ---------------------------------------------------------------------------
def test_adjoint_dot_product():
    dims = (10, 12, 8)
    rng = np.random.default_rng(13)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=12))
    f = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
    G = rng.standard_normal((bank.n_o,) + dims) + 1j * rng.standard_normal((bank.n_o,) + dims)
    fh = np.fft.fftn(f)
    Wf = np.stack([np.fft.ifftn(fh * bank.psi_hat(i)) for i in range(bank.n_o)])
    lhs = np.vdot(Wf, G)
    rhs = np.vdot(f, O.adjoint(G, bank, real=False))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gradient_of_quadratic_loss_by_central_differences():
    dims = (8, 8, 8)
    rng = np.random.default_rng(14)
    bank = O.Bank(dims, O.icosa_orientations(1), O.Params(L=8))
    f = rng.standard_normal(dims)
    w = rng.uniform(0, 1, (bank.n_o,) + dims)

    def loss(x):
        return np.sum(w * np.abs(O.forward(x, bank)) ** 2)

    grad = O.adjoint(2 * w * O.forward(f, bank), bank)
    eps = 1e-3
    for _ in range(3):
        d = rng.standard_normal(dims)
        fd = (loss(f + eps * d) - loss(f - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(grad * d)) < 1e-9 * abs(fd)
    for idx in [(0, 0, 0), (3, 5, 7)]:
        e = np.zeros(dims); e[idx] = 1
        fd = (loss(f + eps * e) - loss(f - eps * e)) / (2 * eps)
        assert abs(fd - grad[idx]) < 1e-9 * max(1.0, abs(fd))
