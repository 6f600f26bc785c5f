"""FP64 CPU oracle of the invertible 3D orientation-score transform.

Janssen, Duits, Breeuwer, "Invertible Orientation Scores of 3D Images"
(arXiv 1505.07690).

TEST INFRASTRUCTURE. This module is the slow, plain, obviously-correct
statement of what the GPU library computes. Only the test-suite, the smoke
check of ``__graft_entry__`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it. The product path (the C-ABI library and its
Python binding) never imports, links or calls it, and it never calls the
product path. It shares no code, constants or tables with the CUDA side.

Everything is float64 / complex128 numpy. Library primitives used as single
steps: ``numpy.fft.fftn/ifftn`` (the DFT), ``numpy.linalg.pinv`` (the
pseudo-inverse the paper names for the SH fit and the discrete
Laplace-Beltrami operator), ``numpy.polynomial.legendre.leggauss``
(Gauss-Legendre nodes), ``scipy.special.lpmv`` (associated Legendre
functions) and ``scipy.linalg.expm`` (matrix exponential).

Conventions (readings of the paper, each repeated in the design notes):

* Discrete Fourier transform: unnormalised forward DFT ``fftn`` with kernel
  exp(-i w.x) (the paper's sign, Sec. 2, the Fourier transform under
  Eq. Reconstruction1); ``ifftn`` carries 1/n^3. The continuous constants
  (2 pi)^(+-3/2) and the spherical measure d sigma = 4 pi / N_o cancel in the
  exact inverse and are absorbed in the wavelet normalisation kappa.
* Frequency grid: w_j = 2 pi k_j / n_j with k_j the signed FFT index, so the
  Nyquist frequency is rho_N = pi (Sec. 3.1, radial function).
* Ball limit: psi_hat = 0 for |w| >= rho_N (Sec. 2: f is ball-limited with
  varrho = rho_N, Sec. 3.1).
* At w = 0 the direction w/|w| is undefined; the angular factor there is the
  spherical mean of h, i.e. its l = 0 Legendre coefficient.

Pins (tests/test_oracle_*.py): brute-force DFT correlation at 8^3, textbook
Legendre values, B-spline convolution, exact recovery of polynomial
profiles by both fits, great-circle Funk quadrature, the spherical-harmonic
addition theorem, M ~ 1, Parseval, Hermitian/antipodal symmetry, exact
reconstruction, grid-symmetry equivariance, the adjoint identity and finite
differences; for the weighted energy, Parseval with M, a brute-force loop sum
and central differences along complex directions; for the diffusion, harmonic polynomials (the Laplace-Beltrami
eigenvalues and the angular decay exp(-t D44 l(l+1))), plane waves along and
across n (D33 and D11 separately), the heat kernel and the splitting order;
the radial window against the regularised incomplete gamma function and its
inflection point. Every function below is pinned by at least one of them.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.special

PHI = (1.0 + math.sqrt(5.0)) / 2.0
RHO_N = math.pi


# ---------------------------------------------------------------------------
# Wavelet parameters (Sec. 3.1; figure captions of Figs. 3-5)
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Params:
    k: int = 2            # B-spline order of the orientation distribution A
    s_theta: float = 0.7  # angular width of A
    L: int = 16           # maximal Legendre / SH degree
    N: int = 8            # order of the Taylor-corrected Gaussian M_N
    gamma: float = 0.8    # inflection point of g at gamma * rho_N
    eps: float = 1e-4     # clamp M -> max(M, eps) of Sec. 3.1
    fit_mode: int = 1     # 1: paper's pseudo-inverse on tessellation order 15
                          # 0: L2 projection by Gauss-Legendre quadrature
    profile: int = 0      # 0: cake wavelet h = F A + antisym(A) (line + edge detector)
                          # 1: h = A (plate + edge detector, first construction of Sec. 3.1)


# ---------------------------------------------------------------------------
# Frequency grid and radial window (Sec. 3.1, Eq. for g = M_N)
# ---------------------------------------------------------------------------
def freq_grid(dims):
    """Angular frequencies (wz, wy, wx), broadcastable to ``dims`` (nz, ny, nx).

    w_j = 2 pi k_j / n_j, k_j the signed DFT index (numpy.fft order).
    """
    out = []
    for ax, n in enumerate(dims):
        k = np.fft.fftfreq(n) * n
        w = 2.0 * np.pi * k / n
        shape = [1, 1, 1]
        shape[ax] = n
        out.append(w.reshape(shape))
    return tuple(out)


def radial_t(N, gamma):
    """Scale t of g with its inflection point at gamma * rho_N:
    t = 2 (gamma rho_N)^2 / (1 + 2N)  (Sec. 3.1)."""
    return 2.0 * (gamma * RHO_N) ** 2 / (1.0 + 2.0 * N)


def radial_window(rho, N, gamma):
    """g(rho) = M_N(rho^2 / t) = exp(-x) sum_{k=0}^{N} x^k / k!, x = rho^2/t
    (Sec. 3.1). No ball cut here; see ``radial_ball``."""
    x = np.asarray(rho, dtype=np.float64) ** 2 / radial_t(N, gamma)
    s = np.zeros_like(x)
    term = np.ones_like(x)
    for k in range(N + 1):
        if k > 0:
            term = term * x / k
        s = s + term
    return np.exp(-x) * s


def radial_ball(dims, N, gamma):
    """G(w) = g(|w|) inside the ball |w| < rho_N, 0 outside (Sec. 2 ball limit,
    Sec. 3.1 varrho = rho_N)."""
    wz, wy, wx = freq_grid(dims)
    rho = np.sqrt(wz ** 2 + wy ** 2 + wx ** 2)
    return np.where(rho < RHO_N, radial_window(rho, N, gamma), 0.0)


# ---------------------------------------------------------------------------
# Orientation distribution A = B^k(theta / s_theta) (Sec. 3.1)
# ---------------------------------------------------------------------------
def bspline(x, k):
    """Centred cardinal B-spline B^k = B^{k-1} * B^0, B^0 the indicator of
    (-1/2, 1/2) (Sec. 3.1). Closed form of the k-fold convolution:
    B^k(x) = 1/k! sum_{j=0}^{k+1} (-1)^j C(k+1, j) (x + (k+1)/2 - j)_+^k."""
    x = np.asarray(x, dtype=np.float64)
    if k == 0:
        return np.where(np.abs(x) < 0.5, 1.0, 0.0)
    s = np.zeros_like(x)
    for j in range(k + 2):
        u = x + (k + 1) / 2.0 - j
        s = s + (-1.0) ** j * math.comb(k + 1, j) * np.where(u > 0, u, 0.0) ** k
    return s / math.factorial(k)


def bspline_knots_theta(k, s_theta):
    """Angles theta in (0, pi) where A(theta) = B^k(theta/s_theta) has a knot."""
    kn = sorted({abs(s_theta * (j - (k + 1) / 2.0)) for j in range(k + 2)})
    return [t for t in kn if 0.0 < t < math.pi]


def orientation_distribution(theta, k, s_theta):
    """A(theta) = B^k(theta / s_theta), theta in [0, pi] (Sec. 3.1)."""
    return bspline(np.asarray(theta, dtype=np.float64) / s_theta, k)


# ---------------------------------------------------------------------------
# Legendre polynomials (Bonnet recurrence)
# ---------------------------------------------------------------------------
def legendre_table(L, t):
    """P_0..P_L at t, shape (L+1,) + t.shape; (l+1)P_{l+1} = (2l+1)tP_l - lP_{l-1}."""
    t = np.asarray(t, dtype=np.float64)
    P = np.empty((L + 1,) + t.shape)
    P[0] = 1.0
    if L >= 1:
        P[1] = t
    for l in range(1, L):
        P[l + 1] = ((2 * l + 1) * t * P[l] - l * P[l - 1]) / (l + 1)
    return P


def legendre_series(c, t):
    """h(t) = sum_l c_l P_l(t)."""
    c = np.asarray(c, dtype=np.float64)
    P = legendre_table(len(c) - 1, t)
    return np.tensordot(c, P, axes=(0, 0))


# ---------------------------------------------------------------------------
# Orientation sets: icosahedron and its tessellations (Sec. 2.1)
# ---------------------------------------------------------------------------
def icosahedron():
    """12 unit vertices (cyclic permutations of (0, +-1, +-phi)) and 20 faces."""
    v = []
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            a = (0.0, s1, s2 * PHI)
            v += [a, (a[1], a[2], a[0]), (a[2], a[0], a[1])]
    V = np.array(v) / math.sqrt(1.0 + PHI * PHI)
    d = np.linalg.norm(V[:, None, :] - V[None, :, :], axis=-1)
    edge = d[d > 1e-9].min()
    adj = np.abs(d - edge) < 1e-9
    F = [(i, j, k) for i in range(12) for j in range(i + 1, 12) for k in range(j + 1, 12)
         if adj[i, j] and adj[j, k] and adj[i, k]]
    return V, F


def subdivide(V, F):
    """One edge-midpoint subdivision with projection onto S^2."""
    V = [np.asarray(x) for x in V]
    mid = {}

    def m(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            p = V[a] + V[b]
            V.append(p / np.linalg.norm(p))
            mid[key] = len(V) - 1
        return mid[key]

    F2 = []
    for a, b, c in F:
        ab, bc, ca = m(a, b), m(b, c), m(c, a)
        F2 += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.array(V), F2


_TOL = 1e-9


def _canonical_order(V):
    """Order of an antipodally closed set: the representatives (z > 0, or z = 0
    and y > 0, or z = y = 0 and x > 0) sorted by decreasing z, then by azimuth
    atan2(y, x) in (-pi, pi]; then their antipodes in the same order, so that
    orientation i + N_o/2 is -n_i."""
    def is_rep(p):
        x, y, z = p
        if z > _TOL:
            return True
        if abs(z) <= _TOL:
            return y > _TOL or (abs(y) <= _TOL and x > 0.0)
        return False

    def az(p):
        a = math.atan2(p[1], p[0])
        return math.pi if a <= -math.pi + _TOL else a

    def cmp(p, q):
        if abs(p[2] - q[2]) > _TOL:
            return -1 if p[2] > q[2] else 1
        ap, aq = az(p), az(q)
        return -1 if ap < aq else (1 if ap > aq else 0)

    reps = sorted([tuple(p) for p in V if is_rep(p)], key=functools.cmp_to_key(cmp))
    reps = np.array(reps)
    out = np.concatenate([reps, -reps], axis=0)
    assert out.shape[0] == V.shape[0], "orientation set is not antipodally closed"
    return out


def octahedron():
    """6 unit vertices +-e_x, +-e_y, +-e_z and the 8 faces (one per octant)."""
    V = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 1.0, 0], [0, -1.0, 0], [0, 0, 1.0], [0, 0, -1.0]])
    F = [(a, b, c) for a in (0, 1) for b in (2, 3) for c in (4, 5)]
    return V, F


def octa_orientations(subdiv):
    """Octahedron subdivided ``subdiv`` times (the other platonic-solid sampling
    of Sec. 2.1): 6, 18, 66, ... unit vectors, in canonical order. Unlike the
    icosahedral sets it is mapped onto itself by the 90-degree rotations
    about the coordinate axes."""
    V, F = octahedron()
    for _ in range(subdiv):
        V, F = subdivide(V, F)
    return _canonical_order(np.asarray(V))


def icosa_orientations(subdiv):
    """Icosahedron subdivided ``subdiv`` times: 12, 42, 162, ... unit vectors,
    both members of every antipodal pair kept, in canonical order."""
    V, F = icosahedron()
    for _ in range(subdiv):
        V, F = subdivide(V, F)
    return _canonical_order(np.asarray(V))


def icosa_tessellation(order):
    """Icosahedron of tessellation order nu: every face split into nu^2
    triangles (barycentric grid), points projected onto S^2; 10 nu^2 + 2
    points. This is the sampling the paper names for the SH fit (Sec. 3.2)."""
    V, F = icosahedron()
    pts = {}
    for a, b, c in F:
        for i in range(order + 1):
            for j in range(order + 1 - i):
                kk = order - i - j
                p = (i * V[a] + j * V[b] + kk * V[c]) / order
                p = p / np.linalg.norm(p)
                key = tuple(np.round(p * 1e9).astype(np.int64))
                pts[key] = p
    return np.array(list(pts.values()))


# ---------------------------------------------------------------------------
# Zonal SH fit of A (Sec. 3.2)
# ---------------------------------------------------------------------------
def fit_legendre_projection(profile, L, knots=(), nodes_per_piece=96):
    """b_l = (2l+1)/2 int_0^pi A(theta) P_l(cos theta) sin(theta) dtheta, by
    Gauss-Legendre quadrature in theta on pieces split at the knots of A.
    Returns b with A(arccos t) ~ sum_l b_l P_l(t)."""
    edges = [0.0] + [float(x) for x in knots] + [math.pi]
    xg, wg = np.polynomial.legendre.leggauss(nodes_per_piece)
    b = np.zeros(L + 1)
    for lo, hi in zip(edges[:-1], edges[1:]):
        th = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
        w = 0.5 * (hi - lo) * wg
        P = legendre_table(L, np.cos(th))
        b += P @ (w * profile(th) * np.sin(th))
    return b * (2.0 * np.arange(L + 1) + 1.0) / 2.0


def fit_legendre_lsq(profile, L, order=15):
    """Paper's route (Sec. 3.2): pseudo-inverse of the discretised inverse SHT
    restricted to the zonal harmonics Y_l^0, sampled on the icosahedron of
    tessellation order 15; then b_l = a_l sqrt((2l+1)/(4 pi)) converts the
    Y_l^0 coefficients a_l to the Legendre basis."""
    pts = icosa_tessellation(order)
    z = np.clip(pts[:, 2], -1.0, 1.0)
    norm = np.sqrt((2.0 * np.arange(L + 1) + 1.0) / (4.0 * math.pi))
    Y = (legendre_table(L, z) * norm[:, None]).T          # (points, L+1)
    a = np.linalg.pinv(Y) @ profile(np.arccos(z))
    return a * norm


def fit_coefficients(p: Params):
    """Legendre coefficients b_l of A(theta) = B^k(theta/s_theta)."""
    A = functools.partial(orientation_distribution, k=p.k, s_theta=p.s_theta)
    if p.fit_mode == 0:
        return fit_legendre_projection(A, p.L, bspline_knots_theta(p.k, p.s_theta))
    return fit_legendre_lsq(A, p.L)


def funk_antisym(b):
    """Line part c^e_l = 2 pi P_l(0) b_l (Funk transform, Sec. 3.2) and edge
    part c^o_l = (1 - (-1)^l) b_l (anti-symmetrisation, Sec. 3.2)."""
    b = np.asarray(b, dtype=np.float64)
    L = len(b) - 1
    P0 = legendre_table(L, np.array(0.0))
    l = np.arange(L + 1)
    ce = 2.0 * math.pi * P0 * b
    co = (1.0 - (-1.0) ** l) * b
    return ce, co


def normalise(c, n_o):
    """kappa c with kappa^2 = 1 / (N_o sum_l c_l^2/(2l+1)): the spherical
    mean of sum_i h(w.n_i)^2 becomes 1, the paper's aim M ~ 1 (Sec. 2,
    requirement 2 of Sec. 3)."""
    c = np.asarray(c, dtype=np.float64)
    l = np.arange(len(c))
    kappa = 1.0 / math.sqrt(n_o * np.sum(c * c / (2.0 * l + 1.0)))
    return kappa * c


def wavelet_coefficients(p: Params, n_o):
    """Normalised Legendre coefficients c of the angular part: for the cake
    wavelet h = h_Re + h_Im (Sec. 3.1, Eq. CakeWaveletRe and
    Eq. Antisymmetrize); for the plate detector h = A itself (Sec. 3.1,
    the construction before Eq. Antisymmetrize, Fig. 3)."""
    b = fit_coefficients(p)
    if p.profile == 1:
        return normalise(b, n_o)
    ce, co = funk_antisym(b)
    return normalise(ce + co, n_o)


# ---------------------------------------------------------------------------
# Wavelet bank psi_hat_i(w) = G(|w|) h(w_hat . n_i)  (Sec. 3.2, Eq. Rotationh
# in its zonal / addition-theorem form)
# ---------------------------------------------------------------------------
class Bank:
    """Everything the transform needs for one (dims, orientations, params)."""

    def __init__(self, dims, orients, p: Params = Params()):
        self.dims = tuple(int(d) for d in dims)
        self.orients = np.asarray(orients, dtype=np.float64)
        self.p = p
        self.c = wavelet_coefficients(p, len(self.orients))
        wz, wy, wx = freq_grid(self.dims)
        rho = np.sqrt(wz ** 2 + wy ** 2 + wx ** 2)
        self.G = radial_ball(self.dims, p.N, p.gamma)
        safe = np.where(rho > 0, rho, 1.0)
        self.what = (np.broadcast_to(wz / safe, self.dims),
                     np.broadcast_to(wy / safe, self.dims),
                     np.broadcast_to(wx / safe, self.dims))
        self.zero = rho == 0
        self._M = None

    @property
    def n_o(self):
        return len(self.orients)

    def angular(self, i):
        """h(w_hat . n_i), with h(.) = c_0 at w = 0."""
        nx, ny, nz = self.orients[i]
        t = self.what[0] * nz + self.what[1] * ny + self.what[2] * nx
        h = legendre_series(self.c, np.clip(t, -1.0, 1.0))
        return np.where(self.zero, self.c[0], h)

    def psi_hat(self, i):
        """Real Fourier multiplier psi_hat_i on the DFT grid (nz, ny, nx)."""
        return self.G * self.angular(i)

    def M_part(self, orients_idx):
        """sum over the given orientations of |psi_hat_i|^2 (M splits into such
        parts over a partition of the orientations)."""
        M = np.zeros(self.dims)
        for i in orients_idx:
            M += self.psi_hat(i) ** 2
        return M

    def M(self):
        """M_psi^d = sum_i |psi_hat_i|^2 (Sec. 2.1; constants absorbed in kappa)."""
        if self._M is None:
            self._M = self.M_part(range(self.n_o))
        return self._M

    def set_M(self, M):
        """Installs M summed from M_part over a partition of the orientations
        (computed elsewhere, e.g. in parallel)."""
        M = np.asarray(M, dtype=np.float64)
        assert M.shape == self.dims
        self._M = M

    def M_inv(self):
        """1 / max(M, eps) where M > 0, else 0 (Sec. 3.1 clamp)."""
        M = self.M()
        return np.where(M > 0, 1.0 / np.maximum(M, self.p.eps), 0.0)


# ---------------------------------------------------------------------------
# The transform (Sec. 2.1, Eq. construction1Discrete / Reconstruction1Discrete)
# ---------------------------------------------------------------------------
def forward_one(fhat, bank: Bank, i):
    """U_i = IDFT[ f_hat * conj(psi_hat_i) ]: the correlation conj(psi_i) * f."""
    return np.fft.ifftn(fhat * np.conj(bank.psi_hat(i)))


def forward(f, bank: Bank, orients_idx=None):
    """Orientation score U (N_o, nz, ny, nx) complex128 of a 3D volume f."""
    fhat = np.fft.fftn(np.asarray(f, dtype=np.float64))
    idx = range(bank.n_o) if orients_idx is None else orients_idx
    return np.stack([forward_one(fhat, bank, i) for i in idx])


def backproject(U, bank: Bank, orients_idx=None):
    """sum_i psi_hat_i * DFT(U_i): the DFT of sum_i (psi_check_i * U_i); with
    ``orients_idx`` the sum over those orientations only, U[j] holding
    orientation orients_idx[j] (the orientation sum splits into such parts)."""
    idx = range(bank.n_o) if orients_idx is None else orients_idx
    acc = np.zeros(bank.dims, dtype=np.complex128)
    for j, i in enumerate(idx):
        acc += bank.psi_hat(i) * np.fft.fftn(U[j])
    return acc


def reconstruct(acc, bank: Bank, real=True):
    """IDFT[ max(M, eps)^-1 acc ] of an orientation sum acc = sum_i psi_hat_i
    DFT(U_i) (the last step of Eq. Reconstruction1Discrete)."""
    f = np.fft.ifftn(acc * bank.M_inv())
    return f.real if real else f


def inverse(U, bank: Bank, real=True):
    """Exact reconstruction f = IDFT[ max(M, eps)^-1 sum_i psi_hat_i DFT(U_i) ]
    (Eq. Reconstruction1Discrete with the Sec. 3.1 clamp); the real part is
    the reconstructed real image."""
    return reconstruct(backproject(U, bank), bank, real)


def adjoint(G, bank: Bank, real=True):
    """W^* G = sum_i IDFT[ psi_hat_i DFT(G_i) ] (the adjoint of the forward map
    for the l2 inner products, used in Sec. 4.1 and App. A); for a real image
    the gradient is its real part."""
    g = np.fft.ifftn(backproject(G, bank))
    return g.real if real else g


def orientation_pairs(orients, tol=1e-9):
    """Index of the antipode of each orientation, or -1."""
    o = np.asarray(orients)
    out = np.full(len(o), -1, dtype=np.int64)
    for i in range(len(o)):
        d = np.abs(o + o[i]).max(axis=1)
        j = np.nonzero(d < tol)[0]
        if len(j):
            out[i] = int(j[0])
    return out


# ---------------------------------------------------------------------------
# Approximate reconstruction and projection (Sec. 2.1, Eq.
# Reconstruction2Approximation; App. A, corollary on P_psi)
# ---------------------------------------------------------------------------
def approx_weight(bank: Bank):
    """Discrete weight of the orientation integral in Eq.
    Reconstruction2Approximation: the paper's condition that the orientation
    integral of the wavelets' Fourier transforms be ~1 is met exactly at w = 0,
    where every psi_hat_i equals c_0, so d sigma -> 1 / (N_o c_0)."""
    return 1.0 / (bank.n_o * bank.c[0])


def approx_reconstruct(U, bank: Bank):
    """f ~ Re sum_i U_i d sigma (Eq. Reconstruction2Approximation)."""
    acc = np.zeros(bank.dims, dtype=np.float64)
    for i in range(bank.n_o):
        acc += np.real(U[i])
    return approx_weight(bank) * acc


def project(U, bank: Bank):
    """P_psi U = W W^{*,ext} U: the exact reconstruction (the adjoint extended
    to the embedding space with the M_psi inner product) followed by the
    forward transform (App. A, corollary)."""
    return forward(inverse(U, bank), bank)


# ---------------------------------------------------------------------------
# Weighted energy of a score (Sec. 2, the norm-preservation identity)
# ---------------------------------------------------------------------------
def weighted_energy(U, w=None):
    """L = sum_e w_e |U_e|^2: the squared L_2(R^3 x S^2) norm of a score on
    the grid (Sec. 2, ||W f||^2 in the norm-preservation identity), with real
    weights w per element (w = 1 when None)."""
    a = np.abs(np.asarray(U, dtype=np.complex128)) ** 2
    if w is not None:
        a = np.asarray(w, dtype=np.float64) * a
    return float(np.sum(a))


def weighted_energy_grad(U, w=None, g=1.0):
    """g dL/dconj(U) x 2 = 2 g w U: the gradient of weighted_energy in the
    convention of PyTorch for complex inputs (the one os3d adjoint consumes)."""
    U = np.asarray(U, dtype=np.complex128)
    ww = 1.0 if w is None else np.asarray(w, dtype=np.float64)
    return 2.0 * g * ww * U


# ---------------------------------------------------------------------------
# Score-domain processing Upsilon = W^{*,ext} o Phi o W (Sec. 4.1)
# ---------------------------------------------------------------------------
def soft_threshold(U, power=1.5):
    """Phi(U) = |U|^p sgn(U) (Sec. 4.1, Fig. 6), applied to the real part
    (line response) and the imaginary part (edge response) separately."""
    U = np.asarray(U)
    re = np.sign(U.real) * np.abs(U.real) ** power
    im = np.sign(U.imag) * np.abs(U.imag) ** power
    return re + 1j * im


def upsilon(f, bank: Bank, power=1.5):
    """Upsilon f = W^{*,ext} Phi W f = W^* P_psi Phi W f (Sec. 4.1), with the
    soft threshold Phi and the exact (clamped) reconstruction as W^{*,ext}."""
    return inverse(soft_threshold(forward(f, bank), power), bank)


# ---------------------------------------------------------------------------
# Linear left-invariant diffusion on R^3 x| S^2 (Sec. 4.1, the flows with a
# constant diagonal D_ij; the adaptive choice of D_ij is not part of the paper)
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Diffusion:
    """dW/dt = [D11 (A1^2 + A2^2) + D33 A3^2 + D44 (A4^2 + A5^2)] W. For a
    function of (x, n) the left-invariant fields give A3 = n . grad_x,
    A1^2 + A2^2 = Laplace_x - (n . grad_x)^2 and A4^2 + A5^2 = the
    Laplace-Beltrami operator of S^2 in n at fixed x (D66 is irrelevant by the
    equivalence relation of Sec. 4.1)."""
    t: float = 10.0       # diffusion time (Fig. 5 uses t = 10)
    steps: int = 8        # Strang steps
    D11: float = 0.0      # spatial, perpendicular to n
    D33: float = 1.0      # spatial, along n
    D44: float = 0.01     # angular
    sh_degree: int = 0    # degree of the discrete Laplace-Beltrami; 0 = the largest
                          # l whose (l + 1)^2 harmonics are independent on the set


def _sh_full_rank(lmax, V):
    s = np.linalg.svd(real_sh_basis(lmax, V)[0], compute_uv=False)
    return s[-1] > 1e-6 * s[0]


def sh_degree_for(V, sh_degree=0):
    """The degree of the discrete Laplace-Beltrami operator: the given one, or
    the largest l with (l + 1)^2 <= N_o whose real harmonics are linearly
    independent on the orientation set (on the subdivided octahedra a few
    harmonics of the top degree coincide)."""
    if sh_degree > 0:
        return sh_degree
    l = 0
    while (l + 2) ** 2 <= len(V):
        l += 1
    while l > 0 and not _sh_full_rank(l, V):
        l -= 1
    return l


def real_sh_basis(lmax, V):
    """Orthonormal real spherical harmonics up to degree lmax at the unit
    vectors V: N_lm P_l^|m|(z) cos(m phi) or sin(|m| phi), with N_lm^2 =
    (2 - delta_m0) (2l+1)/(4 pi) (l-|m|)!/(l+|m|)!; and the degree of every
    column. (Unit norms on the sphere keep a harmonic that vanishes on the
    set visible as a near-zero column.)"""
    V = np.asarray(V, dtype=np.float64)
    z = np.clip(V[:, 2], -1.0, 1.0)
    ph = np.arctan2(V[:, 1], V[:, 0])
    cols, deg = [], []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            nrm = math.sqrt((2.0 - (m == 0)) * (2 * l + 1) / (4.0 * math.pi)
                            * math.factorial(l - am) / math.factorial(l + am))
            P = scipy.special.lpmv(am, l, z)
            cols.append(nrm * P * (np.sin(am * ph) if m < 0 else np.cos(am * ph)))
            deg.append(l)
    return np.stack(cols, axis=1), np.array(deg)


def angular_laplacian(V, lmax):
    """Discrete Laplace-Beltrami operator on the orientation set: fit the
    values by real spherical harmonics up to degree lmax (pseudo-inverse,
    as for the profile fit of Sec. 3.2), scale degree l by -l(l+1), evaluate."""
    Y, deg = real_sh_basis(lmax, V)
    return Y @ np.diag(-(deg * (deg + 1.0))) @ np.linalg.pinv(Y)


def spatial_rates(bank: Bank, D: Diffusion):
    """r_i(w) = D11 (|w|^2 - (w.n_i)^2) + D33 (w.n_i)^2: the symbol of
    -[D11 (A1^2 + A2^2) + D33 A3^2] for orientation i, (N_o, nz, ny, nx)."""
    wz, wy, wx = freq_grid(bank.dims)
    r2 = wz ** 2 + wy ** 2 + wx ** 2
    out = np.empty((bank.n_o,) + bank.dims)
    for i, (nx, ny, nz) in enumerate(bank.orients):
        a2 = (wx * nx + wy * ny + wz * nz) ** 2
        out[i] = D.D11 * (r2 - a2) + D.D33 * a2
    return out


def diffuse(U, bank: Bank, D: Diffusion):
    """Phi_t U for a stored score: in the Fourier domain of x, K Strang steps
    of the spatial part exp(-dt/2 r_i) (exact per orientation), the angular
    part exp(dt D44 L) (a matrix over the orientations) and the spatial part
    again, dt = t / K."""
    K = int(D.steps)
    dt = D.t / K
    half = np.exp(-0.5 * dt * spatial_rates(bank, D))
    EA = scipy.linalg.expm(dt * D.D44 * angular_laplacian(bank.orients,
                                                           sh_degree_for(bank.orients, D.sh_degree)))
    Uh = np.stack([np.fft.fftn(U[i]) for i in range(bank.n_o)])
    for _ in range(K):
        Uh = half * Uh
        Uh = np.tensordot(EA, Uh, axes=(1, 0))
        Uh = half * Uh
    return np.stack([np.fft.ifftn(Uh[i]) for i in range(bank.n_o)])


def enhance_linear(f, bank: Bank, D: Diffusion):
    """Upsilon f = W^{*,ext} Phi_t W f with the linear diffusion Phi_t
    (Sec. 4.1): forward transform, evolution of the score, exact
    reconstruction."""
    return inverse(diffuse(forward(f, bank), bank, D), bank)
