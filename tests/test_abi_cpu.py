"""CPU checks of the C-ABI library: it builds, loads, exports what the header
declares, and its host-only logic (orientation sets, argument checks)
matches the oracle. No CUDA compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import os3d_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1505_07690_gb300 import build, os3d
    build.build()
    return os3d.lib()


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "os3d.h")).read()
    names = set(re.findall(r"\b(os3d_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n


def test_orientations_match_oracle(L):
    from paper_1505_07690_gb300 import os3d
    for s in (0, 1, 2, 3):
        a = os3d.os3d_icosa_orientations(s)
        b = O.icosa_orientations(s)
        assert a.shape == b.shape
        assert np.abs(a - b).max() < 1e-12


def test_octahedral_orientations_match_oracle(L):
    from paper_1505_07690_gb300 import os3d
    for s in (0, 1, 2, 3):
        a = os3d.os3d_octa_orientations(s)
        b = O.octa_orientations(s)
        assert a.shape == b.shape
        assert np.abs(a - b).max() < 1e-12
    n = ctypes.c_int(0)
    assert L.os3d_octa_orientations(6, None, 0, ctypes.byref(n)) == 1


@pytest.mark.parametrize("make,sub", [(O.icosa_orientations, 0), (O.icosa_orientations, 1),
                                      (O.octa_orientations, 1), (O.octa_orientations, 2),
                                      (O.octa_orientations, 0)])
def test_angular_propagator_matches_oracle(L, make, sub):
    """Host FP64 closed form exp(tau L) = I + Y (e^{tau Lambda} - I) Y^+ against
    the oracle's matrix exponential of its Laplace-Beltrami matrix."""
    import scipy.linalg
    from paper_1505_07690_gb300 import os3d
    V = make(sub)
    for tau in (0.0, 0.05, 0.7):
        E, deg = os3d.os3d_angular_propagator(V, tau)
        assert deg == O.sh_degree_for(V)
        ref = scipy.linalg.expm(tau * O.angular_laplacian(V, deg))
        assert np.abs(E - ref).max() < 1e-10
    E, deg = os3d.os3d_angular_propagator(V, 0.3, sh_degree=1)
    assert deg == 1
    assert np.abs(E - scipy.linalg.expm(0.3 * O.angular_laplacian(V, 1))).max() < 1e-10


def test_orientation_capacity_and_range(L):
    n = ctypes.c_int(0)
    buf = (ctypes.c_double * 30)()
    assert L.os3d_icosa_orientations(1, buf, 10, ctypes.byref(n)) == 1   # EINVAL
    assert n.value == 42
    assert L.os3d_icosa_orientations(7, buf, 10, ctypes.byref(n)) == 1


def test_default_params_and_status_strings(L):
    from paper_1505_07690_gb300 import os3d
    p = os3d.os3d_default_params()
    assert (p.k, p.s_theta, p.L, p.N, p.gamma, p.eps, p.fit_mode) == (2, 0.7, 16, 8, 0.8, 1e-4, 1)
    for s in range(6):
        assert len(L.os3d_status_string(s)) > 0


def test_argument_errors_before_any_launch(L):
    from paper_1505_07690_gb300 import os3d
    p = os3d.os3d_default_params()
    V = O.icosa_orientations(1)
    Vp = V.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p(0)
    dims = (ctypes.c_int * 3)(32, 32, 32)
    # NULL orientation pointer, n_o < 1
    assert L.os3d_make_wavelets(dims, None, 42, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert L.os3d_make_wavelets(dims, Vp, 0, ctypes.byref(p), None, ctypes.byref(h)) == 1
    # non-unit orientation
    bad = V.copy(); bad[3] *= 1.01
    assert L.os3d_make_wavelets(dims, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 42,
                                ctypes.byref(p), None, ctypes.byref(h)) == 1
    # parameters out of range
    for field, val in (("L", 33), ("eps", 0.0), ("gamma", 1.0), ("k", 9), ("fit_mode", 2),
                       ("s_theta", -1.0), ("block_slots", 13), ("profile", 2)):
        q = os3d.os3d_default_params(**{field: val})
        assert L.os3d_make_wavelets(dims, Vp, 42, ctypes.byref(q), None, ctypes.byref(h)) == 1, field
    # grid without a compiled plan
    for d in ((30, 32, 32), (32, 32, 40), (512, 64, 64), (32, 64, 80)):
        dd = (ctypes.c_int * 3)(*d)
        st = L.os3d_make_wavelets(dd, Vp, 42, ctypes.byref(p), None, ctypes.byref(h))
        assert st == 5, d
    # transform calls on a NULL bank
    assert L.os3d_forward(None, None, 1, None, 0, None, None) == 1
    assert L.os3d_inverse(None, None, 0, 1, None, None, None) == 1
    assert L.os3d_adjoint(None, None, 0, 1, None, None, None) == 1
    assert L.os3d_adjoint_weighted(None, None, None, None, 0, 1, None, None, None) == 1
    assert L.os3d_score_energy_grad(None, None, None, None, 1, None, None, None, 0, None,
                                    None) == 1
    n = ctypes.c_size_t(0)
    assert L.os3d_score_energy_scratch(None, 1, ctypes.byref(n)) == 1
    assert L.os3d_bank_info(None, None, None) == 1
    assert L.os3d_destroy_bank(None) == 1
    assert L.os3d_approx_reconstruct(None, None, 0, 1, None, None) == 1
    assert L.os3d_project(None, None, 0, 1, None, None, None) == 1
    assert L.os3d_upsilon(None, None, 1, None, 1.5, None, None) == 1
    # soft threshold: pointers, count, alignment and exponent are checked first
    buf = ctypes.create_string_buffer(64)
    a16 = (ctypes.addressof(buf) + 15) // 16 * 16
    assert L.os3d_soft_threshold(None, None, 0, 4, 1.5, None) == 1
    assert L.os3d_soft_threshold(a16, a16, 0, 6, 1.5, None) == 1       # not a multiple of 4
    assert L.os3d_soft_threshold(a16 + 8, a16 + 8, 0, 4, 1.5, None) == 1  # misaligned
    for pw in (0.0, -1.0, float("inf"), float("nan")):
        assert L.os3d_soft_threshold(a16, a16, 0, 4, pw, None) == 1
    assert L.os3d_soft_threshold(a16, a16, 2, 4, 1.5, None) == 1       # unknown udtype
    assert L.os3d_soft_threshold(a16, a16, 0, 0, 1.5, None) == 0       # nothing to do
    # weighted energy and its gradient: count, pointers, alignment, udtype
    assert L.os3d_weighted_energy(a16, None, 0, 6, a16, None, None) == 1      # count % 4
    assert L.os3d_weighted_energy(a16, None, 0, -4, a16, None, None) == 1
    assert L.os3d_weighted_energy(a16, None, 0, 4, None, None, None) == 1     # no scratch
    assert L.os3d_weighted_energy(None, None, 0, 4, a16, None, None) == 1     # no score
    assert L.os3d_weighted_energy(a16 + 8, None, 0, 4, a16, None, None) == 1  # misaligned U
    assert L.os3d_weighted_energy(a16, a16 + 4, 0, 4, a16, None, None) == 1   # misaligned w
    assert L.os3d_weighted_energy(a16, None, 0, 4, a16 + 4, None, None) == 1  # scratch
    assert L.os3d_weighted_energy(a16, None, 2, 4, a16, None, None) == 1      # udtype
    assert L.os3d_weighted_energy_grad(a16, None, 0, 4, None, a16, None) == 1  # no g
    assert L.os3d_weighted_energy_grad(a16, None, 0, 4, a16, None, None) == 1  # no G
    assert L.os3d_weighted_energy_grad(a16, None, 0, 4, a16, a16 + 8, None) == 1
    assert L.os3d_weighted_energy_grad(a16, None, 0, 5, a16, a16, None) == 1
    assert L.os3d_weighted_energy_grad(a16, None, 2, 4, a16, a16, None) == 1
    assert L.os3d_weighted_energy_grad(None, None, 0, 0, None, None, None) == 0  # nothing to do
    assert L.os3d_scale_by(a16, a16, -1, a16, None) == 1
    assert L.os3d_scale_by(a16 + 4, a16, 4, a16, None) == 1
    assert L.os3d_scale_by(a16, a16, 4, None, None) == 1
    assert L.os3d_scale_by(None, None, 0, None, None) == 0
    d = os3d.os3d_default_diffusion()
    assert (d.t, d.steps, d.D11, d.D33, d.D44, d.sh_degree) == (10.0, 8, 0.0, 1.0, 0.01, 0)
    assert L.os3d_enhance_linear(None, None, 1, None, ctypes.byref(d), None, None) == 1
    E = (ctypes.c_double * 36)()
    Vp6 = O.octa_orientations(0)
    assert L.os3d_angular_propagator(None, 6, 0, 0.1, E, None) == 1
    assert L.os3d_angular_propagator(Vp6.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 6, 0,
                                     -0.1, E, None) == 1
    # degree 2 needs 9 independent harmonics: impossible on 6 points
    assert L.os3d_angular_propagator(Vp6.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 6, 2,
                                     0.1, E, None) == 1


def test_injected_allocation_failure(L, monkeypatch):
    from paper_1505_07690_gb300 import os3d
    p = os3d.os3d_default_params()
    V = O.icosa_orientations(1)
    h = ctypes.c_void_p(0)
    dims = (ctypes.c_int * 3)(32, 32, 32)
    monkeypatch.setenv("OS3D_FAULT", "alloc")
    st = L.os3d_make_wavelets(dims, V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 42,
                              ctypes.byref(p), None, ctypes.byref(h))
    assert st == 2 and not h.value


def test_server_config_checked_before_any_cuda_call(L):
    from paper_1505_07690_gb300 import os3d
    h = ctypes.c_void_p(0)
    assert os3d.os3d_server_default_config().use_graphs == 1
    assert L.os3d_server_stats(None, None, None, None) == 1
    for field, val in (("max_inflight", 0), ("max_inflight", 65), ("udtype", 3), ("arena_bytes", 0),
                       ("use_graphs", 2)):
        c = os3d.os3d_server_default_config(**{field: val})
        assert L.os3d_server_create(ctypes.byref(c), None, ctypes.byref(h)) == 1, field
    assert L.os3d_server_destroy(None) == 1
    assert L.os3d_server_wait(None, 1, 1.0, None) == 1
