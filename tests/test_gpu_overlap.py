"""Parity of the overlap building blocks (Sec. 2.3) with the FP64 oracle:
the fused g5 D_w(-rho) kernel, and the Chebyshev/Clenshaw sign function of
g5 D_w(-rho) against the oracle's evaluation and against the exact sign from a
dense eigendecomposition on 2^4."""
import numpy as np
import pytest

from helpers import TOL, ensure_library, rel_err
from paper_2201_09004_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    ensure_library()
    from paper_2201_09004_b300 import lib
    return lib


def make(L, dims, seed):
    U = synth.thin_links(dims, seed, 0.3).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.THIN, U)
    return lat, U


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 4, 6)])
@pytest.mark.parametrize("prec", [0, 3, 1])
def test_gamma5_dw_matches_oracle(L, orc, dims, prec):
    lat, U = make(L, dims, 81)
    v = synth.gaussian_field(dims, 82).numpy()
    ref = orc.hermitian_wilson(dims, U, 1.5)(v)
    got = lat.gamma5_dw_apply(1.5, v, prec=prec)
    assert rel_err(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (3, 1e-10), (1, 2e-4)])
def test_overlap_sign_matches_oracle(L, orc, prec, tol):
    """Same interval and bound on both sides: the GPU Clenshaw evaluation (about two
    hundred terms, two g5 D_w applications each) equals the oracle's. lambda_max is
    the bound |4 - rho| + 8 of |g5 D_w(-rho)| (eight hops of norm one), so the
    polynomial is never evaluated outside [-1, 1], where it grows without bound."""
    dims = (4, 4, 4, 4)
    lat, U = make(L, dims, 83)
    v = synth.gaussian_field(dims, 84).numpy()
    lmin, lmax, delta = 0.3, 2.5 + 8.0, 1e-6
    got, info = lat.overlap_sign_apply(1.5, lmin, lmax, delta, v, prec=prec)
    c, dev = orc.chebyshev_sign_coeffs(lmin / lmax, delta)
    assert info["order"] == len(c) and info["max_deviation"] <= delta
    ref = orc.overlap_sign(orc.hermitian_wilson(dims, U, 1.5), v, lmin, lmax, c)
    assert rel_err(got, ref) < tol


def test_overlap_sign_equals_exact_sign_2x4(L, orc):
    dims, rho, delta = (2, 2, 2, 2), 1.5, 1e-6
    lat, U = make(L, dims, 85)
    hw = orc.hermitian_wilson(dims, U, rho)
    shape = (2, 2, 2, 2, 4, 3)
    n = 192
    H = np.zeros((n, n), dtype=complex)
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        H[:, j] = hw(e.reshape(shape)).ravel()
    lam, V = np.linalg.eigh(H)
    lmin, lmax = 0.9 * np.min(np.abs(lam)), 1.1 * np.max(np.abs(lam))
    v = synth.gaussian_field(dims, 86).numpy()
    exact = (V @ (np.sign(lam) * (V.conj().T @ v.ravel()))).reshape(shape)
    got, info = lat.overlap_sign_apply(rho, lmin, lmax, delta, v, prec=0)
    assert np.linalg.norm(got - exact) <= 2 * delta * np.linalg.norm(v)
    # the overlap operator D_ov = (1 + g5 eps(H_w)) / rho then obeys Ginsparg-Wilson:
    # g5 D + D g5 = rho D g5 D, checked on v through eps^2 = 1
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[:, None]
    eps_v = got
    eps_g5v, _ = lat.overlap_sign_apply(rho, lmin, lmax, delta, g5 * v, prec=0)
    Dv = (v + g5 * eps_v) / rho
    Dg5v = (g5 * v + g5 * eps_g5v) / rho
    lhs = g5 * Dv + Dg5v
    w = g5 * Dv
    eps_w, _ = lat.overlap_sign_apply(rho, lmin, lmax, delta, w, prec=0)
    rhs = w + g5 * eps_w  # rho D (g5 D v)
    assert np.linalg.norm(lhs - rhs) <= 20 * delta * np.linalg.norm(v)
