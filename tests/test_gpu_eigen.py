"""The low-mode eigensolver of H_w = g5 D_w(-rho) and the deflated sign
function (Sec. 2.3) against the FP64 oracle's dense eigendecomposition:
eigenvalues, eigenvectors up to a phase, residuals recomputed by the oracle,
and eps(H_w) v against the exact sign Z sign(Lambda) Z^+ v."""
import numpy as np
import pytest

from helpers import ensure_library, rel_err
from paper_2201_09004_b300 import synth

pytestmark = pytest.mark.gpu

RHO, LMAX = 1.5, 10.5


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


@pytest.mark.parametrize("dims,nev", [((2, 2, 2, 2), 4), ((4, 4, 4, 4), 8)])
def test_low_modes_match_dense_eigendecomposition(L, orc, dims, nev):
    lat, U = make(L, dims, 91)
    ref, Zref, w = orc.hw_low_modes(dims, U, RHO, nev + 6)
    cut = float(np.abs(ref[nev + 4]))  # the filter edge a few modes above the wanted ones
    ev, Z, info = lat.hw_eigensolve(RHO, nev, cut, LMAX, tol=1e-10, degree=16)
    assert info["converged"] == 1, info
    assert np.allclose(ev, ref[:nev], atol=1e-10, rtol=0), (ev, ref[:nev])
    hw = orc.hermitian_wilson(dims, U, RHO)
    for i in range(nev):
        z = Z[i]
        assert abs(np.linalg.norm(z) - 1.0) < 1e-10
        assert np.linalg.norm(hw(z) - ev[i] * z) < 1e-9
        # eigenvector up to a phase where |lambda_i| is separated from its neighbours
        gaps = np.abs(np.abs(w) - abs(ref[i]))
        if np.sort(gaps)[1] > 1e-6 * max(1.0, abs(ref[i])):
            assert abs(abs(np.vdot(Zref[i].ravel(), z.ravel())) - 1.0) < 1e-8


def test_deflated_sign_matches_exact_sign(L, orc):
    dims = (4, 4, 4, 4)
    lat, U = make(L, dims, 93)
    nev = 6
    ref, _, w = orc.hw_low_modes(dims, U, RHO, nev + 1)
    ev, Z, info = lat.hw_eigensolve(RHO, nev, float(np.abs(ref[nev]) * 1.5), LMAX, tol=1e-11, degree=16)
    assert info["converged"] == 1, info
    v = synth.gaussian_field(dims, 94).numpy()
    exact = orc.sign_exact(dims, U, RHO, v)
    lmin = 0.99 * float(np.abs(ref[nev]))  # below the spectrum left after deflation
    got, sinfo = lat.overlap_sign_apply_deflated(RHO, lmin, LMAX, 1e-10, ev, Z, v)
    assert rel_err(got, exact) < 1e-8
    # deflation lets the polynomial start at the (nev+1)-th mode: fewer terms than
    # covering the lowest mode at the same bound
    _, plain = lat.overlap_sign_apply(RHO, 0.99 * float(np.abs(ref[0])), LMAX, 1e-10, v, prec=L.F32X2)
    assert sinfo["order"] < plain["order"]


def test_eigensolve_argument_errors(L):
    lat, _ = make(L, (2, 2, 2, 2), 95)
    with pytest.raises(L.LqError):
        lat.hw_eigensolve(RHO, 0, 1.0, LMAX)
    with pytest.raises(L.LqError):
        lat.hw_eigensolve(RHO, 4, 11.0, LMAX)       # lambda_cut above lambda_max
    with pytest.raises(L.LqError):
        lat.hw_eigensolve(RHO, 4, 1.0, LMAX, nkv=5)  # basis smaller than nev + 2
