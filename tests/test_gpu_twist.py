"""The scalar reading of the complex mass (Sec. 2.1 Eq. 1: m_cri + omega taken
literally as (4+m) + i mu instead of the twisted (4+m) + i mu g5) against the
FP64 oracle's twist_mode = 1: the full operator and its adjoint, the even-odd
Schur operator, and mixed-precision solves (oracle true residual <= 1e-10);
the twisted multi-shift solve, which needs the g5 twist, refuses it.
"""
import numpy as np
import pytest

from helpers import TOL, ensure_library, parity_mask, rel_err
from paper_2201_09004_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    ensure_library()
    from paper_2201_09004_b300 import lib
    return lib


def make(L, dims, seed, c_sw=None):
    U = synth.thin_links(dims, seed).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.THIN, U)
    if c_sw is not None:
        lat.load_clover(c_sw)
    return lat, U


def schur_scalar_reference(orc, dims, U, C, m, mu, v_even, dagger=False):
    """A_ee v - H_eo A_oo^{-1} H_oe v with A = (4+m) + i mu + C (adjoint: -mu),
    from oracle pieces; A^{-1} by a dense 12x12 solve per site."""
    mask = parity_mask(dims)
    A = ((4 + m) + 1j * (-mu if dagger else mu)) * np.eye(12, dtype=complex)
    Afull = np.broadcast_to(A, mask.shape + (12, 12)).copy()
    if C is not None:
        Afull = Afull + C
    W = orc.Wilson(dims, U, 0.0, 0.0)
    v = np.where((mask == 0)[..., None, None], v_even, 0)
    h = W.hop(v, dagger=dagger)
    t = np.linalg.solve(Afull, h.reshape(h.shape[:4] + (12,))[..., None])[..., 0].reshape(h.shape)
    t = np.where((mask == 1)[..., None, None], t, 0)
    h2 = W.hop(t, dagger=dagger)
    av = (Afull @ v.reshape(v.shape[:4] + (12, 1)))[..., 0].reshape(v.shape)
    return np.where((mask == 0)[..., None, None], av - h2, 0)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("clover", [False, True])
def test_scalar_twist_full_operator(L, orc, prec, clover):
    dims = (4, 4, 4, 6)
    lat, U = make(L, dims, 21, c_sw=1.05 if clover else None)
    C = orc.clover(dims, U, 1.05) if clover else None
    action = L.WILSON_TM_CLOVER if clover else L.WILSON_TM
    op = L.op_params(action, 0.05, 0.1, c_sw=1.05, twist_mode=L.TWIST_SCALAR)
    psi = synth.gaussian_field(dims, 22).numpy()
    for dagger in (False, True):
        ref = orc.Wilson(dims, U, 0.05, 0.1, clover=C, twist_mode=1).apply(psi, dagger=dagger)
        got = lat.operator_apply(op, psi, form=L.OP_FULL, dagger=dagger, prec=prec)
        assert rel_err(got, ref) < TOL[prec], (prec, clover, dagger)
        # the g5 twist gives a different operator on the same lattice
        g5 = orc.Wilson(dims, U, 0.05, 0.1, clover=C, twist_mode=0).apply(psi, dagger=dagger)
        assert rel_err(got, g5) > 1e-3


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("clover", [False, True])
def test_scalar_twist_schur_operator(L, orc, prec, clover):
    dims = (4, 4, 4, 6)
    lat, U = make(L, dims, 31, c_sw=1.05 if clover else None)
    C = orc.clover(dims, U, 1.05) if clover else None
    action = L.WILSON_TM_CLOVER if clover else L.WILSON_TM
    op = L.op_params(action, 0.05, 0.1, c_sw=1.05, twist_mode=L.TWIST_SCALAR)
    v = synth.gaussian_field(dims, 32).numpy()
    mask = parity_mask(dims)
    for dagger in (False, True):
        ref = schur_scalar_reference(orc, dims, U, C, 0.05, 0.1, v, dagger=dagger)
        got = lat.operator_apply(op, v, form=L.OP_SCHUR, dagger=dagger, prec=prec)
        assert np.all(got[mask == 1] == 0)
        assert rel_err(got, ref) < 10 * TOL[prec], (prec, clover, dagger)


@pytest.mark.parametrize("solver", ["cgnr", "bicgstab"])
@pytest.mark.parametrize("prec", [1, 2])
def test_scalar_twist_mixed_solves(L, orc, solver, prec):
    dims = (4, 4, 4, 8)
    lat, U = make(L, dims, 41, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05, twist_mode=L.TWIST_SCALAR)
    bs = [synth.z2_source(dims, 42 + k).numpy() for k in range(3)]
    kind = L.MIXED_CGNR if solver == "cgnr" else L.BICGSTAB
    xs, info = lat.solve(op, L.solve_params(solver=kind, tol=1e-10, prec_sloppy=prec), bs)
    M = orc.Wilson(dims, U, 0.05, 0.1, clover=C, twist_mode=1)
    for b, x, i in zip(bs, xs, info):
        assert i["status"] == 0, i
        assert np.linalg.norm(b - M.apply(x)) / np.linalg.norm(b) <= 1e-10


def test_scalar_twist_multishift_is_refused(L):
    dims = (4, 4, 4, 4)
    lat, _ = make(L, dims, 51)
    op = L.op_params(L.WILSON_TM, 0.05, 0.0, twist_mode=L.TWIST_SCALAR)
    b = synth.z2_source(dims, 52).numpy()
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=L.F32, masses=[0.01, 0.02])
    with pytest.raises(L.LqError) as e:
        lat.solve(op, sp, [b])
    assert "g5 twist" in str(e.value)
