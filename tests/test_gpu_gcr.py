"""Restarted GCR directly on the even-odd Schur operator (the paper's GPU
twisted-mass solver family, Sec. 2.1 and Table 2), mixed precision with FP64
defect correction, against the FP64 oracle: every solution's true residual of
the full system, recomputed by the oracle, is <= 1e-10, and equals the CGNR
solution within that accuracy; ragged restart lengths and several right-hand
sides; argument errors.
"""
import numpy as np
import pytest

from helpers import ensure_library
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


def true_residual(orc, dims, U, C, m, mu, b, x):
    r = b - orc.Wilson(dims, U, m, mu, clover=C).apply(x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("clover", [False, True])
def test_gcr_single_rhs(L, orc, prec, clover):
    dims = (4, 4, 4, 8)
    lat, U = make(L, dims, 61, c_sw=1.05 if clover else None)
    C = orc.clover(dims, U, 1.05) if clover else None
    action = L.WILSON_TM_CLOVER if clover else L.WILSON_TM
    op = L.op_params(action, 0.05, 0.1, c_sw=1.05)
    b = synth.z2_source(dims, 62).numpy()
    xs, info = lat.solve(op, L.solve_params(solver=L.GCR, tol=1e-10, prec_sloppy=prec), [b])
    assert info[0]["status"] == 0, info
    assert info[0]["true_rel_residual"] <= 1e-10
    assert true_residual(orc, dims, U, C, 0.05, 0.1, b, xs[0]) <= 1e-10
    xc, _ = lat.solve(op, L.solve_params(solver=L.MIXED_CGNR, tol=1e-12, prec_sloppy=L.F32), [b])
    assert np.linalg.norm(xs[0] - xc[0]) <= 1e-6 * np.linalg.norm(xc[0])


@pytest.mark.parametrize("restart", [1, 3, 16])
def test_gcr_multi_rhs_restart_lengths(L, orc, restart):
    dims = (6, 4, 4, 6)
    lat, U = make(L, dims, 63, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.05)
    bs = [synth.z2_source(dims, 64 + k).numpy() for k in range(3)]
    sp = L.solve_params(solver=L.GCR, tol=1e-10, prec_sloppy=L.F16, restart=restart)
    xs, info = lat.solve(op, sp, bs)
    for b, x, i in zip(bs, xs, info):
        assert i["status"] == 0, (restart, i)
        assert true_residual(orc, dims, U, C, 0.05, 0.02, b, x) <= 1e-10


def test_gcr_argument_errors(L):
    dims = (4, 4, 4, 4)
    lat, _ = make(L, dims, 65)
    op = L.op_params(L.WILSON_TM, 0.05, 0.1)
    b = synth.z2_source(dims, 66).numpy()
    with pytest.raises(L.LqError):
        lat.solve(op, L.solve_params(solver=L.GCR, restart=17), [b])
    h = L.Lattice(dims)
    h.load_gauge(L.FAT, synth.fat_links(dims, 67))
    h.load_gauge(L.LONG, synth.long_links(dims, 68))
    with pytest.raises(L.LqError) as e:
        h.solve(L.op_params(L.HISQ, 0.05), L.solve_params(solver=L.GCR), [synth.z2_source(dims, 69, ncomp=3).numpy()])
    assert "Wilson" in str(e.value)
