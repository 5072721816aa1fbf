"""Solves with host buffers. Each solution goes back to the host on a side stream as
soon as the solver has written it, next to the solve's remaining kernels: the final
residual check, or the next mass's solve in a multi-mass solve. Host and device
buffers give the same solutions, bit for bit, whether the host memory is pageable or
pinned. Each solution also meets the oracle's true residual."""
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


def three_ways(lat, op, sp, bs):
    """(device, pageable host, pinned host) solutions and infos of the same solve;
    one device solve first so that every launch shape is tuned before the three."""
    import torch
    dev = [torch.from_numpy(b).cuda() for b in bs]
    lat.solve(op, sp, dev)
    xd, id_ = lat.solve(op, sp, dev)
    xd = [x.cpu().numpy() for x in xd]
    xh, ih = lat.solve(op, sp, bs)
    pinned = [torch.empty(b.shape, dtype=torch.complex128).pin_memory() for b in xh]
    xp, ip = lat.solve(op, sp, bs, out=pinned)
    xp = [x.numpy() for x in xp]
    return (xd, id_), (xh, ih), (xp, ip)


def check_same(runs):
    (xd, id_), *rest = runs
    for xs, infos in rest:
        assert len(xs) == len(xd)
        for a, b in zip(xs, xd):
            assert np.array_equal(a, b)
        assert [i["iters"] for i in infos] == [i["iters"] for i in id_]
        assert all(i["status"] == 0 for i in infos)


def test_wilson_clover_mixed_solve(L, orc):
    dims = (4, 4, 4, 8)
    U = synth.thin_links(dims, 131, 0.3).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.THIN, U)
    lat.load_clover(1.0)
    m, mu = 0.1, 0.02
    op = L.op_params(L.WILSON_TM_CLOVER, m, mu, c_sw=1.0)
    sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16)
    bs = [synth.z2_source(dims, 231 + k).numpy() for k in range(3)]
    runs = three_ways(lat, op, sp, bs)
    check_same(runs)
    D = orc.Wilson(dims, U, m, mu, clover=orc.clover(dims, U, 1.0))
    for b, x in zip(bs, runs[1][0]):
        assert np.linalg.norm(b - D.apply(x)) / np.linalg.norm(b) <= 1e-10


def test_twisted_multishift_solve(L, orc):
    dims = (4, 4, 4, 8)
    U = synth.thin_links(dims, 132, 0.3).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.THIN, U)
    m, mus = 0.1, [0.01, 0.05]
    op = L.op_params(L.WILSON_TM, m, mus[0])
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=L.F32, masses=mus)
    bs = [synth.z2_source(dims, 232 + k).numpy() for k in range(2)]
    runs = three_ways(lat, op, sp, bs)
    check_same(runs)
    for k, b in enumerate(bs):
        for i, mu in enumerate(mus):
            x = runs[2][0][k * len(mus) + i]
            D = orc.Wilson(dims, U, m, mu)
            assert np.linalg.norm(b - D.apply(x)) / np.linalg.norm(b) <= 1e-10, (k, mu)


def test_hisq_multi_mass_solve(L, orc):
    dims = (6, 6, 6, 8)
    V = synth.fat_links(dims, 133).numpy()
    W = synth.long_links(dims, 134).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.FAT, V)
    lat.load_gauge(L.LONG, W)
    masses = [0.02, 0.05, 0.1]
    op = L.op_params(L.HISQ, masses[0])
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=L.F16, masses=masses)
    bs = [synth.z2_source(dims, 233 + k, ncomp=3).numpy() for k in range(2)]
    runs = three_ways(lat, op, sp, bs)
    check_same(runs)
    for k, b in enumerate(bs):
        for i, m in enumerate(masses):
            x = runs[1][0][k * len(masses) + i]
            D = orc.Hisq(dims, V, W, m)
            assert np.linalg.norm(b - D.apply(x)) / np.linalg.norm(b) <= 1e-10, (k, m)
