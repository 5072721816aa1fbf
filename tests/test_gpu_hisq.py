"""Parity of the CUDA HISQ path (fat one-hop + long three-hop links, Sec. 2.2)
with the FP64 oracle: hopping term per parity, full operator, Schur operator,
single-mass and multi-shift solves (oracle true residual <= 1e-10)."""
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


def make(L, dims, seed):
    V = synth.fat_links(dims, seed).numpy()
    W = synth.long_links(dims, seed + 1).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.FAT, V)
    lat.load_gauge(L.LONG, W)
    return lat, V, W


# 6^4: the three-hop wraps; 4x4x4x6 ragged; 2^4: all hops land on one site
DIMS = [(6, 6, 6, 6), (4, 4, 4, 6), (2, 2, 2, 2), (8, 6, 4, 10)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_hisq_hopping_term(L, orc, dims, prec):
    lat, V, W = make(L, dims, 41)
    psi = synth.gaussian_field(dims, 42, ncomp=3).numpy()
    D = orc.Hisq(dims, V, W, 0.0)
    op = L.op_params(L.HISQ, 0.0, c_naik=-1.0 / 24.0)
    mask = parity_mask(dims)
    for dagger in (False, True):
        ref = D.hop(psi, dagger=dagger)
        for p in (0, 1):
            got = lat.dslash_apply(op, p, psi, dagger=dagger, prec=prec)
            sel = mask == p
            assert np.all(got[~sel] == 0)
            assert rel_err(got[sel], ref[sel]) < TOL[prec], (dims, prec, dagger, p)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_hisq_full_and_schur_operator(L, orc, prec):
    dims = (4, 4, 6, 6)
    lat, V, W = make(L, dims, 43)
    m = 0.07
    D = orc.Hisq(dims, V, W, m)
    op = L.op_params(L.HISQ, m)
    psi = synth.gaussian_field(dims, 44, ncomp=3).numpy()
    for dagger in (False, True):
        ref = D.apply(psi, dagger=dagger)
        got = lat.operator_apply(op, psi, form=L.OP_FULL, dagger=dagger, prec=prec)
        assert rel_err(got, ref) < TOL[prec]
    mask = parity_mask(dims)
    ve = np.where((mask == 0)[..., None], psi, 0)
    Hv = D.hop(ve)
    ref = m * m * ve - np.where((mask == 0)[..., None], D.hop(np.where((mask == 1)[..., None], Hv, 0)), 0)
    got = lat.operator_apply(op, psi, form=L.OP_SCHUR, prec=prec)
    assert rel_err(got, ref) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_hisq_single_mass_solve(L, orc, prec):
    dims = (6, 6, 6, 8)
    lat, V, W = make(L, dims, 45)
    m = 0.05
    b = synth.z2_source(dims, 46, ncomp=3).numpy()
    op = L.op_params(L.HISQ, m)
    xs, info = lat.solve(op, L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec), [b])
    assert info[0]["status"] == 0
    D = orc.Hisq(dims, V, W, m)
    r = b - D.apply(xs[0])
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    x_ref, _ = D.cgnr(b, tol=1e-13)
    assert rel_err(xs[0], x_ref) < 1e-8


@pytest.mark.parametrize("prec", [1, 2])
def test_hisq_multishift_solve(L, orc, prec):
    """Multi-shift over four masses (the HISQ configuration's {0.002, 0.01, 0.02, 0.05}
    reduced in range for a small lattice), two right-hand sides."""
    dims = (6, 6, 6, 8)
    lat, V, W = make(L, dims, 47)
    masses = [0.01, 0.02, 0.05, 0.1]
    bs = [synth.z2_source(dims, 48, ncomp=3).numpy(), synth.point_source(dims, (1, 0, 2, 3), None, 2).numpy()]
    op = L.op_params(L.HISQ, masses[0])
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=prec, masses=masses)
    xs, info = lat.solve(op, sp, bs)
    assert len(xs) == len(bs) * len(masses)
    for k, b in enumerate(bs):
        assert info[k]["status"] == 0
        for i, m in enumerate(masses):
            D = orc.Hisq(dims, V, W, m)
            r = b - D.apply(xs[k * len(masses) + i])
            assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10, (k, m)


@pytest.mark.parametrize("nrhs,nmass", [(5, 4), (1, 9)])
def test_hisq_multishift_beyond_the_fused_update(L, orc, nrhs, nmass):
    """Multi-shift solves whose stage has more right-hand sides (2 x 5 = 10) or more
    shifts (9) than the one-pass vector update takes, so that the separate updates run:
    every mass of every right-hand side against the oracle."""
    dims = (4, 4, 4, 8)
    lat, V, W = make(L, dims, 57)
    masses = [0.02 * (1 + i) for i in range(nmass)]
    bs = [synth.z2_source(dims, 58 + k, ncomp=3).numpy() for k in range(nrhs)]
    op = L.op_params(L.HISQ, masses[0])
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=1, masses=masses)
    xs, info = lat.solve(op, sp, bs)
    for k, b in enumerate(bs):
        assert info[k]["status"] == 0
        for i, m in enumerate(masses):
            D = orc.Hisq(dims, V, W, m)
            r = b - D.apply(xs[k * nmass + i])
            assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10, (k, m)


def test_hisq_repeated_solves_reuse_workspace(L, orc):
    """Consecutive solves on one lattice reuse its work buffers (including the
    pinned scalar block): single-mass CG with 1 and 4 right-hand sides, graph
    replay on and off, FP16 and FP32, and a multi-shift solve after them, all
    meet the oracle's true residual."""
    dims = (6, 6, 6, 8)
    lat, V, W = make(L, dims, 49)
    m = 0.05
    b = synth.z2_source(dims, 50, ncomp=3).numpy()
    D = orc.Hisq(dims, V, W, m)
    op = L.op_params(L.HISQ, m)
    for prec in (2, 1):
        for n in (1, 4):
            for gk in (0, -1):
                sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec, graph_iters=gk)
                xs, info = lat.solve(op, sp, [b] * n)
                for x, inf in zip(xs, info):
                    assert inf["status"] == 0, (prec, n, gk)
                    assert np.linalg.norm(b - D.apply(x)) / np.linalg.norm(b) <= 1e-10
    masses = [0.01, 0.02, 0.05]
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=2, masses=masses)
    xs, info = lat.solve(L.op_params(L.HISQ, masses[0]), sp, [b])
    assert info[0]["status"] == 0
    for i, mi in enumerate(masses):
        Di = orc.Hisq(dims, V, W, mi)
        assert np.linalg.norm(b - Di.apply(xs[i])) / np.linalg.norm(b) <= 1e-10


def test_hisq_full_size_sampled_sites(L, orc):
    """48^3x144 (the HISQ configuration) would need 18 GB of FP64 links on the
    host for the oracle; the kernel is checked at 24^3x48 full size instead on
    2000 sampled sites, in FP32 and FP16."""
    dims = (24, 24, 24, 48)
    V = synth.fat_links(dims, 104, device="cuda")
    W = synth.long_links(dims, 105, device="cuda")
    psi = synth.gaussian_field(dims, 204, ncomp=3, device="cuda")
    lat = L.Lattice(dims)
    lat.load_gauge(L.FAT, V)
    lat.load_gauge(L.LONG, W)
    op = L.op_params(L.HISQ, 0.01)
    Vh, Wh, ph = V.cpu().numpy(), W.cpu().numpy(), psi.cpu().numpy()
    D = orc.Hisq(dims, Vh, Wh, 0.0)
    rng = np.random.default_rng(9)
    lx, ly, lz, lt = dims
    for prec in (1, 2):
        for p in (0, 1):
            got = lat.dslash_apply(op, p, psi, prec=prec).cpu().numpy().reshape(-1, 3)
            cand = rng.integers(0, lx * ly * lz * lt, size=6000)
            par = (cand % lx + (cand // lx) % ly + (cand // (lx * ly)) % lz + cand // (lx * ly * lz)) % 2
            sites = cand[par == p][:2000]
            ref = D.hop_sites(ph, sites)
            assert rel_err(got[sites], ref) < TOL[prec], (prec, p)


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("code", [3064, 3128, 4128, 5128])
def test_hisq_packed_pair_kernel_every_geometry(L, orc, dims, code):
    """The FP16 packed-pair HISQ kernel (its own neighbour indexing at distances 1 and 3,
    wrapping twice on extents of 2) for each tuning code: hopping term per parity and
    adjoint, and the Schur operator, against the oracle."""
    lat, V, W = make(L, dims, 51)
    psi = synth.gaussian_field(dims, 52, ncomp=3).numpy()
    m = 0.07
    D = orc.Hisq(dims, V, W, 0.0)
    op = L.op_params(L.HISQ, m, c_naik=-1.0 / 24.0)
    mask = parity_mask(dims)
    try:
        L.tune_reset()
        L.tune_force(code)
        for dagger in (False, True):
            ref = D.hop(psi, dagger=dagger)
            for p in (0, 1):
                got = lat.dslash_apply(op, p, psi, dagger=dagger, prec=2)
                sel = mask == p
                assert np.all(got[~sel] == 0)
                assert rel_err(got[sel], ref[sel]) < TOL[2], (dims, code, dagger, p)
        ve = np.where((mask == 0)[..., None], psi, 0)
        Hv = D.hop(ve)
        ref = m * m * ve - np.where((mask == 0)[..., None], D.hop(np.where((mask == 1)[..., None], Hv, 0)), 0)
        got = lat.operator_apply(op, psi, form=L.OP_SCHUR, prec=2)
        assert rel_err(got, ref) < 10 * TOL[2], (dims, code)
    finally:
        L.tune_force(0)
        L.tune_reset()


@pytest.mark.parametrize("nrhs", [2, 3, 4])
@pytest.mark.parametrize("code", [9064, 9128])
def test_hisq_packed_pair_kernel_per_right_hand_side(L, orc, nrhs, code):
    """Two to four right-hand sides through the FP16 packed-pair kernel launched once per
    right-hand side (the tuning candidate beside the scalar kernel's lanes): the hopping
    term and its adjoint of every right-hand side, and a mixed CG solve of the three
    columns of a propagator, against the oracle."""
    import torch
    dims = (6, 6, 6, 6)
    lat, V, W = make(L, dims, 53)
    m = 0.07
    D = orc.Hisq(dims, V, W, 0.0)
    op = L.op_params(L.HISQ, m, c_naik=-1.0 / 24.0)
    mask = parity_mask(dims)
    vs = [synth.gaussian_field(dims, 800 + k, ncomp=3).numpy() for k in range(nrhs)]
    try:
        L.tune_reset()
        L.tune_force(code)
        for dagger in (False, True):
            fi = L.Field(lat, L.STAGGERED_FIELD, 2, nrhs)
            fo = L.Field(lat, L.STAGGERED_FIELD, 2, nrhs)
            for k, v in enumerate(vs):
                fi.load(k, 1, torch.from_numpy(v).cuda())
            L.dslash_field(lat, op, 0, fi, fo, dagger=dagger)
            for k, v in enumerate(vs):
                got = fo.store(k, 0, torch.zeros(v.shape, dtype=torch.complex128, device="cuda")).cpu().numpy()
                ref = D.hop(np.where((mask == 1)[..., None], v, 0), dagger=dagger)
                assert rel_err(got[mask == 0], ref[mask == 0]) < TOL[2], (code, nrhs, k, dagger)
        if nrhs == 3:
            Dm = orc.Hisq(dims, V, W, m)
            bs = [synth.z2_source(dims, 810 + k, ncomp=3).numpy() for k in range(3)]
            sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=2)
            xs, info = lat.solve(op, sp, bs)
            for b, x, i in zip(bs, xs, info):
                assert i["status"] == 0
                assert np.linalg.norm(b - Dm.apply(x)) / np.linalg.norm(b) <= 1e-10
    finally:
        L.tune_force(0)
        L.tune_reset()
