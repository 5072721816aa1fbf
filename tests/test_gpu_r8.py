"""R8 link compression against the FP64 oracle.

An SU(3) link is stored as u01, u02, u10 and the phases of u00 and u20 (eight
reals); the kernels rebuild the rest from unit rows and columns and det = 1.
The oracle works with the full FP64 links, so these tests check the
reconstruction itself: the Wilson hopping term per parity and adjoint, the
Schur operator for each launch configuration the autotuner may pick, the fused
multi-RHS kernels, the HISQ operator with R8 long links, the no-allocation
entry point, a mixed-precision solve with an R8 sloppy operator (oracle true
residual <= 1e-10), and the refusal of a field where R8 is undefined (unit
links, |u00| = 1).
"""
import numpy as np
import pytest

from helpers import TOL, ensure_library, parity_mask, rel_err
from paper_2201_09004_b300 import synth
from test_gpu_wilson import schur_reference

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


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 4, 6), (2, 2, 2, 2)])
@pytest.mark.parametrize("prec", [1, 2])
def test_r8_hopping_term_each_parity_and_adjoint(L, orc, dims, prec):
    lat, U = make(L, dims, 11)
    psi = synth.gaussian_field(dims, 12).numpy()
    W = orc.Wilson(dims, U, 0.1, 0.05)
    op = L.op_params(L.WILSON_TM, 0.1, 0.05, recon=L.R8)
    mask = parity_mask(dims)
    for dagger in (False, True):
        ref = W.hop(psi, dagger=dagger)
        for p in (0, 1):
            src = np.where((mask == 1 - p)[..., None, None], psi, 0)
            got = lat.dslash_apply(op, p, src, dagger=dagger, prec=prec)
            sel = mask == p
            assert np.all(got[~sel] == 0)
            assert rel_err(got[sel], ref[sel]) < TOL[prec], (dims, prec, dagger, p)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("code", [0, 64, 256, 1128, 2064, 2128])
def test_r8_schur_operator_each_tuning_candidate(L, orc, prec, code):
    dims = (6, 4, 4, 6)
    lat, U = make(L, dims, 33, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05, recon=L.R8)
    v = synth.gaussian_field(dims, 34).numpy()
    mask = parity_mask(dims)
    try:
        L.tune_reset()
        if code:
            L.tune_force(code)
        for dagger in (False, True):
            ref = schur_reference(orc, dims, U, C, 0.05, 0.1, v, dagger=dagger)
            got = lat.operator_apply(op, v, form=L.OP_SCHUR, dagger=dagger, prec=prec)
            assert np.all(got[mask == 1] == 0)
            assert rel_err(got, ref) < 10 * TOL[prec], (code, prec, dagger)
    finally:
        L.tune_force(0)
        L.tune_reset()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("nrhs", [2, 5])
def test_r8_multi_rhs_operator_equals_single(L, prec, nrhs):
    import torch
    dims = (4, 4, 6, 8)
    lat, U = make(L, dims, 106, c_sw=1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.05, recon=L.R8)
    psis = [synth.gaussian_field(dims, 300 + k).cuda() for k in range(nrhs)]
    mask = parity_mask(dims) == 0
    for dagger in (False, True):
        fi = L.Field(lat, L.WILSON_FIELD, prec, nrhs)
        fo = L.Field(lat, L.WILSON_FIELD, prec, nrhs)
        ft = L.Field(lat, L.WILSON_FIELD, prec, nrhs)
        for k, p in enumerate(psis):
            fi.load(k, 0, p)
        L.schur_field(lat, op, fi, fo, ft, dagger=dagger)
        for k, p in enumerate(psis):
            got = fo.store(k, 0, torch.zeros_like(p)).cpu().numpy()
            one = lat.operator_apply(op, p, form=L.OP_SCHUR, dagger=dagger, prec=prec).cpu().numpy()
            assert rel_err(got[mask], one[mask]) < TOL[prec], (prec, nrhs, k, dagger)


@pytest.mark.parametrize("prec", [1, 2])
def test_r8_hisq_long_links(L, orc, prec):
    dims = (6, 6, 6, 6)
    V = synth.fat_links(dims, 41).numpy()
    Wl = synth.long_links(dims, 42).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.FAT, V)
    lat.load_gauge(L.LONG, Wl)
    D = orc.Hisq(dims, V, Wl, 0.0)
    op = L.op_params(L.HISQ, 0.0, c_naik=-1.0 / 24.0, recon=L.R8)
    psi = synth.gaussian_field(dims, 43, ncomp=3).numpy()
    mask = parity_mask(dims)
    for dagger in (False, True):
        ref = D.hop(psi, dagger=dagger)
        for p in (0, 1):
            got = lat.dslash_apply(op, p, psi, dagger=dagger, prec=prec)
            sel = mask == p
            assert rel_err(got[sel], ref[sel]) < TOL[prec], (prec, dagger, p)


@pytest.mark.parametrize("action", ["wilson", "hisq"])
@pytest.mark.parametrize("prec", [1, 2])
def test_r8_noalloc_matches_dslash_apply(L, action, prec):
    import torch
    dims = (8, 8, 8, 16)
    lat = L.Lattice(dims)
    if action == "wilson":
        lat.load_gauge(L.THIN, synth.thin_links(dims, 61).cuda())
        op = L.op_params(L.WILSON_TM, 0.1, 0.05, recon=L.R8)
        ncomp = 12
    else:
        lat.load_gauge(L.FAT, synth.fat_links(dims, 62).cuda())
        lat.load_gauge(L.LONG, synth.long_links(dims, 63).cuda())
        op = L.op_params(L.HISQ, 0.05, recon=L.R8)
        ncomp = 3
    mask = parity_mask(dims)
    psi = synth.gaussian_field(dims, 70, ncomp=ncomp).cuda()
    ref = lat.dslash_apply(op, 1, psi, prec=prec)
    out = torch.full_like(psi, complex(7.0, -3.0))
    lat.dslash_apply_noalloc(op, 1, psi, out, prec=prec)
    got, exp = out.cpu().numpy(), ref.cpu().numpy()
    assert np.all(got[mask == 0] == 0)
    assert rel_err(got[mask == 1], exp[mask == 1]) <= TOL[prec], (action, prec)


@pytest.mark.parametrize("solver", ["cgnr", "bicgstab"])
def test_r8_mixed_solve_meets_the_oracle_residual(L, orc, solver):
    dims = (4, 4, 4, 8)
    lat, U = make(L, dims, 21, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05)
    b = synth.z2_source(dims, 22).numpy()
    kind = L.MIXED_CGNR if solver == "cgnr" else L.BICGSTAB
    sp = L.solve_params(solver=kind, tol=1e-10, prec_sloppy=L.F16, recon_sloppy=L.R8)
    xs, info = lat.solve(op, sp, [b])
    assert info[0]["status"] == 0, info
    r = b - orc.Wilson(dims, U, 0.05, 0.1, clover=C).apply(xs[0])
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


def test_r8_refuses_unit_links(L):
    dims = (4, 4, 4, 4)
    lat = L.Lattice(dims)
    lat.load_gauge(L.THIN, synth.unit_links(dims))
    psi = synth.gaussian_field(dims, 5).numpy()
    op = L.op_params(L.WILSON_TM, 0.1, 0.0, recon=L.R8)
    with pytest.raises(L.LqError) as e:
        lat.dslash_apply(op, 0, psi, prec=L.F32)
    assert "recon 8" in str(e.value)
    # the refused packing leaves the lattice usable with R12
    op12 = L.op_params(L.WILSON_TM, 0.1, 0.0, recon=L.R12)
    got = lat.dslash_apply(op12, 0, psi, prec=L.F32)
    assert np.isfinite(got).all()
