"""Parity of the CUDA Wilson twisted-mass / clover path with the FP64 oracle.

Every quantity goes through the C ABI (lib.py is marshalling only) and is
compared element by element with the oracle on the same seeded inputs:
hopping term per parity and adjoint, the full operator with clover, the
even-odd Schur operator, and solves whose true residual the oracle recomputes.
Tolerances of the operator: FP64 1e-13, FP32 1e-6, FP16 storage 5e-3 (relative
L2); solutions: oracle true residual <= 1e-10.
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


def make(L, dims, seed, c_sw=None, eps=0.3):
    U = synth.thin_links(dims, seed, eps).numpy()
    lat = L.Lattice(dims, -1)
    lat.load_gauge(L.THIN, U)
    if c_sw is not None:
        lat.load_clover(c_sw)
    return lat, U


# 4^3x8 spans several thread blocks; 6x4x4x6 has a ragged last block (vh = 288);
# 2^4 makes x+mu and x-mu the same site
DIMS = [(4, 4, 4, 8), (6, 4, 4, 6), (2, 2, 2, 2)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_hopping_term_each_parity_and_adjoint(L, orc, dims, prec):
    lat, U = make(L, dims, 11)
    psi = synth.gaussian_field(dims, 12).numpy()
    W = orc.Wilson(dims, U, 0.1, 0.05)
    op = L.op_params(L.WILSON_TM, 0.1, 0.05)
    mask = parity_mask(dims)
    for dagger in (False, True):
        ref = W.hop(psi, dagger=dagger)
        for p in (0, 1):
            src = np.where((mask == 1 - p)[..., None, None], psi, 0)
            got = lat.dslash_apply(op, p, src, dagger=dagger, prec=prec)
            sel = (mask == p)
            assert np.all(got[~sel] == 0)
            assert rel_err(got[sel], ref[sel]) < TOL[prec], (dims, prec, dagger, p)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("clover", [False, True])
def test_full_operator_twisted_clover(L, orc, prec, clover):
    dims = (4, 4, 4, 6)
    lat, U = make(L, dims, 21, c_sw=1.05 if clover else None)
    C = orc.clover(dims, U, 1.05) if clover else None
    action = L.WILSON_TM_CLOVER if clover else L.WILSON_TM
    op = L.op_params(action, 0.05, 0.1, c_sw=1.05)
    psi = synth.gaussian_field(dims, 22).numpy()
    for dagger in (False, True):
        ref = orc.Wilson(dims, U, 0.05, 0.1, clover=C).apply(psi, dagger=dagger)
        got = lat.operator_apply(op, psi, form=L.OP_FULL, dagger=dagger, prec=prec)
        assert rel_err(got, ref) < TOL[prec], (prec, clover, dagger)


def test_device_clover_matches_oracle_clover_loaded_canonically(L, orc):
    """The on-device clover build equals loading the oracle's clover as an array."""
    dims = (4, 4, 4, 4)
    U = synth.thin_links(dims, 23).numpy()
    C = orc.clover(dims, U, 1.3)
    a = L.Lattice(dims)
    a.load_gauge(L.THIN, U)
    a.load_clover(1.3)
    b = L.Lattice(dims)
    b.load_gauge(L.THIN, U)
    b.load_clover(1.3, clover=C)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.3)
    psi = synth.gaussian_field(dims, 24).numpy()
    ra = a.operator_apply(op, psi)
    rb = b.operator_apply(op, psi)
    assert rel_err(ra, rb) < 1e-14


def schur_reference(orc, dims, U, C, m, mu, v_even, dagger=False):
    """Mhat v = A_ee v - H_eo A_oo^{-1} H_oe v, composed from oracle pieces; the
    site-local A^{-1} is a dense 12x12 solve per site (numpy LU)."""
    mask = parity_mask(dims)
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    A = (4 + m) * np.eye(12, dtype=complex) + np.kron(1j * (-mu if dagger else mu) * g5, np.eye(3))
    Afull = np.broadcast_to(A, mask.shape + (12, 12)).copy()
    if C is not None:
        Afull = Afull + C
    W = orc.Wilson(dims, U, 0.0, 0.0)
    v = np.where((mask == 0)[..., None, None], v_even, 0)
    h = W.hop(v, dagger=dagger)                                   # H_oe v on odd sites
    t = np.linalg.solve(Afull, h.reshape(h.shape[:4] + (12,))[..., None])[..., 0].reshape(h.shape)
    t = np.where((mask == 1)[..., None, None], t, 0)
    h2 = W.hop(t, dagger=dagger)                                  # H_eo A_oo^{-1} H_oe v
    av = (Afull @ v.reshape(v.shape[:4] + (12, 1)))[..., 0].reshape(v.shape)
    out = av - h2
    return np.where((mask == 0)[..., None, None], out, 0)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_schur_operator(L, orc, prec):
    dims = (4, 4, 4, 6)
    lat, U = make(L, dims, 31, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05)
    v = synth.gaussian_field(dims, 32).numpy()
    mask = parity_mask(dims)
    for dagger in (False, True):
        ref = schur_reference(orc, dims, U, C, 0.05, 0.1, v, dagger=dagger)
        got = lat.operator_apply(op, v, form=L.OP_SCHUR, dagger=dagger, prec=prec)
        assert np.all(got[mask == 1] == 0)
        assert rel_err(got, ref) < 10 * TOL[prec], (prec, dagger)


# tuning codes: block size; 1000 + block: registers capped at 85; 2000 + block: two hops
# in flight; 3000 - 6000 + block: the FP16 packed-pair kernels (128 / 85 registers with
# two hops in flight, 102 / 85 registers with one)
CODES = [(p, c) for p in (1, 2) for c in (64, 128, 256, 1064, 1128, 1256, 2064, 2128)] + \
        [(2, c) for c in (3064, 3128, 4064, 4128, 5064, 5128, 6064, 6128, 7256)] + \
        [(3, c) for c in (64, 128, 256, 1064, 1128, 1256)]  # double-float; 1000 + block: no row prefetch


@pytest.mark.parametrize("prec,code", CODES)
def test_each_tuning_candidate(L, orc, prec, code):
    """Every launch configuration the autotuner may pick (block sizes; the
    register-capped build; two hops of gathers in flight) gives the oracle's hopping term and Schur operator,
    on a lattice with a ragged last block."""
    dims = (6, 4, 4, 6)
    lat, U = make(L, dims, 33, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05)
    v = synth.gaussian_field(dims, 34).numpy()
    mask = parity_mask(dims)
    W = orc.Wilson(dims, U, 0.0, 0.0)
    try:
        L.tune_reset()
        L.tune_force(code)
        for dagger in (False, True):
            ref = W.hop(v, dagger=dagger)
            for p in (0, 1):
                src = np.where((mask == 1 - p)[..., None, None], v, 0)
                got = lat.dslash_apply(op, p, src, dagger=dagger, prec=prec)
                assert rel_err(got[mask == p], ref[mask == p]) < TOL[prec], (code, prec, dagger, p)
            ref = schur_reference(orc, dims, U, C, 0.05, 0.1, v, dagger=dagger)
            got = lat.operator_apply(op, v, form=L.OP_SCHUR, dagger=dagger, prec=prec)
            assert rel_err(got, ref) < 10 * TOL[prec], (code, prec, dagger)
    finally:
        L.tune_force(0)
        L.tune_reset()


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 4, 6), (2, 2, 2, 2), (2, 4, 6, 8), (8, 2, 4, 4)])
@pytest.mark.parametrize("code", [3128, 4064, 5128, 6064, 7256])
def test_packed_pair_kernels_on_every_geometry(L, orc, dims, code):
    """The FP16 packed-pair kernels (their own neighbour indexing) on extents of 2,
    ragged blocks and unequal extents: hopping term per parity and adjoint, and the
    clover Schur operator, against the oracle."""
    lat, U = make(L, dims, 35, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05)
    v = synth.gaussian_field(dims, 36).numpy()
    mask = parity_mask(dims)
    W = orc.Wilson(dims, U, 0.0, 0.0)
    try:
        L.tune_reset()
        L.tune_force(code)
        for dagger in (False, True):
            ref = W.hop(v, dagger=dagger)
            for p in (0, 1):
                src = np.where((mask == 1 - p)[..., None, None], v, 0)
                got = lat.dslash_apply(op, p, src, dagger=dagger, prec=2)
                assert np.all(got[mask != p] == 0)
                assert rel_err(got[mask == p], ref[mask == p]) < TOL[2], (dims, code, dagger, p)
            ref = schur_reference(orc, dims, U, C, 0.05, 0.1, v, dagger=dagger)
            got = lat.operator_apply(op, v, form=L.OP_SCHUR, dagger=dagger, prec=2)
            assert rel_err(got, ref) < 10 * TOL[2], (dims, code, dagger)
    finally:
        L.tune_force(0)
        L.tune_reset()


def true_residual(orc, dims, U, C, m, mu, b, x):
    r = b - orc.Wilson(dims, U, m, mu, clover=C).apply(x)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("solver,prec", [(0, 0), (1, 1), (1, 2)])
def test_solve_plain_method_tiny(L, orc, solver, prec):
    """4^3x8 Wilson twisted mass, no clover, m = 0.1, mu = 0.05, Z2 source, 1e-10."""
    dims = (4, 4, 4, 8)
    lat, U = make(L, dims, 101)
    b = synth.z2_source(dims, 201).numpy()
    op = L.op_params(L.WILSON_TM, 0.1, 0.05)
    sp = L.solve_params(solver=solver, tol=1e-10, prec_sloppy=prec)
    xs, info = lat.solve(op, sp, [b])
    assert info[0]["status"] == 0
    assert info[0]["true_rel_residual"] <= 1e-10
    res = true_residual(orc, dims, U, None, 0.1, 0.05, b, xs[0])
    assert res <= 1e-10, res
    x_ref, _ = orc.Wilson(dims, U, 0.1, 0.05).cgnr(b, tol=1e-13)
    assert rel_err(xs[0], x_ref) < 1e-8


@pytest.mark.parametrize("prec", [1, 2])
def test_solve_clover_mixed_multi_rhs(L, orc, prec):
    """Twisted clover, even-odd, three right-hand sides solved together equal the oracle."""
    dims = (4, 4, 6, 8)
    lat, U = make(L, dims, 102, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.01, c_sw=1.05)
    bs = [synth.z2_source(dims, 202 + k).numpy() for k in range(3)]
    bs.append(synth.point_source(dims, (1, 2, 3, 4), 2, 1).numpy())
    sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec)
    xs, info = lat.solve(op, sp, bs)
    for b, x, inf in zip(bs, xs, info):
        assert inf["status"] == 0
        assert true_residual(orc, dims, U, C, 0.05, 0.01, b, x) <= 1e-10
    # one at a time gives the same solutions within the tolerance
    x1, _ = lat.solve(op, sp, [bs[1]])
    assert rel_err(x1[0], xs[1]) < 1e-8


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_bicgstab_tiny(L, orc, prec):
    """BiCGStab directly on the even-odd Schur operator (the paper's Table 2 CPU
    solver), plain FP64 or mixed with reliable updates: the oracle's true
    residual <= 1e-10 and the solution equals the oracle's."""
    dims = (4, 4, 4, 8)
    lat, U = make(L, dims, 101)
    b = synth.z2_source(dims, 201).numpy()
    op = L.op_params(L.WILSON_TM, 0.1, 0.05)
    xs, info = lat.solve(op, L.solve_params(solver=L.BICGSTAB, tol=1e-10, prec_sloppy=prec), [b])
    assert info[0]["status"] == 0
    assert true_residual(orc, dims, U, None, 0.1, 0.05, b, xs[0]) <= 1e-10
    x_ref, _ = orc.Wilson(dims, U, 0.1, 0.05).bicgstab(b, tol=1e-13)
    assert rel_err(xs[0], x_ref) < 1e-8


@pytest.mark.parametrize("prec", [1, 2])
def test_bicgstab_clover_multi_rhs_equals_cgnr(L, orc, prec):
    """Twisted clover, three right-hand sides at once: every BiCGStab solution
    meets the oracle's true residual and agrees with the CGNR solution."""
    dims = (4, 4, 6, 8)
    lat, U = make(L, dims, 108, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.01, c_sw=1.05)
    bs = [synth.z2_source(dims, 208 + k).numpy() for k in range(2)]
    bs.append(synth.point_source(dims, (1, 2, 3, 4), 2, 1).numpy())
    xs, info = lat.solve(op, L.solve_params(solver=L.BICGSTAB, tol=1e-10, prec_sloppy=prec), bs)
    xc, _ = lat.solve(op, L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec), bs)
    for b, x, y, inf in zip(bs, xs, xc, info):
        assert inf["status"] == 0
        assert true_residual(orc, dims, U, C, 0.05, 0.01, b, x) <= 1e-10
        assert rel_err(x, y) < 1e-8


@pytest.mark.parametrize("prec", [1, 2])
def test_twisted_multishift_solve(L, orc, prec):
    """Several twisted masses at once (no clover): one multi-shift CG on
    M0^+ M0 + mu^2 for the two sources M0^+ b and g5 b, then each mass refined by
    the mixed CGNR from that guess; every solution meets the oracle's true
    residual for its own mu and equals the single-mass solve."""
    dims = (4, 4, 4, 8)
    lat, U = make(L, dims, 109)
    m, mus = 0.1, [0.01, 0.03, 0.1]
    bs = [synth.z2_source(dims, 209).numpy(), synth.point_source(dims, (1, 2, 3, 4), 0, 2).numpy()]
    op = L.op_params(L.WILSON_TM, m, mus[0])
    sp = L.solve_params(solver=L.MULTISHIFT_CG, tol=1e-10, prec_sloppy=prec, masses=mus)
    xs, info = lat.solve(op, sp, bs)
    assert len(xs) == len(bs) * len(mus)
    for k, b in enumerate(bs):
        assert info[k]["status"] == 0
        for i, mu in enumerate(mus):
            x = xs[k * len(mus) + i]
            assert true_residual(orc, dims, U, None, m, mu, b, x) <= 1e-10, (k, mu)
            x1, _ = lat.solve(L.op_params(L.WILSON_TM, m, mu),
                              L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec), [b])
            assert rel_err(x, x1[0]) < 1e-8


def test_twisted_multishift_rejects_clover(L):
    dims = (4, 4, 4, 4)
    lat, U = make(L, dims, 110, c_sw=1.0)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.1, 0.01, c_sw=1.0)
    b = synth.z2_source(dims, 210).numpy()
    with pytest.raises(L.LqError) as e:
        lat.solve(op, L.solve_params(solver=L.MULTISHIFT_CG, masses=[0.01, 0.02]), [b])
    assert e.value.code == L.LQ_EINVAL


def test_workspace_kept_between_solves(L, orc):
    """The work buffers a solve takes stay with the lattice: a second solve
    allocates nothing more and returns bit-identical solutions (the reductions
    run in a fixed order), on the same stream and on another one; releasing
    them frees device memory and the next solve is unchanged."""
    import torch
    dims = (4, 4, 6, 8)
    lat, U = make(L, dims, 106, c_sw=1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.01, c_sw=1.05)
    b = synth.z2_source(dims, 206).numpy()
    sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16)
    x1, _ = lat.solve(op, sp, [b])
    held = lat.device_bytes()
    x2, _ = lat.solve(op, sp, [b])
    assert lat.device_bytes() == held
    assert np.array_equal(x1[0], x2[0])
    side = torch.cuda.Stream()
    x3, _ = lat.solve(op, sp, [b], stream=side)
    torch.cuda.synchronize()
    assert lat.device_bytes() == held
    assert np.array_equal(x1[0], x3[0])
    freed = lat.release_workspace()
    assert freed > 0 and lat.device_bytes() == held - freed
    x4, _ = lat.solve(op, sp, [b])
    assert np.array_equal(x1[0], x4[0])
    C = orc.clover(dims, U, 1.05)
    assert true_residual(orc, dims, U, C, 0.05, 0.01, b, x4[0]) <= 1e-10


def test_graph_replay_matches_eager_launches(L, orc):
    """CG iterations replayed from CUDA graphs give the same solution, bit for
    bit, as eager launches (same kernels, same order), and the launch counter
    counts every replayed kernel. Several iterations per graph converge too."""
    dims = (4, 4, 6, 8)
    lat, U = make(L, dims, 107, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.01, c_sw=1.05)
    b = synth.z2_source(dims, 207).numpy()
    res = {}
    for gk in (-1, 0, 3):
        sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16, graph_iters=gk)
        lat.solve(op, sp, [b])  # tunes
        n0 = L.launch_count()
        xs, info = lat.solve(op, sp, [b])
        res[gk] = (xs[0], info[0], L.launch_count() - n0)
    x_e, i_e, n_e = res[-1]
    x_g, i_g, n_g = res[0]
    assert np.array_equal(x_e, x_g)
    assert i_e["iters"] == i_g["iters"] and n_e == n_g
    x_3, i_3, _ = res[3]
    assert i_3["status"] == 0 and i_3["iters"] <= i_e["iters"] + 8
    assert true_residual(orc, dims, U, C, 0.05, 0.01, b, x_3) <= 1e-10


def test_solve_device_arrays_and_2x4(L, orc):
    import torch
    dims = (2, 2, 2, 2)
    lat, U = make(L, dims, 103, c_sw=1.0)
    C = orc.clover(dims, U, 1.0)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.1, 0.05, c_sw=1.0)
    b = synth.z2_source(dims, 203)
    xs, info = lat.solve(op, L.solve_params(tol=1e-12), [b.cuda()])
    x = xs[0].cpu().numpy()
    A_apply = orc.Wilson(dims, U, 0.1, 0.05, clover=C)
    n = 192
    A = np.zeros((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        A[:, j] = A_apply.apply(e.reshape(A_apply.shape())).ravel()
    x_lu = np.linalg.solve(A, b.numpy().ravel())
    assert rel_err(x.ravel(), x_lu) < 1e-10


def test_zero_source_and_nan_source(L):
    dims = (4, 4, 4, 4)
    lat, U = make(L, dims, 104)
    op = L.op_params(L.WILSON_TM, 0.1, 0.05)
    b = np.zeros((4, 4, 4, 4, 4, 3), dtype=complex)
    b[0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(L.LqError) as e:
        lat.solve(op, L.solve_params(), [b])
    assert e.value.code == L.LQ_ENAN


def test_largest_right_hand_side_count_per_call(L, orc):
    """The largest number of right-hand sides one Wilson solve call takes (64): sixteen
    groups of four threads per site on the FP16 multi-RHS kernels, every column's true
    residual recomputed by the oracle at most 1e-10; one more is refused."""
    dims = (4, 4, 4, 6)
    lat, U = make(L, dims, 106, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.01, c_sw=1.05)
    bs = [synth.z2_source(dims, 700 + k).numpy() for k in range(64)]
    sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16)
    xs, info = lat.solve(op, sp, bs)
    for b, x, inf in zip(bs, xs, info):
        assert inf["status"] == 0
        assert true_residual(orc, dims, U, C, 0.05, 0.01, b, x) <= 1e-10
    with pytest.raises(L.LqError) as e:
        lat.solve(op, sp, bs + [bs[0]])
    assert e.value.code == L.LQ_EINVAL


def test_maxiter_reports_not_converged(L):
    dims = (4, 4, 4, 4)
    lat, U = make(L, dims, 105)
    op = L.op_params(L.WILSON_TM, 0.1, 0.05)
    b = synth.z2_source(dims, 205).numpy()
    xs, info = lat.solve(op, L.solve_params(tol=1e-10, maxiter=3), [b], check=False)
    assert info[0]["status"] == L.LQ_ENOTCONV
    assert info[0]["iters"] == 3
    assert info[0]["true_rel_residual"] > 1e-10


def test_full_size_hopping_term_sampled_sites(L, orc):
    """24^3x64 (the benchmark lattice), FP32 and FP16 kernels at full size, checked
    on 2000 sampled output sites computed one by one by the oracle."""
    import torch
    dims = (24, 24, 24, 64)
    U = synth.thin_links(dims, 102, device="cuda")
    psi = synth.gaussian_field(dims, 303, device="cuda")
    lat = L.Lattice(dims)
    lat.load_gauge(L.THIN, U)
    op = L.op_params(L.WILSON_TM, 0.05, 0.01)
    Uh = U.cpu().numpy()
    psih = psi.cpu().numpy()
    rng = np.random.default_rng(5)
    lx, ly, lz, lt = dims
    for prec in (1, 2):
        for p in (0, 1):
            got = lat.dslash_apply(op, p, psi, prec=prec).cpu().numpy().reshape(-1, 4, 3)
            cand = rng.integers(0, lx * ly * lz * lt, size=6000)
            xs = cand % lx
            ys = (cand // lx) % ly
            zs = (cand // (lx * ly)) % lz
            ts = cand // (lx * ly * lz)
            sites = cand[((xs + ys + zs + ts) % 2) == p][:2000]
            W = orc.Wilson(dims, Uh, 0.05, 0.01)
            ref = W.hop_sites(psih, sites)
            assert rel_err(got[sites], ref) < TOL[prec], (prec, p)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("nrhs", [2, 3, 4, 5])
def test_multi_rhs_operator_equals_single(L, prec, nrhs):
    """The fused multi-right-hand-side kernels (NB = 2 / 4 per thread, ragged
    remainders) give each right-hand side what the single kernel gives."""
    import torch
    dims = (4, 4, 6, 8)
    lat, U = make(L, dims, 106, c_sw=1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.05)
    psis = [synth.gaussian_field(dims, 300 + k).cuda() for k in range(nrhs)]
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
            mask = parity_mask(dims) == 0
            assert rel_err(got[mask], one[mask]) < TOL[prec], (prec, nrhs, k, dagger)


@pytest.mark.parametrize("per_launch", [1, 4, 16])
def test_persistent_cg_solve(L, orc, per_launch):
    """The mixed CGNR with its inner iterations in one persistent cooperative kernel
    (grid-wide barriers between the operator, vector and reduction phases): FP16
    sloppy operator with clover, on a lattice with a ragged last block; the oracle's
    true residual meets 1e-10 and the solution agrees with the per-kernel path."""
    dims = (6, 4, 4, 10)
    lat, U = make(L, dims, 37, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.05)
    b = synth.z2_source(dims, 38).numpy()
    base = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16)
    pers = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16, persistent=per_launch)
    (x0,), (i0,) = lat.solve(op, base, [b])
    (x1,), (i1,) = lat.solve(op, pers, [b])
    assert i1["status"] == 0
    assert true_residual(orc, dims, U, C, 0.05, 0.02, b, x1) <= 1e-10
    assert rel_err(x1, x0) < 1e-8
    assert i1["iters"] >= i0["iters"] - 2


@pytest.mark.parametrize("prec,nrhs", [(2, 1), (1, 1), (2, 5)])
def test_correction_form_late_updates(L, orc, prec, nrhs):
    """Reliable updates below 1e-4 |bhat| in correction form with the FP32 operator
    (update_f32_below): every solution's true residual recomputed by the oracle meets
    1e-10, the library's own final residual (recomputed from b) agrees with it, and the
    solution agrees with the one of FP64-accuracy updates throughout."""
    dims = (6, 4, 4, 10)
    lat, U = make(L, dims, 41, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.05)
    bs = [synth.z2_source(dims, 42 + k).numpy() for k in range(nrhs)]
    base = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec)
    corr = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=prec, update_f32_below=1e-4)
    x0s, i0s = lat.solve(op, base, bs)
    x1s, i1s = lat.solve(op, corr, bs)
    for b, x0, x1, i0, i1 in zip(bs, x0s, x1s, i0s, i1s):
        assert i1["status"] == 0
        res = true_residual(orc, dims, U, C, 0.05, 0.02, b, x1)
        assert res <= 1e-10, res
        assert abs(res / i1["true_rel_residual"] - 1) < 0.01
        assert rel_err(x1, x0) < 1e-8
        assert i1["iters"] <= i0["iters"] + 4


def test_bounded_grid_barrier_reports_a_wait_that_runs_out(L):
    """The barrier of the persistent kernel: complete when every block arrives, and
    a status (not a hang) when one never does."""
    code, failed = L.barrier_selftest(4, 4, rounds=50)
    assert code == 0 and failed == 0
    code, failed = L.barrier_selftest(2, 3, rounds=1)
    assert code == L.LQ_ETIMEOUT and failed == 1
    code, failed = L.barrier_selftest(4, 4, rounds=3)  # the GPU is usable afterwards
    assert code == 0 and failed == 0


@pytest.mark.parametrize("nrhs", [4, 5, 12])
@pytest.mark.parametrize("code", [3064, 3128, 5064, 5128])
def test_packed_pair_multi_rhs_kernels(L, orc, nrhs, code):
    """The FP16 packed-pair kernels with four threads per site (one right-hand side
    each, shared links and clover records; a ragged last group for 5 right-hand
    sides): hopping term and clover Schur operator of every right-hand side against
    the oracle, on a lattice with a ragged last block."""
    import torch
    dims = (6, 4, 4, 6)
    lat, U = make(L, dims, 39, c_sw=1.05)
    C = orc.clover(dims, U, 1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.1, c_sw=1.05)
    mask = parity_mask(dims)
    W = orc.Wilson(dims, U, 0.0, 0.0)
    vs = [synth.gaussian_field(dims, 400 + k).numpy() for k in range(nrhs)]
    try:
        L.tune_reset()
        L.tune_force(code)
        for dagger in (False, True):
            fi = L.Field(lat, L.WILSON_FIELD, 2, nrhs)
            fo = L.Field(lat, L.WILSON_FIELD, 2, nrhs)
            ft = L.Field(lat, L.WILSON_FIELD, 2, nrhs)
            for k, v in enumerate(vs):
                fi.load(k, 1, torch.from_numpy(v).cuda())
            L.dslash_field(lat, op, 0, fi, fo, dagger=dagger)
            for k, v in enumerate(vs):
                got = fo.store(k, 0, torch.zeros(v.shape, dtype=torch.complex128, device="cuda")).cpu().numpy()
                ref = W.hop(np.where((mask == 1)[..., None, None], v, 0), dagger=dagger)
                assert rel_err(got[mask == 0], ref[mask == 0]) < TOL[2], (code, nrhs, k, dagger)
            for k, v in enumerate(vs):
                fi.load(k, 0, torch.from_numpy(v).cuda())
            L.schur_field(lat, op, fi, fo, ft, dagger=dagger)
            for k, v in enumerate(vs):
                got = fo.store(k, 0, torch.zeros(v.shape, dtype=torch.complex128, device="cuda")).cpu().numpy()
                ref = schur_reference(orc, dims, U, C, 0.05, 0.1, v, dagger=dagger)
                assert rel_err(got[mask == 0], ref[mask == 0]) < 10 * TOL[2], (code, nrhs, k, dagger)
    finally:
        L.tune_force(0)
        L.tune_reset()
