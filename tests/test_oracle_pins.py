"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an exact identity of the
operators of Sec. 2.1 Eq. 2-3 and Sec. 2.2 Eq. 4, the convention relation the
paper prints in Sec. 2.2, a brute-force dense solve, or a property of the
synthetic generator. All CPU; no GPU.
"""
import math

import numpy as np
import pytest

from paper_2201_09004_b300 import synth

# --------------------------------------------------------------------- helpers

S1 = np.array([[0, 1], [1, 0]], dtype=complex)
S2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
S3 = np.array([[1, 0], [0, -1]], dtype=complex)
Z2 = np.zeros((2, 2), dtype=complex)
E2 = np.eye(2, dtype=complex)


def dr_gammas():
    """DeGrand-Rossi basis written from its block definition."""
    g1 = np.block([[Z2, 1j * S1], [-1j * S1, Z2]])
    g2 = np.block([[Z2, -1j * S2], [1j * S2, Z2]])
    g3 = np.block([[Z2, 1j * S3], [-1j * S3, Z2]])
    g4 = np.block([[Z2, E2], [E2, Z2]])
    return [g1, g2, g3, g4]


def coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x, y, z, t


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def gauge_transform(U, g):
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^+ ; array axes (Lt,Lz,Ly,Lx): mu -> axis 3-mu."""
    out = np.empty_like(U)
    for mu in range(4):
        gp = np.roll(g, -1, axis=3 - mu)
        out[mu] = g @ U[mu] @ np.conj(np.swapaxes(gp, -1, -2))
    return out


def gauge_transform_k(U, g, k):
    out = np.empty_like(U)
    for mu in range(4):
        gp = np.roll(g, -k, axis=3 - mu)
        out[mu] = g @ U[mu] @ np.conj(np.swapaxes(gp, -1, -2))
    return out


# ------------------------------------------------------------- generator pins

def test_generator_plaquette_and_unitarity(orc):
    dims = (6, 6, 6, 6)
    U = synth.thin_links(dims, 101).numpy()
    plaq = orc.plaquette(dims, U)
    assert abs(plaq - 0.61) < 0.01, plaq
    u = U.reshape(-1, 3, 3)
    unit = np.abs(np.conj(np.swapaxes(u, -1, -2)) @ u - np.eye(3)).max()
    assert unit < 1e-13
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-13
    # free field has plaquette exactly 1
    assert abs(orc.plaquette(dims, synth.unit_links(dims).numpy()) - 1.0) < 1e-15


def test_generator_fat_and_long_links():
    dims = (4, 4, 4, 6)
    V = synth.fat_links(dims, 104).numpy()
    assert np.allclose(np.linalg.norm(V.reshape(-1, 3, 3), axis=(1, 2)), math.sqrt(3.0), atol=1e-12)
    W = synth.long_links(dims, 105).numpy().reshape(-1, 3, 3)
    assert np.abs(np.conj(np.swapaxes(W, -1, -2)) @ W - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-13


def test_generator_is_counter_based():
    """A field depends only on (seed, site), not on the lattice it is cut from."""
    a = synth.z2_source((4, 4, 4, 4), 201).numpy()
    assert np.allclose(np.abs(a), 1.0)
    b = synth.z2_source((4, 4, 4, 4), 201).numpy()
    assert np.array_equal(a, b)
    c = synth.z2_source((4, 4, 4, 4), 202).numpy()
    assert not np.array_equal(a, c)


# ------------------------------------------------------------------ gamma pins

def test_gamma_basis_is_degrand_rossi(orc):
    g = dr_gammas()
    for mu in range(4):
        assert np.array_equal(orc.gamma(mu), g[mu])
        assert np.allclose(g[mu], g[mu].conj().T)
    for a in range(4):
        for b in range(4):
            anti = orc.gamma(a) @ orc.gamma(b) + orc.gamma(b) @ orc.gamma(a)
            assert np.allclose(anti, 2 * (a == b) * np.eye(4))
    g5 = orc.gamma(4)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3])


# ------------------------------------------------------- Wilson operator pins

def plane_wave(dims, n, u, antiperiodic=True):
    """psi(x) = exp(i p.x) u, p_i = 2 pi n_i / L_i, p_t = 2 pi (n_t + 1/2)/L_t."""
    x, y, z, t = coords(dims)
    p = [2 * math.pi * n[i] / dims[i] for i in range(3)]
    p.append(2 * math.pi * (n[3] + (0.5 if antiperiodic else 0.0)) / dims[3])
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return phase[..., None, None] * u.reshape(4, 3)[None, None, None, None], p


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (2, 2, 2, 2), (6, 4, 2, 4)])
def test_wilson_free_field_closed_form(orc, dims):
    """U = 1: M e^{ipx} u = e^{ipx} [(4+m-sum cos p) - i sum g_mu sin p_mu + i mu g5] u."""
    rng = np.random.default_rng(1)
    m, mu = 0.1, 0.05
    U = synth.unit_links(dims).numpy()
    W = orc.Wilson(dims, U, m, mu)
    g = dr_gammas()
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    for n in [(0, 0, 0, 0), (1, 0, 1, 2), (1, 1, 1, 1)]:
        u = rng.normal(size=12) + 1j * rng.normal(size=12)
        psi, p = plane_wave(dims, n, u)
        k = (4 + m - sum(math.cos(pp) for pp in p)) * np.eye(4) \
            - 1j * sum(g[i] * math.sin(p[i]) for i in range(4)) + 1j * mu * g5
        # apply k (spin) to each site's 4x3 block
        expect = np.einsum("ab,...bc->...ac", k, psi)
        got = W.apply(psi)
        assert rel(got, expect) < 1e-14
        # the dagger of the free operator: k^+
        got_d = W.apply(psi, dagger=True)
        expect_d = np.einsum("ab,...bc->...ac", k.conj().T, psi)
        assert rel(got_d, expect_d) < 1e-14


def test_wilson_scalar_twist_mode(orc):
    """twist_mode=1 is the literal complex mass: M = M(mu=0) + i mu."""
    dims = (4, 4, 4, 4)
    U = synth.thin_links(dims, 11).numpy()
    psi = synth.gaussian_field(dims, 3).numpy()
    a = orc.Wilson(dims, U, 0.1, 0.07, twist_mode=1).apply(psi)
    b = orc.Wilson(dims, U, 0.1, 0.0).apply(psi) + 1j * 0.07 * psi
    assert rel(a, b) < 1e-15


@pytest.fixture(scope="module")
def rough_field():
    dims = (4, 4, 4, 6)
    U = synth.thin_links(dims, 102).numpy()
    return dims, U


def g5(psi):
    out = psi.copy()
    out[..., 2:, :] *= -1
    return out


@pytest.mark.parametrize("twist_mode", [0, 1])
def test_wilson_adjoint_and_gamma5_hermiticity(orc, rough_field, twist_mode):
    dims, U = rough_field
    C = orc.clover(dims, U, 1.05)
    phi = synth.gaussian_field(dims, 5).numpy()
    psi = synth.gaussian_field(dims, 6).numpy()
    Mp = orc.Wilson(dims, U, 0.05, 0.1, clover=C, twist_mode=twist_mode)
    Mm = orc.Wilson(dims, U, 0.05, -0.1, clover=C, twist_mode=twist_mode)
    # adjoint: <phi, M psi> = <M^+ phi, psi>
    lhs = vdot(phi, Mp.apply(psi))
    rhs = vdot(Mp.apply(phi, dagger=True), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    # M(omega)^+ = g5 M(omega*) g5
    assert rel(Mp.apply(psi, dagger=True), g5(Mm.apply(g5(psi)))) < 1e-14


def test_twisted_norm_identity(orc, rough_field):
    """|M(mu) psi|^2 = |M(0) psi|^2 + mu^2 |psi|^2 (twisted reading), with clover."""
    dims, U = rough_field
    C = orc.clover(dims, U, 1.05)
    psi = synth.gaussian_field(dims, 7).numpy()
    mu = 0.23
    a = np.linalg.norm(orc.Wilson(dims, U, 0.05, mu, clover=C).apply(psi)) ** 2
    b = np.linalg.norm(orc.Wilson(dims, U, 0.05, 0.0, clover=C).apply(psi)) ** 2
    c = mu ** 2 * np.linalg.norm(psi) ** 2
    assert abs(a - (b + c)) / a < 1e-13


def test_clover_hermitian_chiral_and_free(orc, rough_field):
    dims, U = rough_field
    C = orc.clover(dims, U, 1.05).reshape(-1, 12, 12)
    assert np.abs(C - np.conj(np.swapaxes(C, -1, -2))).max() < 1e-14
    G5 = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    assert np.abs(C @ G5 - G5 @ C).max() < 1e-14
    assert np.abs(C).max() > 0.05
    C0 = orc.clover(dims, synth.unit_links(dims).numpy(), 1.05)
    assert np.abs(C0).max() == 0.0


@pytest.mark.parametrize("plane", [(0, 1), (0, 2), (1, 3), (2, 3)])
def test_clover_constant_abelian_field_closed_form(orc, plane):
    """Constant abelian field strength in plane (mu,nu): every leaf is e^{iBT}, so
    Fhat = i sin(BT) made traceless and C = -(c_sw/2) sigma_{mu nu} (x) Fhat/i."""
    mu, nu = plane
    dims = (4, 4, 6, 4)
    nflux = 1
    B = 2 * math.pi * nflux / (dims[mu] * dims[nu])
    T = np.array([1.0, 1.0, -2.0])
    U = synth.unit_links(dims).numpy()
    x = coords(dims)
    xm, xn = x[mu], x[nu]
    # U_mu(x) = exp(-i B x_nu T); U_nu(x) = exp(i B L_nu x_mu T) on the last nu slice
    for c in range(3):
        U[mu][..., c, c] = np.exp(-1j * B * xn * T[c])
        last = (xn == dims[nu] - 1)
        U[nu][..., c, c] = np.where(last, np.exp(1j * B * dims[nu] * xm * T[c]), 1.0)
    plaq = orc.plaquette(dims, U)
    assert abs(plaq - (5 + np.mean(np.cos(B * T))) / 6) < 1e-14
    c_sw = 1.3
    C = orc.clover(dims, U, c_sw).reshape(-1, 12, 12)
    g = dr_gammas()
    sigma = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
    S = np.diag(np.sin(B * T))
    S = S - np.trace(S) / 3 * np.eye(3)
    expect = -(c_sw / 2) * np.kron(sigma, S)
    assert np.abs(C - expect[None]).max() < 1e-14


def test_wilson_gauge_covariance(orc, rough_field):
    """M[U'] (g psi) = g M[U] psi with U'_mu(x) = g(x) U_mu(x) g(x+mu)^+, clover rebuilt from U'."""
    dims, U = rough_field
    g = synth.random_su3(dims, 9).numpy()
    U2 = gauge_transform(U, g)
    assert abs(orc.plaquette(dims, U) - orc.plaquette(dims, U2)) < 1e-13
    C = orc.clover(dims, U, 1.05)
    C2 = orc.clover(dims, U2, 1.05)
    G = np.einsum("...ij,ab->...aibj", g, np.eye(4)).reshape(g.shape[:-2] + (12, 12))
    assert np.abs(C2 - G @ C @ np.conj(np.swapaxes(G, -1, -2))).max() < 1e-13
    psi = synth.gaussian_field(dims, 8).numpy()
    gpsi = np.einsum("...ij,...aj->...ai", g, psi)
    a = orc.Wilson(dims, U2, 0.05, 0.1, clover=C2).apply(gpsi)
    b = np.einsum("...ij,...aj->...ai", g, orc.Wilson(dims, U, 0.05, 0.1, clover=C).apply(psi))
    assert rel(a, b) < 1e-13


def dense(apply, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        A[:, j] = apply(e.reshape(shape)).ravel()
    return A


def test_wilson_solvers_against_dense_lu_2x4(orc):
    """Dense LU (192x192) on a 2^4 lattice, where x+mu and x-mu are the same site."""
    dims = (2, 2, 2, 2)
    U = synth.thin_links(dims, 21).numpy()
    C = orc.clover(dims, U, 1.0)
    W = orc.Wilson(dims, U, 0.1, 0.05, clover=C)
    A = dense(W.apply, W.shape())
    b = synth.z2_source(dims, 22).numpy()
    x_lu = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    x_cg, info = W.cgnr(b, tol=1e-13)
    assert info["status"] == 0 and info["true_rel_residual"] < 1e-12
    x_bi, info2 = W.bicgstab(b, tol=1e-13)
    assert info2["status"] == 0
    assert rel(x_cg, x_lu) < 1e-11
    assert rel(x_bi, x_lu) < 1e-11
    # dagger operator is the conjugate transpose of the dense matrix
    Ad = dense(lambda v: W.apply(v, dagger=True), W.shape())
    assert np.abs(Ad - A.conj().T).max() < 1e-14


# ------------------------------------------------------------ staggered pins

def test_staggered_phases_from_spin_diagonalisation(orc):
    """eta_mu(x) 1 = Omega(x)^+ g_mu Omega(x+mu) with Omega = g4^t g1^x g2^y g3^z (MILC)
    or g1^x g2^y g3^z g4^t (CPS), the two orderings of Sec. 2.2."""
    g = dr_gammas()
    mp = np.linalg.matrix_power

    def omega(c, conv):
        x, y, z, t = c
        if conv == 0:
            return mp(g[3], t) @ mp(g[0], x) @ mp(g[1], y) @ mp(g[2], z)
        return mp(g[0], x) @ mp(g[1], y) @ mp(g[2], z) @ mp(g[3], t)

    for conv in (0, 1):
        for x in range(2):
            for y in range(2):
                for z in range(2):
                    for t in range(2):
                        c = [x, y, z, t]
                        for mu in range(4):
                            cp = list(c)
                            cp[mu] += 1
                            m = omega(c, conv).conj().T @ g[mu] @ omega(cp, conv)
                            e = orc.eta(conv, mu, c)
                            assert np.allclose(m, e * np.eye(4)), (conv, c, mu)


def free_hisq(dims):
    V = synth.unit_links(dims).numpy() * (9.0 / 8.0)
    W = synth.unit_links(dims).numpy()
    return V, W


@pytest.mark.parametrize("dims", [(6, 6, 6, 6), (4, 6, 8, 6)])
def test_hisq_free_field_closed_form(orc, dims):
    """V = 9/8, W = 1, c_N = -1/24: H e^{ipx} = i sum_mu eta_mu(x)(9/8 sin p_mu - 1/24 sin 3p_mu) e^{ipx},
    and (m^2 - H^2) e^{ipx} = [m^2 + sum_mu (9/8 sin p_mu - 1/24 sin 3p_mu)^2] e^{ipx}."""
    rng = np.random.default_rng(2)
    V, W = free_hisq(dims)
    m = 0.07
    D = orc.Hisq(dims, V, W, m)
    x = coords(dims)
    for n in [(0, 0, 0, 0), (1, 2, 0, 1), (2, 1, 1, 2)]:
        u = rng.normal(size=3) + 1j * rng.normal(size=3)
        p = [2 * math.pi * n[i] / dims[i] for i in range(3)] + [2 * math.pi * (n[3] + 0.5) / dims[3]]
        ph = np.exp(1j * sum(p[i] * x[i] for i in range(4)))
        psi = ph[..., None] * u
        s = [9 / 8 * math.sin(pp) - 1 / 24 * math.sin(3 * pp) for pp in p]
        etas = [np.vectorize(lambda a, b, c, d, mu=mu: orc.eta(0, mu, (a, b, c, d)))(*x) for mu in range(4)]
        expect = 1j * sum(etas[mu] * s[mu] for mu in range(4))[..., None] * psi
        assert rel(D.hop(psi), expect) < 1e-14
        Hpsi = D.hop(psi)
        got = m * m * psi - D.hop(Hpsi)
        assert rel(got, (m * m + sum(v * v for v in s)) * psi) < 1e-13


@pytest.fixture(scope="module")
def hisq_field():
    dims = (4, 4, 4, 6)
    V = synth.fat_links(dims, 104).numpy()
    W = synth.long_links(dims, 105).numpy()
    return dims, V, W


def test_hisq_antihermitian_and_eps_symmetry(orc, hisq_field):
    dims, V, W = hisq_field
    D = orc.Hisq(dims, V, W, 0.0)
    phi = synth.gaussian_field(dims, 31, ncomp=3).numpy()
    psi = synth.gaussian_field(dims, 32, ncomp=3).numpy()
    lhs = vdot(phi, D.hop(psi))
    rhs = vdot(D.hop(phi, dagger=True), psi)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14
    assert rel(D.hop(psi, dagger=True), -D.hop(psi)) < 1e-14
    x = coords(dims)
    eps = ((-1.0) ** (x[0] + x[1] + x[2] + x[3]))[..., None]
    assert rel(eps * D.hop(eps * psi), -D.hop(psi)) < 1e-14


def test_hisq_gauge_covariance(orc, hisq_field):
    dims, V, W = hisq_field
    g = synth.random_su3(dims, 33).numpy()
    V2 = gauge_transform_k(V, g, 1)
    W2 = gauge_transform_k(W, g, 3)
    psi = synth.gaussian_field(dims, 34, ncomp=3).numpy()
    a = orc.Hisq(dims, V2, W2, 0.1).apply(np.einsum("...ij,...j->...i", g, psi))
    b = np.einsum("...ij,...j->...i", g, orc.Hisq(dims, V, W, 0.1).apply(psi))
    assert rel(a, b) < 1e-13


def test_milc_cps_relation(orc, hisq_field):
    """Sec. 2.2: psi^Chroma(x) = (-1)^{(t%2)((x+y+z)%2) + (x+y+z+t)%2} psi^QUDA(x), where
    QUDA solves (m + H_MILC) and Chroma (m - H_CPS), from a point source at the origin.
    The printed relation carries no overall sign, which fixes the reading of the
    "different sign on the mass term" as m - H_CPS (not -m + H_CPS)."""
    dims, V, W = hisq_field
    m = 0.1
    b = synth.point_source(dims, (0, 0, 0, 0), None, 1).numpy()
    xq, iq = orc.Hisq(dims, V, W, m, conv=0, hop_sign=1).cgnr(b, tol=1e-13)
    xc, ic = orc.Hisq(dims, V, W, m, conv=1, hop_sign=-1).cgnr(b, tol=1e-13)
    assert iq["true_rel_residual"] < 1e-12 and ic["true_rel_residual"] < 1e-12
    x, y, z, t = coords(dims)
    f = ((-1.0) ** ((t % 2) * ((x + y + z) % 2) + (x + y + z + t) % 2))[..., None]
    assert rel(xc, f * xq) < 1e-11
    # without the phase map the two differ
    assert rel(xc, xq) > 0.1


def test_hisq_multishift_against_dense_lu_2x4(orc):
    dims = (2, 2, 2, 2)
    V = synth.fat_links(dims, 41).numpy()
    W = synth.long_links(dims, 42).numpy()
    b = synth.z2_source(dims, 43, ncomp=3).numpy()
    masses = [0.05, 0.1, 0.2, 0.5]
    xs, info = orc.Hisq(dims, V, W, 0.0).multishift(b, masses, tol=1e-13)
    assert info["status"] == 0
    for m, x in zip(masses, xs):
        D = orc.Hisq(dims, V, W, m)
        A = dense(D.apply, D.shape())
        x_lu = np.linalg.solve(A, b.ravel()).reshape(b.shape)
        assert rel(x, x_lu) < 1e-11


def test_hisq_multishift_equals_independent_solves(orc, hisq_field):
    dims, V, W = hisq_field
    b = synth.z2_source(dims, 44, ncomp=3).numpy()
    masses = [0.02, 0.05, 0.1, 0.3]
    xs, info = orc.Hisq(dims, V, W, 0.0).multishift(b, masses, tol=1e-12)
    assert info["status"] == 0
    assert max(info["true_rel_residual"]) < 1e-10
    for m, x in zip(masses, xs):
        xi, ii = orc.Hisq(dims, V, W, m).cgnr(b, tol=1e-12)
        assert rel(x, xi) < 1e-9


# ------------------------------------------------------------ overlap pins
# Sec. 2.3: eps(H_w) ~ x P(x^2) with a Chebyshev polynomial evaluated by Clenshaw.

def test_clenshaw_equals_cosine_series(orc):
    """The recurrence reproduces sum_k c_k T_k(z) with T_k(z) = cos(k arccos z)."""
    rng = np.random.default_rng(5)
    c = rng.normal(size=40)
    z = np.linspace(-1, 1, 101)
    direct = sum(c[k] * np.cos(k * np.arccos(z)) for k in range(len(c)))
    assert np.max(np.abs(orc.clenshaw(c, z) - direct)) < 1e-12
    # and on vectors through an operator: a diagonal Z gives the same numbers
    v = rng.normal(size=101)
    got = orc.clenshaw(c, v, matvec=lambda w: z * w)
    assert np.max(np.abs(got - direct * v)) < 1e-12


def test_chebyshev_sign_interpolates_and_meets_the_bound(orc):
    """The polynomial equals 1/sqrt(y) at its Chebyshev nodes, and |1 - x P(x^2)|
    stays below the bound on random points of [eps, 1] not used to choose the order."""
    eps, delta = 0.05, 1e-5
    c, dev = orc.chebyshev_sign_coeffs(eps, delta)
    n = len(c)
    a, b = eps * eps, 1.0
    theta = np.pi * (np.arange(n) + 0.5) / n
    y = 0.5 * ((b - a) * np.cos(theta) + a + b)
    assert np.max(np.abs(orc.clenshaw(c, np.cos(theta)) - 1 / np.sqrt(y))) < 1e-9
    x = np.random.default_rng(6).uniform(eps, 1.0, size=20000)
    z = (2 * x * x - a - b) / (b - a)
    assert np.max(np.abs(1 - x * orc.clenshaw(c, z))) <= 1.2 * delta
    assert dev <= delta


def _dense(op, shape):
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=complex)
        e[j] = 1
        cols.append(op(e.reshape(shape)).ravel())
    return np.array(cols).T


def test_overlap_sign_against_dense_eigendecomposition_2x4(orc):
    """On 2^4 (192 x 192): g5 D_w(-rho) is hermitian, and the Chebyshev/Clenshaw sign
    function applied to a vector equals V sign(L) V^+ v from the exact eigensystem
    within the deviation bound; applied twice it is the identity."""
    dims, rho, delta = (2, 2, 2, 2), 1.5, 1e-6
    U = synth.thin_links(dims, 71, 0.3).numpy()
    hw = orc.hermitian_wilson(dims, U, rho)
    shape = (2, 2, 2, 2, 4, 3)
    H = _dense(hw, shape)
    assert np.max(np.abs(H - H.conj().T)) < 1e-13
    lam, V = np.linalg.eigh(H)
    lmin, lmax = 0.9 * np.min(np.abs(lam)), 1.1 * np.max(np.abs(lam))
    c, dev = orc.chebyshev_sign_coeffs(lmin / lmax, delta)
    v = synth.gaussian_field(dims, 72).numpy()
    exact = (V @ (np.sign(lam) * (V.conj().T @ v.ravel()))).reshape(shape)
    got = orc.overlap_sign(hw, v, lmin, lmax, c)
    assert np.linalg.norm(got - exact) <= 2 * delta * np.linalg.norm(v)
    twice = orc.overlap_sign(hw, got, lmin, lmax, c)
    assert np.linalg.norm(twice - v) <= 4 * delta * np.linalg.norm(v)


@pytest.mark.parametrize("dagger", [False, True])
def test_site_sampled_operators_equal_full_lattice_ones(orc, rough_field, hisq_field, dagger):
    """The site-list forms of the oracle (used by the full-size GPU tests, where
    the whole-lattice operator is too slow to repeat) give exactly the values of
    the whole-lattice operator at the same sites, in any site order, for the
    Wilson hopping term, the clover twisted-mass operator and the HISQ hop."""
    dims, U = rough_field
    C = orc.clover(dims, U, 1.05)
    psi = synth.gaussian_field(dims, 61).numpy()
    V = int(np.prod(dims))
    sites = np.random.default_rng(62).permutation(V)[: V // 3]
    W = orc.Wilson(dims, U, 0.05, 0.1, clover=C)
    assert np.array_equal(W.hop_sites(psi, sites, dagger=dagger),
                          W.hop(psi, dagger=dagger).reshape(V, 4, 3)[sites])
    assert np.array_equal(W.apply_sites(psi, sites, dagger=dagger),
                          W.apply(psi, dagger=dagger).reshape(V, 4, 3)[sites])
    hdims, Vf, Wl = hisq_field
    H = orc.Hisq(hdims, Vf, Wl, 0.0)
    chi = synth.gaussian_field(hdims, 63, ncomp=3).numpy()
    hv = int(np.prod(hdims))
    hsites = np.random.default_rng(64).permutation(hv)[: hv // 3]
    assert np.array_equal(H.hop_sites(chi, hsites, dagger=dagger), H.hop(chi, dagger=dagger).reshape(hv, 3)[hsites])
