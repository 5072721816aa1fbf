"""The eigensolver's host pieces, CPU only: the dense hermitian
eigen-decomposition of its projected matrices (cyclic Jacobi, csrc/herm_eig.h,
compiled with g++ against the header alone; eigenvalues against numpy's LAPACK
routine, eigenvectors by A V = V diag(w) and V^+ V = 1, on random, diagonal,
degenerate and 1x1 matrices), and the oracle's low modes of g5 D_w(-rho) pinned
to the free-field spectrum in closed form."""
import os
import subprocess

import numpy as np
import pytest

from helpers import ROOT

DRIVER = r"""
#include <cstdio>
#include "herm_eig.h"
int main() {
    int m;
    if (std::scanf("%d", &m) != 1) return 1;
    std::vector<lq::zcx> A((size_t)m * m);
    for (auto& a : A) { double re, im; if (std::scanf("%lf %lf", &re, &im) != 2) return 1; a = lq::zcx(re, im); }
    std::vector<double> w; std::vector<lq::zcx> V;
    lq::herm_eig(m, A, w, V);
    for (double x : w) std::printf("%.17e\n", x);
    for (auto& v : V) std::printf("%.17e %.17e\n", v.real(), v.imag());
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("herm")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2201_09004_b300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    return str(exe)


def run(driver, A):
    m = A.shape[0]
    inp = f"{m}\n" + "\n".join(f"{z.real:.17e} {z.imag:.17e}" for z in A.ravel()) + "\n"
    out = subprocess.run([driver], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    w = np.array([float(x) for x in out[:m]])
    V = np.array([complex(float(a), float(b)) for a, b in (l.split() for l in out[m:m + m * m])]).reshape(m, m)
    return w, V


def check(A, w, V):
    m = A.shape[0]
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12 * max(1.0, np.abs(A).max()), rtol=0)
    assert np.allclose(V.conj().T @ V, np.eye(m), atol=1e-12)
    assert np.allclose(A @ V, V * w[None, :], atol=1e-11 * max(1.0, np.abs(A).max()))


@pytest.mark.parametrize("m", [1, 2, 5, 17, 48])
def test_random_hermitian(driver, m):
    rng = np.random.default_rng(m)
    X = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    A = (X + X.conj().T) / 2
    w, V = run(driver, A)
    check(A, w, V)


def test_degenerate_and_diagonal(driver):
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12)))
    d = np.array([-3.0, -3.0, -3.0, 0.5, 0.5, 1.0, 2.0, 2.0, 2.0, 2.0, 7.0, 1e-9])
    A = Q @ np.diag(d) @ Q.conj().T
    w, V = run(driver, A)
    check(A, w, V)
    D = np.diag(np.array([4.0, -1.0, 2.5]) + 0j)
    w, V = run(driver, D)
    assert np.allclose(w, [-1.0, 2.5, 4.0])
    check(D, w, V)


def test_oracle_free_field_hw_spectrum(orc):
    """Pins the oracle's low-mode function: on the free field g5 D_w(-rho) acts on a
    plane wave of momentum p as a 4x4 matrix whose square is
    E(p)^2 = (4 - rho - sum_mu cos p_mu)^2 + sum_mu sin^2 p_mu (the gamma matrices
    anticommute), with trace 0, so its spectrum is +-E(p), each six-fold (two
    spins, three colours); p_mu = 2 pi n / L, and p_t = 2 pi (n + 1/2) / L_t for
    the antiperiodic time direction."""
    from paper_2201_09004_b300 import synth
    dims = (2, 2, 2, 4)
    rho = 1.5
    U = synth.unit_links(dims).numpy()
    _, _, w = orc.hw_low_modes(dims, U, rho, 4)
    lx, ly, lz, lt = dims
    E = []
    for nx in range(lx):
        for ny in range(ly):
            for nz in range(lz):
                for nt in range(lt):
                    p = [2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz, 2 * np.pi * (nt + 0.5) / lt]
                    E.append(np.sqrt((4 - rho - sum(np.cos(p))) ** 2 + sum(np.sin(q) ** 2 for q in p)))
    expected = np.sort([s * e for e in E for s in (1.0, -1.0) for _ in range(6)])
    assert np.allclose(np.sort(w), expected, atol=1e-12)


def test_oracle_low_modes_and_exact_sign(orc):
    """On a random field: the returned pairs have the smallest |lambda| of the full
    spectrum and satisfy H z = lambda z; the exact sign squares to one and
    commutes with H_w."""
    from paper_2201_09004_b300 import synth
    dims = (2, 2, 2, 2)
    U = synth.thin_links(dims, 3).numpy()
    ev, Z, w = orc.hw_low_modes(dims, U, 1.5, 5)
    assert np.allclose(np.sort(np.abs(ev)), np.sort(np.abs(w))[:5])
    hw = orc.hermitian_wilson(dims, U, 1.5)
    for lam, z in zip(ev, Z):
        assert np.linalg.norm(hw(z) - lam * z) < 1e-12
    v = synth.gaussian_field(dims, 4).numpy()
    s = orc.sign_exact(dims, U, 1.5, v)
    assert np.allclose(orc.sign_exact(dims, U, 1.5, s), v, atol=1e-12)
    assert np.allclose(hw(s), orc.sign_exact(dims, U, 1.5, hw(v)), atol=1e-11)
