"""FP64 CPU oracle: test infrastructure, never part of the product path.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. It wraps ``oracle.c`` (plain C, FP64,
full lattice) through ctypes and shares no code with the CUDA library;
the only thing both sides read is the seeded input from ``synth.py``.

Every function takes and returns canonical complex128 arrays:
gauge (4, Lt, Lz, Ly, Lx, 3, 3), Wilson spinor (Lt, Lz, Ly, Lx, 4, 3),
staggered vector (Lt, Lz, Ly, Lx, 3), clover (Lt, Lz, Ly, Lx, 12, 12);
dims are given as (Lx, Ly, Lz, Lt).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")


def _host_tag() -> str:
    """A tag of this host's CPU (model and instruction-set flags): the library is
    built with -march=native, so a copy built on another machine is not reused."""
    import hashlib
    import platform
    text = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith(("model name", "flags")):
                    text += line
                    if line.startswith("flags"):
                        break
    except OSError:
        pass
    return hashlib.sha1(text.encode()).hexdigest()[:10]


_LIB = os.path.join(_HERE, f"liboracle_{_host_tag()}.so")


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O3 -march=native, OpenMP; ISO C11, so no floating-point
    contraction, and no fast-math: every operation rounds as written) into a library
    named for this host's CPU."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O3", "-march=native", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Wilson(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("bc_t", ctypes.c_int), ("U", ctypes.c_void_p),
                ("clover", ctypes.c_void_p), ("m", ctypes.c_double), ("mu", ctypes.c_double),
                ("twist_mode", ctypes.c_int)]


class _Hisq(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("bc_t", ctypes.c_int), ("V", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("c_naik", ctypes.c_double), ("m", ctypes.c_double),
                ("conv", ctypes.c_int), ("hop_sign", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_plaquette.restype = ctypes.c_double
        _lib.or_wilson_cgnr_fixed.restype = ctypes.c_double
        _lib.or_get_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's site loops use from now on."""
    lib().or_set_threads(ctypes.c_int(int(n)))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _c(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def _np(a):
    """Accept torch tensors or numpy arrays."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return _c(a)


def gamma(mu: int) -> np.ndarray:
    """The oracle's gamma matrix mu (0..3 for x,y,z,t; 4 for gamma_5)."""
    out = np.zeros((4, 4, 2))
    lib().or_gamma(ctypes.c_int(mu), out.ctypes.data_as(ctypes.c_void_p))
    return out[..., 0] + 1j * out[..., 1]


def eta(conv: int, mu: int, coords) -> float:
    out = ctypes.c_double()
    c = (ctypes.c_int * 4)(*coords)
    lib().or_staggered_eta(ctypes.c_int(conv), ctypes.c_int(mu), c, ctypes.byref(out))
    return out.value


def plaquette(dims, U) -> float:
    U = _np(U)
    return lib().or_plaquette(_dims(dims), _p(U))


class Wilson:
    """Wilson twisted-mass (optionally clover) operator M of Sec. 2.1 Eq. 2-3."""

    def __init__(self, dims, U, m, mu, clover=None, bc_t=-1, twist_mode=0):
        self.dims = tuple(int(d) for d in dims)
        self.U = _np(U)
        self.clover = _np(clover) if clover is not None else None
        self.s = _Wilson(_dims(dims), bc_t, self.U.ctypes.data,
                         self.clover.ctypes.data if self.clover is not None else None,
                         float(m), float(mu), int(twist_mode))
        self.bc_t = bc_t

    def shape(self):
        lx, ly, lz, lt = self.dims
        return (lt, lz, ly, lx, 4, 3)

    def apply(self, psi, dagger=False):
        psi = _np(psi)
        out = np.empty(self.shape(), dtype=np.complex128)
        lib().or_wilson_apply(ctypes.byref(self.s), ctypes.c_int(int(dagger)), _p(psi), _p(out))
        return out

    def hop(self, psi, dagger=False):
        psi = _np(psi)
        out = np.empty(self.shape(), dtype=np.complex128)
        lib().or_wilson_hop(_dims(self.dims), ctypes.c_int(self.bc_t), _p(self.U), ctypes.c_int(int(dagger)),
                            _p(psi), _p(out))
        return out

    def apply_sites(self, psi, sites, dagger=False):
        psi = _np(psi)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.empty((len(sites), 4, 3), dtype=np.complex128)
        lib().or_wilson_apply_sites(ctypes.byref(self.s), ctypes.c_int(int(dagger)), _p(psi),
                                    ctypes.c_void_p(sites.ctypes.data), ctypes.c_int64(len(sites)), _p(out))
        return out

    def hop_sites(self, psi, sites, dagger=False):
        psi = _np(psi)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.empty((len(sites), 4, 3), dtype=np.complex128)
        lib().or_wilson_hop_sites(_dims(self.dims), ctypes.c_int(self.bc_t), _p(self.U),
                                  ctypes.c_int(int(dagger)), _p(psi), ctypes.c_void_p(sites.ctypes.data),
                                  ctypes.c_int64(len(sites)), _p(out))
        return out

    def _solve(self, fn, b, tol, maxiter):
        b = _np(b)
        x = np.zeros(self.shape(), dtype=np.complex128)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        st = fn(ctypes.byref(self.s), _p(b), _p(x), ctypes.c_double(tol), ctypes.c_int(maxiter),
                ctypes.byref(it), ctypes.byref(rel))
        return x, {"status": st, "iters": it.value, "true_rel_residual": rel.value}

    def cgnr(self, b, tol=1e-12, maxiter=100000):
        return self._solve(lib().or_wilson_cgnr, b, tol, maxiter)

    def bicgstab(self, b, tol=1e-12, maxiter=100000):
        return self._solve(lib().or_wilson_bicgstab, b, tol, maxiter)

    def cgnr_fixed(self, b, niter):
        """niter CGNR iterations from x = 0 (a bounded timing sample); returns x, rel. residual."""
        b = _np(b)
        x = np.zeros(self.shape(), dtype=np.complex128)
        rel = lib().or_wilson_cgnr_fixed(ctypes.byref(self.s), _p(b), _p(x), ctypes.c_int(niter))
        return x, rel


def clover(dims, U, c_sw):
    """Clover term C(x) (Sec. 2.1 Eq. 3), shape (Lt, Lz, Ly, Lx, 12, 12)."""
    U = _np(U)
    lx, ly, lz, lt = (int(d) for d in dims)
    out = np.empty((lt, lz, ly, lx, 12, 12), dtype=np.complex128)
    lib().or_clover_build(_dims(dims), _p(U), ctypes.c_double(c_sw), _p(out))
    return out


class Hisq:
    """Staggered/HISQ operator D = m + s_h H of Sec. 2.2 Eq. 4 (s_h = hop_sign)."""

    def __init__(self, dims, V, W, m, c_naik=-1.0 / 24.0, bc_t=-1, conv=0, hop_sign=1):
        self.dims = tuple(int(d) for d in dims)
        self.V = _np(V)
        self.W = _np(W) if W is not None else None
        self.s = _Hisq(_dims(dims), bc_t, self.V.ctypes.data,
                       self.W.ctypes.data if self.W is not None else None,
                       float(c_naik), float(m), int(conv), int(hop_sign))

    def shape(self):
        lx, ly, lz, lt = self.dims
        return (lt, lz, ly, lx, 3)

    def apply(self, psi, dagger=False):
        psi = _np(psi)
        out = np.empty(self.shape(), dtype=np.complex128)
        lib().or_hisq_apply(ctypes.byref(self.s), ctypes.c_int(int(dagger)), _p(psi), _p(out))
        return out

    def hop(self, psi, dagger=False):
        psi = _np(psi)
        out = np.empty(self.shape(), dtype=np.complex128)
        lib().or_hisq_hop(ctypes.byref(self.s), ctypes.c_int(int(dagger)), _p(psi), _p(out))
        return out

    def hop_sites(self, psi, sites, dagger=False):
        psi = _np(psi)
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        out = np.empty((len(sites), 3), dtype=np.complex128)
        lib().or_hisq_hop_sites(ctypes.byref(self.s), ctypes.c_int(int(dagger)), _p(psi),
                                ctypes.c_void_p(sites.ctypes.data), ctypes.c_int64(len(sites)), _p(out))
        return out

    def cgnr(self, b, tol=1e-12, maxiter=100000):
        b = _np(b)
        x = np.zeros(self.shape(), dtype=np.complex128)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        st = lib().or_hisq_cgnr(ctypes.byref(self.s), _p(b), _p(x), ctypes.c_double(tol), ctypes.c_int(maxiter),
                                ctypes.byref(it), ctypes.byref(rel))
        return x, {"status": st, "iters": it.value, "true_rel_residual": rel.value}

    def multishift(self, b, masses, tol=1e-12, maxiter=100000):
        """Solves (m_i + s_h H) x_i = b for all masses (ascending) with one multi-shift CG."""
        b = _np(b)
        masses = np.ascontiguousarray(masses, dtype=np.float64)
        xs = [np.zeros(self.shape(), dtype=np.complex128) for _ in masses]
        ptrs = (ctypes.c_void_p * len(xs))(*[x.ctypes.data for x in xs])
        it = ctypes.c_int()
        rel = np.zeros(len(masses))
        st = lib().or_hisq_multishift(ctypes.byref(self.s), ctypes.c_int(len(masses)),
                                      ctypes.c_void_p(masses.ctypes.data), _p(b), ptrs, ctypes.c_double(tol),
                                      ctypes.c_int(maxiter), ctypes.byref(it), ctypes.c_void_p(rel.ctypes.data))
        return xs, {"status": st, "iters": it.value, "true_rel_residual": rel.tolist()}


# ------------------------------------------------------------------ overlap
# Building blocks of the overlap operator (Sec. 2.3): H_w = g5 D_w(-rho) and its
# sign function approximated by eps(x) ~ x P(x^2), x = H_w / lambda_max, with P a
# Chebyshev polynomial of 1/sqrt(y) on [eps^2, 1] evaluated by the Clenshaw
# recurrence. Written from the paper's description; the CUDA library computes its
# own coefficients.

def hermitian_wilson(dims, U, rho, bc_t=-1):
    """The operator v -> g5 D_w(-rho) v (D_w(-rho) = (4 - rho) - H in the sign reading of the Wilson operator used throughout)."""
    W = Wilson(dims, U, -rho, 0.0, bc_t=bc_t)
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[:, None]

    def apply(v):
        return g5 * W.apply(v)
    return apply


def chebyshev_nodes_coeffs(f, a, b, n):
    """Coefficients c_k (c_0 halved) of the degree n-1 polynomial interpolating f at
    the n Chebyshev nodes of [a, b], in the basis T_k((2y - a - b)/(b - a))."""
    j = np.arange(n)
    theta = np.pi * (j + 0.5) / n
    y = 0.5 * ((b - a) * np.cos(theta) + a + b)
    fy = f(y)
    k = np.arange(n)[:, None]
    c = 2.0 / n * (np.cos(k * theta[None, :]) @ fy)
    c[0] *= 0.5
    return c


def clenshaw(c, z, matvec=None):
    """sum_k c_k T_k(z): z a number or array (matvec None), or, with matvec the map
    v -> Z v, the vector sum_k c_k T_k(Z) z (z then the vector)."""
    if matvec is None:
        b1 = np.zeros_like(np.asarray(z, dtype=float))
        b2 = np.zeros_like(b1)
        for ck in c[:0:-1]:
            b1, b2 = ck + 2.0 * z * b1 - b2, b1
        return c[0] + z * b1 - b2
    v = z
    b1 = np.zeros_like(v)
    b2 = np.zeros_like(v)
    for ck in c[:0:-1]:
        b1, b2 = ck * v + 2.0 * matvec(b1) - b2, b1
    return c[0] * v + matvec(b1) - b2


def sign_deviation(c, eps, npts=3000):
    """max over x in [eps, 1] of |1 - x P(x^2)|, log-spaced and linear samples."""
    x = np.concatenate([eps * (1.0 / eps) ** (np.arange(npts + 1) / npts), eps + (1 - eps) * np.arange(npts + 1) / npts])
    a, b = eps * eps, 1.0
    z = (2 * x * x - a - b) / (b - a)
    return float(np.max(np.abs(1.0 - x * clenshaw(c, z))))


def chebyshev_sign_coeffs(eps, delta, max_order=65536):
    """The smallest number of terms (doubling from 8, then bisection) whose sign
    deviation on [eps, 1] is <= delta; returns (coeffs, deviation)."""
    a, b = eps * eps, 1.0
    f = lambda y: 1.0 / np.sqrt(y)
    hi = 8
    while True:
        c = chebyshev_nodes_coeffs(f, a, b, hi)
        if sign_deviation(c, eps) <= delta:
            break
        if hi >= max_order:
            raise ValueError("more than max_order terms needed")
        hi = min(2 * hi, max_order)
    lo = hi // 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if sign_deviation(chebyshev_nodes_coeffs(f, a, b, mid), eps) <= delta:
            hi = mid
        else:
            lo = mid
    c = chebyshev_nodes_coeffs(f, a, b, hi)
    return c, sign_deviation(c, eps)


def overlap_sign(hw, v, lambda_min, lambda_max, coeffs):
    """(H/lmax) P((H/lmax)^2) v by Clenshaw, hw the map v -> H_w v."""
    eps = lambda_min / lambda_max
    a, b = eps * eps, 1.0

    def Z(w):
        return (2.0 * hw(hw(w)) / lambda_max ** 2 - (a + b) * w) / (b - a)
    pv = clenshaw(coeffs, v, matvec=Z)
    return hw(pv) / lambda_max


def hermitian_wilson_dense(dims, U, rho, bc_t=-1):
    """The matrix of v -> g5 D_w(-rho) v in the canonical ordering (site-major,
    spin, colour), built column by column from unit vectors (small lattices)."""
    hw = hermitian_wilson(dims, U, rho, bc_t)
    lx, ly, lz, lt = dims
    n = lx * ly * lz * lt * 12
    H = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        H[:, j] = hw(e.reshape(lt, lz, ly, lx, 4, 3)).ravel()
        e[j] = 0.0
    return H


def hw_low_modes(dims, U, rho, nev, bc_t=-1):
    """The nev eigenpairs of g5 D_w(-rho) with the smallest |lambda| (the target of
    the eigensolver of Sec. 2.3), by a dense hermitian eigendecomposition: (evals
    in ascending |lambda|, evecs as canonical spinors, the whole spectrum ascending)."""
    H = hermitian_wilson_dense(dims, U, rho, bc_t)
    w, Z = np.linalg.eigh(H)
    idx = np.argsort(np.abs(w), kind="stable")[:nev]
    lx, ly, lz, lt = dims
    return w[idx], [Z[:, i].reshape(lt, lz, ly, lx, 4, 3) for i in idx], w


def sign_exact(dims, U, rho, v, bc_t=-1):
    """eps(H_w) v from the dense eigendecomposition: Z sign(Lambda) Z^+ v."""
    H = hermitian_wilson_dense(dims, U, rho, bc_t)
    w, Z = np.linalg.eigh(H)
    return (Z @ (np.sign(w) * (Z.conj().T @ v.ravel()))).reshape(v.shape)
