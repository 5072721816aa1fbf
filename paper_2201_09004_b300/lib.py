"""Thin ctypes binding of the C ABI in include/lq.h (argument marshalling only).

Every operation runs in the CUDA library ``liblq.so`` built from ``csrc/``;
this module converts arrays to pointers and status codes to exceptions. There
is no fallback: if the library is missing or fails to load, ``lib()`` raises.

Arrays may be numpy arrays / CPU tensors (host memory, ``loc = LQ_HOST``) or
CUDA torch tensors (``loc = LQ_DEVICE``), always complex128 in the canonical
layouts of lq.h: gauge (4, Lt, Lz, Ly, Lx, 3, 3), Wilson spinor
(Lt, Lz, Ly, Lx, 4, 3), staggered vector (Lt, Lz, Ly, Lx, 3).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblq.so")

# enums of lq.h
LQ_OK, LQ_EINVAL, LQ_ENOMEM, LQ_ENOTCONV, LQ_EBREAKDOWN, LQ_ENAN, LQ_EAGAIN, LQ_ETIMEOUT, LQ_ECUDA, LQ_EBUSY = range(10)
F64, F32, F16, F32X2 = 0, 1, 2, 3
R18, R12, R8 = 18, 12, 8
TWIST_GAMMA5, TWIST_SCALAR = 0, 1
THIN, FAT, LONG = 0, 1, 2
HOST, DEVICE = 0, 1
WILSON_TM, WILSON_TM_CLOVER, HISQ = 0, 1, 2
CGNR, MIXED_CGNR, MULTISHIFT_CG, BICGSTAB, GCR = 0, 1, 2, 3, 4
OP_FULL, OP_SCHUR = 0, 1
WILSON_FIELD, STAGGERED_FIELD = 0, 1

STATUS_NAMES = {0: "LQ_OK", 1: "LQ_EINVAL", 2: "LQ_ENOMEM", 3: "LQ_ENOTCONV", 4: "LQ_EBREAKDOWN",
                5: "LQ_ENAN", 6: "LQ_EAGAIN", 7: "LQ_ETIMEOUT", 8: "LQ_ECUDA", 9: "LQ_EBUSY"}

# every function lq.h declares (checked by the CPU test of the boundary)
EXPORTS = [
    "lq_last_error", "lq_create_lattice", "lq_destroy_lattice", "lq_lattice_bytes", "lq_lattice_release_workspace", "lq_load_gauge",
    "lq_load_clover", "lq_dslash_apply", "lq_operator_apply", "lq_solve", "lq_field_create",
    "lq_field_destroy", "lq_field_import", "lq_field_export", "lq_dslash_field", "lq_schur_field",
    "lq_profile_enable", "lq_profile_reset", "lq_profile_query", "lq_launch_count", "lq_tune_reset", "lq_tune_force", "lq_gamma5_dw_apply", "lq_chebyshev_sign",
    "lq_overlap_sign_apply", "lq_hw_eigensolve", "lq_overlap_sign_apply_deflated", "lq_server_create",
    "lq_server_destroy", "lq_submit", "lq_poll", "lq_wait", "lq_server_stats", "lq_dslash_apply_noalloc", "lq_request_bytes",
    "lq_barrier_selftest",
]


class LqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class OpParams(ctypes.Structure):
    _fields_ = [("action", ctypes.c_int), ("m", ctypes.c_double), ("mu", ctypes.c_double),
                ("c_sw", ctypes.c_double), ("c_naik", ctypes.c_double), ("recon", ctypes.c_int),
                ("twist_mode", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("maxiter", ctypes.c_int), ("prec_sloppy", ctypes.c_int), ("recon_sloppy", ctypes.c_int),
                ("nshift", ctypes.c_int), ("masses", ctypes.POINTER(ctypes.c_double)),
                ("graph_iters", ctypes.c_int), ("restart", ctypes.c_int), ("persistent", ctypes.c_int),
                ("update_f32_below", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("operator_applications", ctypes.c_int), ("true_rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SignInfo(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("max_deviation", ctypes.c_double)]


class EigParams(ctypes.Structure):
    _fields_ = [("nev", ctypes.c_int), ("nkv", ctypes.c_int), ("degree", ctypes.c_int),
                ("lambda_cut", ctypes.c_double), ("lambda_max", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_restarts", ctypes.c_int)]


class EigInfo(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("restarts", ctypes.c_int), ("operator_applications", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_void_p), ("op", OpParams), ("solve", SolveParams), ("nrhs", ctypes.c_int)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_double), ("admitted", ctypes.c_double), ("finished", ctypes.c_double)]


_lib = None


def lib():
    """Loads liblq.so; raises if it is missing (there is no other code path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run python -m paper_2201_09004_b300.build)")
        L = ctypes.CDLL(LIB_PATH)
        L.lq_last_error.restype = ctypes.c_char_p
        L.lq_launch_count.restype = ctypes.c_int64
        for name in EXPORTS:
            getattr(L, name)
        _lib = L
    return _lib


def _check(code):
    if code != LQ_OK:
        raise LqError(code, lib().lq_last_error().decode(errors="replace"))
    return code


def _is_torch(a):
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _ptr(a):
    """(pointer, loc, keepalive) of a complex128 array."""
    if _is_torch(a):
        if a.is_cuda:
            if not a.is_contiguous():
                raise ValueError("device tensors must be contiguous")
            return ctypes.c_void_p(a.data_ptr()), DEVICE, a
        a = a.numpy()
    if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
        a = np.ascontiguousarray(a, dtype=np.complex128)
    return ctypes.c_void_p(a.ctypes.data), HOST, a


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def op_params(action, m, mu=0.0, c_sw=0.0, c_naik=-1.0 / 24.0, recon=0, twist_mode=0):
    """recon: link compression of the operator-apply calls at F32 / F16 (0 = R12).
    twist_mode: TWIST_GAMMA5 (i mu g5) or TWIST_SCALAR (i mu)."""
    return OpParams(int(action), float(m), float(mu), float(c_sw), float(c_naik), int(recon), int(twist_mode))


def solve_params(solver=MIXED_CGNR, tol=1e-10, delta=0.1, maxiter=100000, prec_sloppy=F32, recon_sloppy=R12,
                 masses=None, graph_iters=0, restart=0, persistent=0, update_f32_below=0.0):
    sp = SolveParams(int(solver), float(tol), float(delta), int(maxiter), int(prec_sloppy), int(recon_sloppy), 0, None,
                     int(graph_iters), int(restart), int(persistent), float(update_f32_below))
    if masses is not None:
        arr = (ctypes.c_double * len(masses))(*[float(m) for m in masses])
        sp.nshift = len(masses)
        sp.masses = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        sp._keep = arr
    return sp


class Lattice:
    """A lattice with its resident gauge / clover fields (lq_lattice)."""

    def __init__(self, dims, t_boundary=-1):
        self.dims = tuple(int(d) for d in dims)
        h = ctypes.c_void_p()
        _check(lib().lq_create_lattice((ctypes.c_int * 4)(*self.dims), ctypes.c_int(t_boundary), ctypes.byref(h)))
        self.h = h
        lx, ly, lz, lt = self.dims
        self.volume = lx * ly * lz * lt

    def close(self):
        if self.h:
            lib().lq_destroy_lattice(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def device_bytes(self):
        b = ctypes.c_size_t()
        _check(lib().lq_lattice_bytes(self.h, ctypes.byref(b)))
        return b.value

    def release_workspace(self):
        """Frees the idle solver work buffers kept between solves; returns the device bytes freed."""
        b = ctypes.c_size_t()
        _check(lib().lq_lattice_release_workspace(self.h, ctypes.byref(b)))
        return b.value

    def load_gauge(self, kind, links):
        p, loc, keep = _ptr(links)
        _check(lib().lq_load_gauge(self.h, ctypes.c_int(kind), ctypes.c_int(loc), p))

    def load_clover(self, c_sw, clover=None):
        if clover is None:
            _check(lib().lq_load_clover(self.h, ctypes.c_int(DEVICE), None, ctypes.c_double(c_sw)))
        else:
            p, loc, keep = _ptr(clover)
            _check(lib().lq_load_clover(self.h, ctypes.c_int(loc), p, ctypes.c_double(c_sw)))

    def _out_like(self, x):
        if _is_torch(x) and x.is_cuda:
            import torch
            return torch.empty_like(x)
        return np.empty(np.shape(x), dtype=np.complex128)

    def dslash_apply(self, op, parity, psi, dagger=False, prec=F64, stream=None):
        p, loc, keep = _ptr(psi)
        out = self._out_like(psi)
        po, loco, keepo = _ptr(out)
        _check(lib().lq_dslash_apply(self.h, ctypes.byref(op), ctypes.c_int(parity), ctypes.c_int(int(dagger)),
                                     ctypes.c_int(prec), ctypes.c_int(loc), p, po, _stream(stream)))
        return out

    def dslash_apply_noalloc(self, op, parity, psi, out, dagger=False, prec=F64, stream=None):
        """lq_dslash_apply_noalloc: device tensors in/out, no device allocation in the library.
        The library writes V * ncomp complex128 entries into out, so both tensors are
        checked for that size, dtype and device before the call."""
        import torch
        if not (_is_torch(psi) and psi.is_cuda and _is_torch(out) and out.is_cuda):
            raise ValueError("lq_dslash_apply_noalloc takes device tensors")
        ncomp = 3 if op.action == HISQ else 12
        for name, t in (("psi", psi), ("out", out)):
            if t.dtype != torch.complex128:
                raise ValueError(f"{name} must be complex128, got {t.dtype}")
            if t.numel() != self.volume * ncomp:
                raise ValueError(f"{name} must hold {self.volume * ncomp} entries for this lattice, got {t.numel()}")
        if psi.device != out.device:
            raise ValueError("psi and out must be on the same device")
        p, loc, keep = _ptr(psi)
        po, loco, keepo = _ptr(out)
        _check(lib().lq_dslash_apply_noalloc(self.h, ctypes.byref(op), ctypes.c_int(parity), ctypes.c_int(int(dagger)),
                                             ctypes.c_int(prec), p, po, _stream(stream)))
        return out

    def operator_apply(self, op, psi, form=OP_FULL, dagger=False, prec=F64, stream=None):
        p, loc, keep = _ptr(psi)
        out = self._out_like(psi)
        po, loco, keepo = _ptr(out)
        _check(lib().lq_operator_apply(self.h, ctypes.byref(op), ctypes.c_int(form), ctypes.c_int(int(dagger)),
                                       ctypes.c_int(prec), ctypes.c_int(loc), p, po, _stream(stream)))
        return out

    def gamma5_dw_apply(self, rho, psi, prec=F64, stream=None):
        """g5 D_w(-rho) psi on the full lattice (the hermitian Wilson operator of the overlap)."""
        p, loc, keep = _ptr(psi)
        out = self._out_like(psi)
        po, loco, keepo = _ptr(out)
        _check(lib().lq_gamma5_dw_apply(self.h, ctypes.c_double(rho), ctypes.c_int(prec), ctypes.c_int(loc), p, po,
                                        _stream(stream)))
        return out

    def overlap_sign_apply(self, rho, lambda_min, lambda_max, delta, psi, prec=F64, stream=None):
        """eps(g5 D_w(-rho)) psi by the Chebyshev/Clenshaw approximation; returns (out, info dict)."""
        p, loc, keep = _ptr(psi)
        out = self._out_like(psi)
        po, loco, keepo = _ptr(out)
        info = SignInfo()
        _check(lib().lq_overlap_sign_apply(self.h, ctypes.c_double(rho), ctypes.c_double(lambda_min),
                                           ctypes.c_double(lambda_max), ctypes.c_double(delta), ctypes.c_int(prec),
                                           ctypes.c_int(loc), p, po, ctypes.byref(info), _stream(stream)))
        return out, {"order": info.order, "max_deviation": info.max_deviation}

    def hw_eigensolve(self, rho, nev, lambda_cut, lambda_max, tol=1e-9, nkv=0, degree=0, max_restarts=0,
                      like=None, stream=None, check=True):
        """The nev lowest-|lambda| eigenpairs of g5 D_w(-rho); returns (evals, evecs list, info dict).
        Eigenvectors are host arrays, or device tensors if `like` is one."""
        p = EigParams(int(nev), int(nkv), int(degree), float(lambda_cut), float(lambda_max), float(tol),
                      int(max_restarts))
        shape = self.dims[::-1] + (4, 3)
        if like is not None and _is_torch(like) and like.is_cuda:
            import torch
            vecs = [torch.empty(shape, dtype=torch.complex128, device=like.device) for _ in range(max(nev, 1))]
        else:
            vecs = [np.empty(shape, dtype=np.complex128) for _ in range(max(nev, 1))]
        ptrs = [_ptr(v) for v in vecs]
        loc = ptrs[0][1]
        arr = (ctypes.c_void_p * len(vecs))(*[q[0].value for q in ptrs])
        evals = (ctypes.c_double * max(nev, 1))()
        info = EigInfo()
        code = lib().lq_hw_eigensolve(self.h, ctypes.c_double(rho), ctypes.byref(p), ctypes.c_int(loc), evals, arr,
                                      ctypes.byref(info), _stream(stream))
        if check or code not in (LQ_OK, LQ_ENOTCONV):
            _check(code)
        return np.array(evals[:nev]), vecs[:nev], info.as_dict()

    def overlap_sign_apply_deflated(self, rho, lambda_min, lambda_max, delta, evals, evecs, psi, stream=None):
        """eps(g5 D_w(-rho)) psi with the given eigenpairs deflated; returns (out, info dict)."""
        p, loc, keep = _ptr(psi)
        out = self._out_like(psi)
        po, loco, keepo = _ptr(out)
        nev = len(evecs)
        vp = [_ptr(v) for v in evecs]
        if any(q[1] != loc for q in vp):
            raise ValueError("eigenvectors and the field must live on the same side (host or device)")
        arr = (ctypes.c_void_p * max(nev, 1))(*[q[0].value for q in vp])
        ev = (ctypes.c_double * max(nev, 1))(*[float(x) for x in evals])
        info = SignInfo()
        _check(lib().lq_overlap_sign_apply_deflated(self.h, ctypes.c_double(rho), ctypes.c_double(lambda_min),
                                                    ctypes.c_double(lambda_max), ctypes.c_double(delta),
                                                    ctypes.c_int(nev), ev, arr, ctypes.c_int(loc), p, po,
                                                    ctypes.byref(info), _stream(stream)))
        return out, {"order": info.order, "max_deviation": info.max_deviation}

    def solve(self, op, params, rhs, stream=None, check=True, out=None):
        """Solves D x = b for every b in rhs (list). Returns (x list, info list).

        For multi-shift, x has nrhs*nshift entries, x[k*nshift + i]."""
        rhs = list(rhs)
        ptrs, keeps = [], []
        loc = None
        for b in rhs:
            p, l, k = _ptr(b)
            ptrs.append(p)
            keeps.append(k)
            loc = l if loc is None else loc
            if l != loc:
                raise ValueError("right-hand sides must all be host or all device arrays")
        nsol = len(rhs) * (params.nshift if params.solver == MULTISHIFT_CG else 1)
        xs = out if out is not None else [self._out_like(rhs[0]) for _ in range(nsol)]
        xptrs = []
        for x in xs:
            p, l, k = _ptr(x)
            if l != loc:
                raise ValueError("solutions must live where the right-hand sides live")
            xptrs.append(p)
            keeps.append(k)
        bp = (ctypes.c_void_p * len(ptrs))(*[p.value for p in ptrs])
        xp = (ctypes.c_void_p * len(xptrs))(*[p.value for p in xptrs])
        info = (SolveInfo * len(rhs))()
        code = lib().lq_solve(self.h, ctypes.byref(op), ctypes.byref(params), ctypes.c_int(len(rhs)), bp, xp,
                              ctypes.c_int(loc), info, _stream(stream))
        infos = [i.as_dict() for i in info]
        if check and code not in (LQ_OK,):
            _check(code)
        return xs, infos


class Field:
    """A resident device field in the library's internal layout (lq_field)."""

    def __init__(self, lat: Lattice, kind, prec, nrhs=1):
        self.lat = lat
        h = ctypes.c_void_p()
        _check(lib().lq_field_create(lat.h, ctypes.c_int(kind), ctypes.c_int(prec), ctypes.c_int(nrhs),
                                     ctypes.byref(h)))
        self.h = h
        self.kind, self.prec, self.nrhs = kind, prec, nrhs

    def close(self):
        if self.h:
            lib().lq_field_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, k, parity, canonical, stream=None):
        p, loc, keep = _ptr(canonical)
        _check(lib().lq_field_import(self.h, ctypes.c_int(k), ctypes.c_int(parity), ctypes.c_int(loc), p,
                                     _stream(stream)))

    def store(self, k, parity, canonical, stream=None):
        p, loc, keep = _ptr(canonical)
        _check(lib().lq_field_export(self.h, ctypes.c_int(k), ctypes.c_int(parity), ctypes.c_int(loc), p,
                                     _stream(stream)))
        return canonical


def dslash_field(lat, op, parity, fin, fout, dagger=False, stream=None):
    _check(lib().lq_dslash_field(lat.h, ctypes.byref(op), ctypes.c_int(parity), ctypes.c_int(int(dagger)), fin.h,
                                 fout.h, _stream(stream)))


def schur_field(lat, op, fin, fout, ftmp, dagger=False, stream=None):
    _check(lib().lq_schur_field(lat.h, ctypes.byref(op), ctypes.c_int(int(dagger)), fin.h, fout.h, ftmp.h,
                                _stream(stream)))


def profile_enable(on=True):
    _check(lib().lq_profile_enable(ctypes.c_int(int(on))))


def profile_reset():
    _check(lib().lq_profile_reset())


def profile_query(name=""):
    n = ctypes.c_int64()
    t = ctypes.c_double()
    _check(lib().lq_profile_query(name.encode(), ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def launch_count():
    return int(lib().lq_launch_count())


def chebyshev_sign(eps, delta, max_order=65536):
    """Coefficients of eps(x) ~ x P(x^2), P = sum_k c_k T_k(z(x^2)) on [eps^2, 1]; returns (coeffs, max_deviation)."""
    order = ctypes.c_int()
    dev = ctypes.c_double()
    _check(lib().lq_chebyshev_sign(ctypes.c_double(eps), ctypes.c_double(delta), ctypes.c_int(max_order), None,
                                   ctypes.byref(order), ctypes.byref(dev)))
    buf = (ctypes.c_double * order.value)()
    _check(lib().lq_chebyshev_sign(ctypes.c_double(eps), ctypes.c_double(delta), ctypes.c_int(order.value), buf,
                                   ctypes.byref(order), ctypes.byref(dev)))
    return list(buf), dev.value


def barrier_selftest(blocks, expect, rounds=1):
    """lq_barrier_selftest: (status code, failed flag) of the bounded grid-barrier test."""
    failed = ctypes.c_int(-1)
    code = lib().lq_barrier_selftest(ctypes.c_int(blocks), ctypes.c_int(expect), ctypes.c_int(rounds),
                                     ctypes.byref(failed))
    return code, failed.value


def tune_reset():
    """Forgets every autotuned launch configuration."""
    _check(lib().lq_tune_reset())


def tune_force(code):
    """Restricts later tuning to one candidate code (block size, or 1000 + block size
    for the register-capped FP32/FP16 Wilson kernel); 0 lifts the restriction."""
    _check(lib().lq_tune_force(ctypes.c_int(code)))


class Server:
    """Request server with HBM-budget admission and per-slot streams (lq_server)."""

    def __init__(self, hbm_budget_bytes, max_slots):
        h = ctypes.c_void_p()
        _check(lib().lq_server_create(ctypes.c_size_t(int(hbm_budget_bytes)), ctypes.c_int(max_slots),
                                      ctypes.byref(h)))
        self.h = h
        self._pending = {}

    def close(self):
        if self.h:
            lib().lq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, lat: Lattice, op, params, rhs):
        rhs = [np.ascontiguousarray(b, dtype=np.complex128) for b in rhs]
        req = Request(lat.h.value, op, params, len(rhs))
        bp = (ctypes.c_void_p * len(rhs))(*[b.ctypes.data for b in rhs])
        t = ctypes.c_uint64()
        _check(lib().lq_submit(self.h, ctypes.byref(req), bp, ctypes.byref(t)))
        nsol = len(rhs) * (params.nshift if params.solver == MULTISHIFT_CG else 1)
        self._pending[t.value] = (nsol, rhs[0].shape, len(rhs))
        return t.value

    def request_bytes(self, lat: Lattice, op, params, nrhs):
        """Device bytes the server reserves for such a request while it runs."""
        req = Request(lat.h.value, op, params, int(nrhs))
        b = ctypes.c_size_t()
        _check(lib().lq_request_bytes(ctypes.byref(req), ctypes.byref(b)))
        return b.value

    def poll(self, ticket):
        """None while running; then (x list, info list, times dict, status)."""
        if ticket not in self._pending:
            _check(lib().lq_poll(self.h, ctypes.c_uint64(ticket), None, None, None))
        nsol, shape, nrhs = self._pending[ticket]
        xs = [np.empty(shape, dtype=np.complex128) for _ in range(nsol)]
        xp = (ctypes.c_void_p * nsol)(*[x.ctypes.data for x in xs])
        info = (SolveInfo * nrhs)()
        times = RequestTimes()
        code = lib().lq_poll(self.h, ctypes.c_uint64(ticket), xp, info, ctypes.byref(times))
        if code == LQ_EAGAIN:
            return None
        del self._pending[ticket]
        if code == LQ_EINVAL:
            _check(code)
        return xs, [i.as_dict() for i in info], {"submitted": times.submitted, "admitted": times.admitted,
                                                  "finished": times.finished}, code

    def wait(self, ticket, timeout_ms=600000):
        code = lib().lq_wait(self.h, ctypes.c_uint64(ticket), ctypes.c_int(timeout_ms))
        if code == LQ_ETIMEOUT:
            return False
        _check(code)
        return True

    def stats(self):
        q, r, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib().lq_server_stats(self.h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
        return {"queued": q.value, "running": r.value, "reserved_bytes": b.value}
