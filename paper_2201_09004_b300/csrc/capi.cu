// capi.cu -- the extern "C" entry points of include/lq.h. Every entry point
// catches the library's exceptions and turns them into an lq_status plus a
// thread-local message; no exception crosses the boundary.
#include <string.h>

#include <new>
#include <vector>

#include "runtime.h"

using namespace lq;

struct lq_field_s {
    Lattice* lat;
    Field f;
};

#define LQ_TRY try {
#define LQ_CATCH                                          \
    }                                                     \
    catch (const Error& e) {                              \
        set_last_error(e.msg);                            \
        return e.code;                                    \
    }                                                     \
    catch (const std::bad_alloc&) {                       \
        set_last_error("host allocation failed");         \
        return LQ_ENOMEM;                                 \
    }                                                     \
    catch (...) {                                         \
        set_last_error("unexpected internal error");      \
        return LQ_EINVAL;                                 \
    }

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// device staging buffer, released on scope exit: plain, or taken from the
// lattice's workspace cache (kept for the next call)
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    Lattice* lat = nullptr;
    cudaStream_t st = nullptr;
    explicit DevBuf(size_t bytes, Lattice* l = nullptr, cudaStream_t s = nullptr) : n(bytes), lat(l), st(s) {
        if (!bytes) return;
        if (lat) {
            p = ws_get(*lat, bytes, false, st);
            return;
        }
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(LQ_ENOMEM, "staging allocation failed");
        }
    }
    ~DevBuf() {
        if (!p) return;
        if (lat) ws_put(*lat, p, st);
        else cudaFree(p);
    }
};

static void check_lattice(lq_lattice lat) {
    if (!lat) fail(LQ_EINVAL, "null lattice handle");
}

static void check_op(const lq_op_params* op) {
    if (!op) fail(LQ_EINVAL, "null operator parameters");
    if (op->action < LQ_WILSON_TM || op->action > LQ_HISQ) fail(LQ_EINVAL, "unknown action");
    if (op->recon != 0 && op->recon != 8 && op->recon != 12 && op->recon != 18)
        fail(LQ_EINVAL, "recon must be 0, 8, 12 or 18");
    if (op->twist_mode != LQ_TWIST_GAMMA5 && op->twist_mode != LQ_TWIST_SCALAR) fail(LQ_EINVAL, "unknown twist_mode");
}

static void check_prec(int prec) {
    if (!valid_prec(prec)) fail(LQ_EINVAL, "unknown precision");
}

static size_t field_canon_bytes(const Lattice& L, int action) {
    return (size_t)L.V * (action == LQ_HISQ ? 6 : 24) * sizeof(double);
}

extern "C" int lq_create_lattice(const int dims[4], int t_boundary, lq_lattice* out) {
    LQ_TRY
    if (!dims || !out) fail(LQ_EINVAL, "null argument");
    if (t_boundary != 1 && t_boundary != -1) fail(LQ_EINVAL, "t_boundary must be +1 or -1");
    long long v = 1;
    for (int d = 0; d < 4; d++) {
        if (dims[d] < 2 || (dims[d] & 1)) fail(LQ_EINVAL, "every extent must be even and >= 2");
        v *= dims[d];
    }
    if (v > (1ll << 30)) fail(LQ_EINVAL, "lattice volume above 2^30 sites");
    lq_lattice h = new lq_lattice_s();
    Lattice& L = h->lat;
    for (int d = 0; d < 4; d++) L.L[d] = dims[d];
    L.bc_t = t_boundary;
    L.V = (int)v;
    L.vh = (int)(v / 2);
    for (int d = 0; d < 4; d++) L.geo.L[d] = dims[d];
    L.geo.lxh = dims[0] / 2;
    L.geo.vh = L.vh;
    L.geo.bc_t = t_boundary;
    {
        const int ds[3] = {dims[0] / 2, dims[1], dims[2]};
        L.geo.fast = 1;
        for (int k = 0; k < 3; k++) {
            const unsigned long long d = (unsigned long long)ds[k];
            L.geo.fdiv[k] = d == 1 ? 0u : (unsigned)(((1ull << 32) + d - 1) / d);
            if ((unsigned long long)L.vh * d >= (1ull << 32)) L.geo.fast = 0;
        }
    }
    cudaGetDevice(&L.device);
    *out = h;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_destroy_lattice(lq_lattice h) {
    LQ_TRY
    if (!h) return LQ_OK;
    Lattice& L = h->lat;
    cudaDeviceSynchronize();
    ws_release(L);
    if (L.own_stream) cudaStreamDestroy(L.own_stream);
    if (L.copy_stream) cudaStreamDestroy(L.copy_stream);
    free_clover(L);
    for (auto& kv : L.packed) dev_free(&L, kv.second.data, kv.second.bytes);
    for (int k = 0; k < 3; k++) dev_free(&L, L.canon[k], (size_t)L.V * 4 * 18 * sizeof(double));
    delete h;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_lattice_bytes(lq_lattice h, size_t* bytes) {
    LQ_TRY
    check_lattice(h);
    if (bytes) {
        Lattice& L = h->lat;
        std::lock_guard<std::mutex> lk(L.mu);
        size_t ws = 0;
        for (auto& b : L.ws)
            if (!b.host) ws += b.bytes;
        *bytes = L.bytes + ws;
    }
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_lattice_release_workspace(lq_lattice h, size_t* freed) {
    LQ_TRY
    check_lattice(h);
    size_t n = ws_release(h->lat);
    if (freed) *freed = n;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_load_gauge(lq_lattice h, int kind, int loc, const double* links) {
    LQ_TRY
    check_lattice(h);
    if (kind < LQ_THIN || kind > LQ_LONG) fail(LQ_EINVAL, "unknown gauge kind");
    if (!links) fail(LQ_EINVAL, "null links");
    Lattice& L = h->lat;
    std::lock_guard<std::mutex> lk(L.mu);
    const size_t bytes = (size_t)L.V * 4 * 18 * sizeof(double);
    if (!L.canon[kind]) L.canon[kind] = (double*)dev_alloc(&L, bytes);
    LQ_CUDA(cudaMemcpy(L.canon[kind], links, bytes, loc == LQ_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
    gauge_maxabs(L.canon[kind], L.V, &L.maxabs[kind], 0);
    // drop packed copies of this kind: they are rebuilt on demand
    for (auto it = L.packed.begin(); it != L.packed.end();) {
        if (std::get<0>(it->first) == kind) {
            dev_free(&L, it->second.data, it->second.bytes);
            it = L.packed.erase(it);
        } else {
            ++it;
        }
    }
    if (kind == LQ_THIN && L.has_clover) free_clover(L);  // the clover belongs to the old links
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_load_clover(lq_lattice h, int loc, const double* clover, double c_sw) {
    LQ_TRY
    check_lattice(h);
    Lattice& L = h->lat;
    std::lock_guard<std::mutex> lk(L.mu);
    if (!clover) {
        build_clover(L, c_sw, 0);
    } else {
        const size_t bytes = (size_t)L.V * 288 * sizeof(double);
        if (loc == LQ_HOST) {
            DevBuf tmp(bytes);
            LQ_CUDA(cudaMemcpy(tmp.p, clover, bytes, cudaMemcpyHostToDevice));
            load_clover_canonical(L, (const double*)tmp.p, 0);
        } else {
            load_clover_canonical(L, clover, 0);
        }
        L.c_sw = c_sw;
    }
    return LQ_OK;
    LQ_CATCH
}

static OpDesc make_desc(const lq_op_params* op, int prec) {
    OpDesc d;
    d.action = op->action;
    d.m = op->m;
    d.mu = op->action == LQ_HISQ ? 0.0 : op->mu;
    d.c_naik = op->c_naik;
    d.prec = prec;
    d.recon = (prec == LQ_F64 || prec == LQ_F32X2) ? 18 : (op->recon == 0 ? 12 : op->recon);
    d.twist = op->twist_mode;
    return d;
}

// stage canonical in (host or device) to device; returns device pointer
static const double* stage_in(const double* p, size_t bytes, int loc, DevBuf& buf, cudaStream_t st) {
    if (loc == LQ_DEVICE) return p;
    LQ_CUDA(cudaMemcpyAsync(buf.p, p, bytes, cudaMemcpyHostToDevice, st));
    return (const double*)buf.p;
}

extern "C" int lq_dslash_apply(lq_lattice h, const lq_op_params* op, int parity, int dagger, int prec, int loc,
                               const double* in, double* out, void* stream) {
    LQ_TRY
    check_lattice(h);
    check_op(op);
    check_prec(prec);
    if (parity != 0 && parity != 1) fail(LQ_EINVAL, "parity must be 0 or 1");
    if (!in || !out) fail(LQ_EINVAL, "null field");
    Lattice& L = h->lat;
    cudaStream_t st = as_stream(stream);
    const bool hisq = op->action == LQ_HISQ;
    const int kind = hisq ? LQ_STAGGERED_FIELD : LQ_WILSON_FIELD;
    const size_t bytes = field_canon_bytes(L, op->action);
    DevBuf bin(loc == LQ_HOST ? bytes : 0), bout(loc == LQ_HOST ? bytes : 0);
    const double* din = stage_in(in, bytes, loc, bin, st);
    double* dout = loc == LQ_HOST ? (double*)bout.p : out;
    Field fi = field_alloc(kind, prec, 1, L.vh), fo = field_alloc(kind, prec, 1, L.vh);
    try {
        OpDesc d = make_desc(op, prec);
        import_field(L, fi, 0, 1 - parity, din, st);
        if (hisq) hisq_dslash(L, d, parity, dagger, EPI_HOP, 0.0, fi, fo, nullptr, nullptr, st);
        else wilson_dslash(L, d, parity, dagger, EPI_HOP, fi, fo, nullptr, nullptr, st);
        LQ_CUDA(cudaMemsetAsync(dout, 0, bytes, st));
        export_field(L, fo, 0, parity, dout, st);
        if (loc == LQ_HOST) LQ_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        field_free(fi);
        field_free(fo);
        throw;
    }
    field_free(fi);
    field_free(fo);
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_operator_apply(lq_lattice h, const lq_op_params* op, int form, int dagger, int prec, int loc,
                                 const double* in, double* out, void* stream) {
    LQ_TRY
    check_lattice(h);
    check_op(op);
    check_prec(prec);
    if (form != LQ_OP_FULL && form != LQ_OP_SCHUR) fail(LQ_EINVAL, "unknown operator form");
    if (!in || !out) fail(LQ_EINVAL, "null field");
    Lattice& L = h->lat;
    cudaStream_t st = as_stream(stream);
    const bool hisq = op->action == LQ_HISQ;
    const int kind = hisq ? LQ_STAGGERED_FIELD : LQ_WILSON_FIELD;
    const size_t bytes = field_canon_bytes(L, op->action);
    DevBuf bin(loc == LQ_HOST ? bytes : 0), bout(loc == LQ_HOST ? bytes : 0);
    const double* din = stage_in(in, bytes, loc, bin, st);
    double* dout = loc == LQ_HOST ? (double*)bout.p : out;
    std::vector<Field> fs;
    try {
        for (int i = 0; i < 4; i++) fs.push_back(field_alloc(kind, prec, 1, L.vh));
        Field &fe = fs[0], &fo = fs[1], &oe = fs[2], &oo = fs[3];
        OpDesc d = make_desc(op, prec);
        LQ_CUDA(cudaMemsetAsync(dout, 0, bytes, st));
        import_field(L, fe, 0, 0, din, st);
        if (form == LQ_OP_FULL) {
            import_field(L, fo, 0, 1, din, st);
            if (hisq) {
                // out_p = m in_p + s H in_{1-p}; the XPAY epilogue gives m y - D, and the
                // kernel's adjoint flag negates D, so H (dagger 0) needs the flag set
                hisq_dslash(L, d, 0, !dagger, EPI_XPAY, op->m, fo, oe, &fe, nullptr, st);
                hisq_dslash(L, d, 1, !dagger, EPI_XPAY, op->m, fe, oo, &fo, nullptr, st);
            } else {
                wilson_dslash(L, d, 0, dagger, EPI_XPAY, fo, oe, &fe, nullptr, st);
                wilson_dslash(L, d, 1, dagger, EPI_XPAY, fe, oo, &fo, nullptr, st);
            }
            export_field(L, oe, 0, 0, dout, st);
            export_field(L, oo, 0, 1, dout, st);
        } else {
            if (hisq) schur_hisq(L, d, op->m * op->m, fe, oe, fo, nullptr, st);
            else schur_wilson(L, d, dagger, fe, oe, fo, nullptr, st);
            export_field(L, oe, 0, 0, dout, st);
        }
        if (loc == LQ_HOST) LQ_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        for (auto& f : fs) field_free(f);
        throw;
    }
    for (auto& f : fs) field_free(f);
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_solve(lq_lattice h, const lq_op_params* op, const lq_solve_params* sp, int nrhs,
                        const double* const* rhs, double* const* x, int loc, lq_solve_info* info, void* stream) {
    LQ_TRY
    check_lattice(h);
    check_op(op);
    if (!sp || !rhs || !x) fail(LQ_EINVAL, "null argument");
    if (nrhs < 1) fail(LQ_EINVAL, "nrhs must be positive");
    Lattice& L = h->lat;
    cudaStream_t st = as_stream(stream);
    if (st == nullptr || st == cudaStreamLegacy) {
        // run on the lattice's own stream, ordered after the caller's earlier default-stream work
        {
            std::lock_guard<std::mutex> g(L.mu);
            if (!L.own_stream) LQ_CUDA(cudaStreamCreateWithFlags(&L.own_stream, cudaStreamNonBlocking));
        }
        cudaEvent_t fork;
        LQ_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        cudaEventRecord(fork, st);
        cudaStreamWaitEvent(L.own_stream, fork, 0);
        cudaEventDestroy(fork);
        st = L.own_stream;
    }
    const size_t bytes = field_canon_bytes(L, op->action);
    const int nsol = nrhs * (sp->solver == LQ_MULTISHIFT_CG ? std::max(1, sp->nshift) : 1);
    for (int k = 0; k < nrhs; k++)
        if (!rhs[k]) fail(LQ_EINVAL, "null right-hand side");
    for (int k = 0; k < nsol; k++)
        if (!x[k]) fail(LQ_EINVAL, "null solution pointer");
    std::vector<const double*> db(nrhs);
    std::vector<double*> dx(nsol);
    DevBuf stage(loc == LQ_HOST ? bytes * (nrhs + nsol) : 0, &L, st);
    if (loc == LQ_HOST) {
        for (int k = 0; k < nrhs; k++) {
            double* d = (double*)stage.p + (size_t)k * (bytes / sizeof(double));
            LQ_CUDA(cudaMemcpyAsync(d, rhs[k], bytes, cudaMemcpyHostToDevice, st));
            db[k] = d;
        }
        for (int k = 0; k < nsol; k++) dx[k] = (double*)stage.p + (size_t)(nrhs + k) * (bytes / sizeof(double));
    } else {
        for (int k = 0; k < nrhs; k++) db[k] = rhs[k];
        for (int k = 0; k < nsol; k++) dx[k] = x[k];
    }
    // Host solutions: each one is copied back on the lattice's copy stream as soon as
    // the solver has written it, beside the solve's remaining kernels (the final
    // residual check, the next mass). The guard waits for this call's copies (an event
    // after the last of them, so not for copies that other calls queue later) before
    // the staging buffer returns to the pool, on every exit.
    struct CopyBack {
        cudaStream_t cs = nullptr;
        cudaEvent_t ev = nullptr, done = nullptr;
        cudaError_t wait() {
            if (!cs) return cudaSuccess;
            cudaError_t e = cudaEventRecord(done, cs);
            if (e == cudaSuccess) e = cudaEventSynchronize(done);
            cs = nullptr;
            return e;
        }
        ~CopyBack() {
            wait();
            if (ev) cudaEventDestroy(ev);
            if (done) cudaEventDestroy(done);
        }
    } cb;
    SolutionReady ready;
    if (loc == LQ_HOST) {
        {
            std::lock_guard<std::mutex> g(L.mu);
            if (!L.copy_stream) LQ_CUDA(cudaStreamCreateWithFlags(&L.copy_stream, cudaStreamNonBlocking));
        }
        LQ_CUDA(cudaEventCreateWithFlags(&cb.ev, cudaEventDisableTiming));
        LQ_CUDA(cudaEventCreateWithFlags(&cb.done, cudaEventDisableTiming));
        cb.cs = L.copy_stream;
        ready = [&](int k, cudaStream_t s) {
            LQ_CUDA(cudaEventRecord(cb.ev, s));
            LQ_CUDA(cudaStreamWaitEvent(cb.cs, cb.ev, 0));
            LQ_CUDA(cudaMemcpyAsync(x[k], dx[k], bytes, cudaMemcpyDeviceToHost, cb.cs));
        };
    }
    const SolutionReady* rp = loc == LQ_HOST ? &ready : nullptr;
    int ret;
    if (op->action == LQ_HISQ) ret = solve_hisq(L, *op, *sp, nrhs, db.data(), dx.data(), info, st, rp);
    else if (sp->solver == LQ_MULTISHIFT_CG)
        ret = solve_wilson_multishift(L, *op, *sp, nrhs, db.data(), dx.data(), info, st, rp);
    else ret = solve_wilson(L, *op, *sp, nrhs, db.data(), dx.data(), info, st, nullptr, rp);
    LQ_CUDA(cudaStreamSynchronize(st));
    LQ_CUDA(cb.wait());
    return ret;
    LQ_CATCH
}

// ----------------------------------------------------------------- fields
extern "C" int lq_field_create(lq_lattice h, int kind, int prec, int nrhs, lq_field* out) {
    LQ_TRY
    check_lattice(h);
    check_prec(prec);
    if (kind != LQ_WILSON_FIELD && kind != LQ_STAGGERED_FIELD) fail(LQ_EINVAL, "unknown field kind");
    if (nrhs < 1 || nrhs > 64 || !out) fail(LQ_EINVAL, "nrhs must be in [1, 64]");
    lq_field f = new lq_field_s();
    f->lat = &h->lat;
    try {
        f->f = field_alloc(kind, prec, nrhs, h->lat.vh);
    } catch (...) {
        delete f;
        throw;
    }
    *out = f;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_field_destroy(lq_field f) {
    LQ_TRY
    if (!f) return LQ_OK;
    cudaDeviceSynchronize();
    field_free(f->f);
    delete f;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_field_import(lq_field f, int k, int parity, int loc, const double* canonical, void* stream) {
    LQ_TRY
    if (!f || !canonical) fail(LQ_EINVAL, "null argument");
    if (k < 0 || k >= f->f.nrhs || (parity != 0 && parity != 1)) fail(LQ_EINVAL, "rhs index or parity");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = (size_t)f->lat->V * f->f.nreals() * sizeof(double);
    DevBuf b(loc == LQ_HOST ? bytes : 0);
    const double* d = stage_in(canonical, bytes, loc, b, st);
    import_field(*f->lat, f->f, k, parity, d, st);
    if (loc == LQ_HOST) LQ_CUDA(cudaStreamSynchronize(st));
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_field_export(lq_field f, int k, int parity, int loc, double* canonical, void* stream) {
    LQ_TRY
    if (!f || !canonical) fail(LQ_EINVAL, "null argument");
    if (k < 0 || k >= f->f.nrhs || (parity != 0 && parity != 1)) fail(LQ_EINVAL, "rhs index or parity");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = (size_t)f->lat->V * f->f.nreals() * sizeof(double);
    if (loc == LQ_HOST) {
        DevBuf b(bytes);
        LQ_CUDA(cudaMemcpyAsync(b.p, canonical, bytes, cudaMemcpyHostToDevice, st));
        export_field(*f->lat, f->f, k, parity, (double*)b.p, st);
        LQ_CUDA(cudaMemcpyAsync(canonical, b.p, bytes, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    } else {
        export_field(*f->lat, f->f, k, parity, canonical, st);
    }
    return LQ_OK;
    LQ_CATCH
}

static void check_pair(lq_lattice h, lq_field a, lq_field b) {
    if (!a || !b) fail(LQ_EINVAL, "null field");
    if (a->lat != &h->lat || b->lat != &h->lat) fail(LQ_EINVAL, "field belongs to another lattice");
    if (a->f.kind != b->f.kind || a->f.prec != b->f.prec || a->f.nrhs != b->f.nrhs)
        fail(LQ_EINVAL, "fields differ in kind, precision or nrhs");
}

extern "C" int lq_dslash_field(lq_lattice h, const lq_op_params* op, int parity, int dagger, lq_field in,
                               lq_field out, void* stream) {
    LQ_TRY
    check_lattice(h);
    check_op(op);
    check_pair(h, in, out);
    if (parity != 0 && parity != 1) fail(LQ_EINVAL, "parity must be 0 or 1");
    OpDesc d = make_desc(op, in->f.prec);
    if (op->action == LQ_HISQ) {
        if (in->f.kind != LQ_STAGGERED_FIELD) fail(LQ_EINVAL, "HISQ needs staggered fields");
        hisq_dslash(h->lat, d, parity, dagger, EPI_HOP, 0.0, in->f, out->f, nullptr, nullptr, as_stream(stream));
    } else {
        if (in->f.kind != LQ_WILSON_FIELD) fail(LQ_EINVAL, "Wilson actions need Wilson fields");
        wilson_dslash(h->lat, d, parity, dagger, EPI_HOP, in->f, out->f, nullptr, nullptr, as_stream(stream));
    }
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_schur_field(lq_lattice h, const lq_op_params* op, int dagger, lq_field in, lq_field out,
                              lq_field tmp, void* stream) {
    LQ_TRY
    check_lattice(h);
    check_op(op);
    check_pair(h, in, out);
    check_pair(h, in, tmp);
    OpDesc d = make_desc(op, in->f.prec);
    if (op->action == LQ_HISQ) schur_hisq(h->lat, d, op->m * op->m, in->f, out->f, tmp->f, nullptr, as_stream(stream));
    else schur_wilson(h->lat, d, dagger, in->f, out->f, tmp->f, nullptr, as_stream(stream));
    return LQ_OK;
    LQ_CATCH
}

// ---------------------------------------------------------------- overlap
static void check_sign_prec(int prec) {
    if (prec != LQ_F64 && prec != LQ_F32 && prec != LQ_F32X2)
        fail(LQ_EINVAL, "the overlap building blocks run in LQ_F64, LQ_F32X2 or LQ_F32");
}

// full-lattice Wilson spinor fields of 2 "rhs" (even sites, odd sites) from / to canonical
static void import_full(Lattice& L, Field& f, const double* canon, cudaStream_t st) {
    import_field(L, f, 0, 0, canon, st);
    import_field(L, f, 1, 1, canon, st);
}
static void export_full(Lattice& L, const Field& f, double* canon, cudaStream_t st) {
    export_field(L, f, 0, 0, canon, st);
    export_field(L, f, 1, 1, canon, st);
}

extern "C" int lq_gamma5_dw_apply(lq_lattice h, double rho, int prec, int loc, const double* in, double* out,
                                  void* stream) {
    LQ_TRY
    check_lattice(h);
    check_sign_prec(prec);
    if (!in || !out) fail(LQ_EINVAL, "null field");
    Lattice& L = h->lat;
    if (!L.canon[LQ_THIN]) fail(LQ_EINVAL, "thin gauge field not loaded");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = field_canon_bytes(L, LQ_WILSON_TM);
    DevBuf bin(loc == LQ_HOST ? bytes : 0, &L, st), bout(loc == LQ_HOST ? bytes : 0, &L, st);
    const double* din = stage_in(in, bytes, loc, bin, st);
    double* dout = loc == LQ_HOST ? (double*)bout.p : out;
    Field fi = ws_field(L, LQ_WILSON_FIELD, prec, 2, st), fo = ws_field(L, LQ_WILSON_FIELD, prec, 2, st);
    try {
        import_full(L, fi, din, st);
        hw_apply_full(L, rho, fi, fo, st);
        export_full(L, fo, dout, st);
        if (loc == LQ_HOST) LQ_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        ws_put(L, fi.data, st);
        ws_put(L, fo.data, st);
        throw;
    }
    ws_put(L, fi.data, st);
    ws_put(L, fo.data, st);
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_chebyshev_sign(double eps, double delta, int max_order, double* coeffs, int* order,
                                 double* max_deviation) {
    LQ_TRY
    if (max_order < 1) fail(LQ_EINVAL, "max_order must be positive");
    std::vector<double> c;
    double dev = 0.0;
    sign_coefficients(eps, delta, max_order, c, dev);
    if (order) *order = (int)c.size();
    if (max_deviation) *max_deviation = dev;
    if (coeffs)
        for (size_t k = 0; k < c.size(); k++) coeffs[k] = c[k];
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_overlap_sign_apply(lq_lattice h, double rho, double lambda_min, double lambda_max, double delta,
                                     int prec, int loc, const double* in, double* out, lq_sign_info* info,
                                     void* stream) {
    LQ_TRY
    check_lattice(h);
    check_sign_prec(prec);
    if (!in || !out) fail(LQ_EINVAL, "null field");
    if (!(lambda_max > 0.0) || !(lambda_min > 0.0) || !(lambda_min < lambda_max))
        fail(LQ_EINVAL, "need 0 < lambda_min < lambda_max");
    Lattice& L = h->lat;
    if (!L.canon[LQ_THIN]) fail(LQ_EINVAL, "thin gauge field not loaded");
    std::vector<double> c;
    double dev = 0.0;
    sign_coefficients(lambda_min / lambda_max, delta, 1 << 16, c, dev);
    cudaStream_t st = as_stream(stream);
    const size_t bytes = field_canon_bytes(L, LQ_WILSON_TM);
    DevBuf bin(loc == LQ_HOST ? bytes : 0, &L, st), bout(loc == LQ_HOST ? bytes : 0, &L, st);
    const double* din = stage_in(in, bytes, loc, bin, st);
    double* dout = loc == LQ_HOST ? (double*)bout.p : out;
    Field fi = ws_field(L, LQ_WILSON_FIELD, prec, 2, st), fo = ws_field(L, LQ_WILSON_FIELD, prec, 2, st);
    try {
        import_full(L, fi, din, st);
        sign_apply(L, rho, lambda_max, lambda_min / lambda_max, c, fi, fo, st);
        export_full(L, fo, dout, st);
        if (loc == LQ_HOST) LQ_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        ws_put(L, fi.data, st);
        ws_put(L, fo.data, st);
        throw;
    }
    ws_put(L, fi.data, st);
    ws_put(L, fo.data, st);
    if (info) {
        info->order = (int)c.size();
        info->max_deviation = dev;
    }
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_hw_eigensolve(lq_lattice h, double rho, const lq_eig_params* p, int loc, double* evals,
                                double* const* evecs, lq_eig_info* info, void* stream) {
    LQ_TRY
    check_lattice(h);
    if (!p || !evals) fail(LQ_EINVAL, "null argument");
    if (loc != LQ_HOST && loc != LQ_DEVICE) fail(LQ_EINVAL, "loc must be LQ_HOST or LQ_DEVICE");
    Lattice& L = h->lat;
    if (!L.canon[LQ_THIN]) fail(LQ_EINVAL, "thin gauge field not loaded");
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e0, e1;
    LQ_CUDA(cudaEventCreate(&e0));
    LQ_CUDA(cudaEventCreate(&e1));
    LQ_CUDA(cudaEventRecord(e0, st));
    std::vector<double> ev;
    std::vector<Field> vecs;
    lq_eig_info inf{};
    try {
        hw_eigensolve(L, rho, *p, ev, vecs, inf, st);
        LQ_CUDA(cudaEventRecord(e1, st));
        if (evecs) {
            const size_t bytes = field_canon_bytes(L, LQ_WILSON_TM);
            DevBuf bout(loc == LQ_HOST ? bytes : 0, &L, st);
            for (int i = 0; i < p->nev; i++) {
                if (!evecs[i]) continue;
                double* dout = loc == LQ_HOST ? (double*)bout.p : evecs[i];
                export_full(L, vecs[i], dout, st);
                if (loc == LQ_HOST) LQ_CUDA(cudaMemcpyAsync(evecs[i], dout, bytes, cudaMemcpyDeviceToHost, st));
                LQ_CUDA(cudaStreamSynchronize(st));
            }
        }
        LQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        for (auto& f : vecs) ws_put(L, f.data, st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    for (auto& f : vecs) ws_put(L, f.data, st);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    inf.seconds = ms * 1e-3;
    for (int i = 0; i < p->nev; i++) evals[i] = ev[i];
    if (info) *info = inf;
    if (!inf.converged) {
        set_last_error("lq_hw_eigensolve: max_restarts reached before every residual met tol");
        return LQ_ENOTCONV;
    }
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_overlap_sign_apply_deflated(lq_lattice h, double rho, double lambda_min, double lambda_max,
                                              double delta, int nev, const double* evals,
                                              const double* const* evecs, int loc, const double* in, double* out,
                                              lq_sign_info* info, void* stream) {
    LQ_TRY
    check_lattice(h);
    if (!in || !out) fail(LQ_EINVAL, "null field");
    if (nev < 0 || nev > 64 || (nev > 0 && (!evals || !evecs))) fail(LQ_EINVAL, "need nev in [0, 64] eigenpairs");
    if (loc != LQ_HOST && loc != LQ_DEVICE) fail(LQ_EINVAL, "loc must be LQ_HOST or LQ_DEVICE");
    if (!(lambda_max > 0.0) || !(lambda_min > 0.0) || !(lambda_min < lambda_max))
        fail(LQ_EINVAL, "need 0 < lambda_min < lambda_max");
    Lattice& L = h->lat;
    if (!L.canon[LQ_THIN]) fail(LQ_EINVAL, "thin gauge field not loaded");
    for (int i = 0; i < nev; i++)
        if (!evecs[i]) fail(LQ_EINVAL, "null eigenvector");
    std::vector<double> c;
    double dev = 0.0;
    sign_coefficients(lambda_min / lambda_max, delta, 1 << 16, c, dev);
    cudaStream_t st = as_stream(stream);
    const size_t bytes = field_canon_bytes(L, LQ_WILSON_TM);
    DevBuf bin(loc == LQ_HOST ? bytes : 0, &L, st), bout(loc == LQ_HOST ? bytes : 0, &L, st);
    std::vector<Field> held;
    try {
        std::vector<Field> vecs;
        std::vector<double> ev(evals, evals + nev);
        for (int i = 0; i < nev; i++) {
            Field f = ws_field(L, LQ_WILSON_FIELD, LQ_F32X2, 2, st);
            held.push_back(f);
            import_full(L, f, stage_in(evecs[i], bytes, loc, bin, st), st);
            vecs.push_back(f);
        }
        Field fi = ws_field(L, LQ_WILSON_FIELD, LQ_F32X2, 2, st);
        held.push_back(fi);
        Field fo = ws_field(L, LQ_WILSON_FIELD, LQ_F32X2, 2, st);
        held.push_back(fo);
        import_full(L, fi, stage_in(in, bytes, loc, bin, st), st);
        sign_apply_deflated(L, rho, lambda_max, lambda_min / lambda_max, c, ev, vecs, fi, fo, st);
        double* dout = loc == LQ_HOST ? (double*)bout.p : out;
        export_full(L, fo, dout, st);
        if (loc == LQ_HOST) LQ_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        for (auto& f : held) ws_put(L, f.data, st);
        throw;
    }
    for (auto& f : held) ws_put(L, f.data, st);
    if (info) {
        info->order = (int)c.size();
        info->max_deviation = dev;
    }
    return LQ_OK;
    LQ_CATCH
}

