// solver.cu -- even-odd preconditioned Krylov solvers on the device.
//
// Wilson twisted mass (+clover), asymmetric even-odd Schur complement:
//   M = [[A_ee, -H_eo], [-H_oe, A_oo]],  Mhat = A_ee - H_eo A_oo^{-1} H_oe,
//   bhat = b_e + H_eo A_oo^{-1} b_o,  Mhat x_e = bhat,  x_o = A_oo^{-1} (b_o + H_oe x_e).
// The odd rows are then solved exactly, so the full residual of M x = b is
// bhat - Mhat x_e. Mhat is solved by CG on the normal equations (CGNR), in one
// precision or mixed with FP64 reliable updates (the mixed-precision solvers
// the paper's GPU inverters rest on, refs. of Sec. 1).
//
// HISQ: D = m + H with H anti-hermitian and connecting even and odd sites only:
//   (m^2 - H_eo H_oe) x_e = m b_e - H_eo b_o,  x_o = (b_o - H_oe x_e) / m,
// and m^2 - H_eo H_oe = m^2 + H_oe^+ H_oe is hermitian positive definite, so
// plain CG applies; several masses share one Krylov space through multi-shift
// CG (Jegerlehner, the multi-mass algorithm named in Sec. 2.3), and each mass
// is then refined by the mixed-precision CG.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "runtime.h"

namespace lq {

// device scalars, their pinned host copy and the partial-sum buffer of one
// solve, taken from the lattice's workspace cache
struct Scalars {
    Lattice* lat = nullptr;
    cudaStream_t st = nullptr;
    double* dev = nullptr;
    double* host = nullptr;
    df* part = nullptr;
    unsigned* count = nullptr;  // ticket of the reductions finalised in their producing kernel
    int nrhs = 0;
    void init(Lattice& l, int n, cudaStream_t s) {
        lat = &l;
        st = s;
        nrhs = n;
        // hopping kernels write one partial per site block: at least 8 sites per block
        // (BiCGStab reductions write 3 partials per BLAS block)
        size_t per = std::max<size_t>((size_t)(l.vh + 7) / 8, (size_t)3 * RED_BLOCKS);
        dev = (double*)ws_get(l, sizeof(double) * SC_N * n, false, s);
        LQ_CUDA(cudaMemsetAsync(dev, 0, sizeof(double) * SC_N * n, s));
        part = (df*)ws_get(l, sizeof(df) * per * n, false, s);
        host = (double*)ws_get(l, sizeof(double) * SC_N * n, true, s);
        memset(host, 0, sizeof(double) * SC_N * n);  // a reused buffer holds an earlier solve's scalars
        count = (unsigned*)ws_get(l, 16, false, s);
        LQ_CUDA(cudaMemsetAsync(count, 0, 16, s));
    }
    // finalise a reduction into `slot` (or apply `op`) inside the kernel producing its partials
    FinArgs f(int slot, int op) const {
        FinArgs a;
        a.sc = dev;
        a.slot = slot;
        a.op = op;
        a.count = count;
        return a;
    }
    void pull(cudaStream_t st) {
        LQ_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * SC_N * nrhs, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    }
    double& h(int k, int slot) { return host[(size_t)k * SC_N + slot]; }
    void set(int k, int slot, double v, cudaStream_t st) {
        h(k, slot) = v;
        LQ_CUDA(cudaMemcpyAsync(dev + (size_t)k * SC_N + slot, &host[(size_t)k * SC_N + slot], sizeof(double),
                                cudaMemcpyHostToDevice, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    }
    void fin(int nb, int slot, cudaStream_t st) { blas_finalize(part, nb, nrhs, dev, slot, FIN_SET, st); }
    ~Scalars() {
        if (!lat) return;
        ws_put(*lat, dev, st);
        ws_put(*lat, part, st);
        ws_put(*lat, host, st);
        ws_put(*lat, count, st);
    }
};

// fields of one solve, returned together to the lattice's workspace cache
struct Pool {
    std::vector<Field> owned;
    Lattice& lat;
    cudaStream_t st;
    Pool(Lattice& l, cudaStream_t s) : lat(l), st(s) {}
    Field get(int kind, int prec, int n) {
        owned.push_back(ws_field(lat, kind, prec, n, st));
        return owned.back();
    }
    ~Pool() {
        for (auto& f : owned) ws_put(lat, f.data, st);
    }
};

static void check_finite(double v, const char* what) {
    if (!std::isfinite(v)) fail(LQ_ENAN, std::string("non-finite value in ") + what);
}

struct CgResult {
    std::vector<int> iters, updates, applications, status;
    explicit CgResult(int n) : iters(n, 0), updates(n, 0), applications(n, 0), status(n, LQ_ENOTCONV) {}
};

// link compression of the sloppy operator: 8, 12, or 18 (also for 0)
static int sloppy_recon(const lq_solve_params& sp) {
    if (sp.recon_sloppy == 8 || sp.recon_sloppy == 12) return sp.recon_sloppy;
    if (sp.recon_sloppy == 0 || sp.recon_sloppy == 18) return 18;
    fail(LQ_EINVAL, "recon_sloppy must be 8, 12 or 18");
}

// =================================================================== Wilson
static OpDesc wilson_desc(const lq_op_params& op, int prec, int recon) {
    OpDesc d;
    d.action = op.action;
    d.m = op.m;
    d.mu = op.mu;
    d.c_naik = op.c_naik;
    d.prec = prec;
    d.recon = prec == LQ_F64 ? 18 : recon;
    d.twist = op.twist_mode;
    return d;
}

// out = Mhat in (dagger: Mhat^+); tmp holds the odd sites. Returns the blocks of the |out|^2 partials.
int schur_wilson(Lattice& lat, const OpDesc& op, int dagger, const Field& in, Field& out, Field& tmp, df* part,
                 cudaStream_t st, const FinArgs& fin) {
    wilson_dslash(lat, op, 1, dagger, EPI_AINV, in, tmp, nullptr, nullptr, st);
    return wilson_dslash(lat, op, 0, dagger, EPI_XPAY, tmp, out, &in, part, st, fin);
}

// s = b - Mhat x in FP64 accuracy, |s|^2 finalised as fin says (partials in part), and
// s_lo = s in the sloppy precision. With the double-float operator the A y - D kernel
// forms the residual and its FP16 copy in its epilogue; otherwise Mhat x is followed
// by a subtraction and a copy.
static void schur_residual(Lattice& lat, const OpDesc& op64, const Field& x, const Field& b, Field& s, Field& s_lo,
                           Field& q64, Field& t64, df* part, cudaStream_t st, const FinArgs& fin) {
    if (op64.prec == LQ_F32X2) {
        wilson_dslash(lat, op64, 1, 0, EPI_AINV, x, t64, nullptr, nullptr, st);
        wilson_dslash(lat, op64, 0, 0, EPI_XPAY, t64, s, &x, part, st, fin, &b, s_lo.prec == LQ_F16 ? &s_lo : nullptr);
        if (s_lo.prec != LQ_F16) blas_copy(s_lo, s, st);
    } else {
        schur_wilson(lat, op64, 0, x, q64, t64, nullptr, st);
        blas_xmy_norm(s, b, q64, part, st, fin);
        blas_copy(s_lo, s, st);
    }
}

// ------------------------------------------------------------ Krylov driver
// The loop shared by the mixed-precision solvers. The host reads the residual
// norms of iteration i while iteration i+1 runs: each iteration ends with an
// asynchronous copy of the device scalars into one of two pinned slots and an
// event, and the host waits on the previous one, so the GPU queue never drains.
// A reliable update (iterated |r| below delta times its value at the last
// update), convergence or a breakdown flag is therefore acted on one iteration
// late, which costs at most one extra iteration. After the first (autotuning)
// iteration, graph_iters iterations are captured into two CUDA graphs (one per
// slot) and replayed with one launch each.
//   iteration(dst): the device work of one iteration; dst (or null) gets the scalars.
//   update(): reliable update, ends with the true |r|^2 in SC_SS (not yet pulled).
//   after_update(k): optional per-rhs fix-up after the pull (returns false to stop rhs k).
struct KrylovState {
    std::vector<double> rmax;
    std::vector<char> done;
};

template <class Iter, class Update, class After>
static void krylov_loop(Lattice& lat, Scalars& sc, CgResult& res, KrylovState& ks, const std::vector<double>& tol_abs,
                        double delta, int maxiter, int graph_iters, int apps_per_iter, cudaStream_t st,
                        Iter iteration, Update update, After after_update, int per_call = 1) {
    const int n = sc.nrhs;
    auto all_done = [&]() {
        for (int k = 0; k < n; k++)
            if (!ks.done[k]) return false;
        return true;
    };
    double* ring = (double*)ws_get(lat, sizeof(double) * SC_N * n * 2, true, st);
    cudaEvent_t ev[2];
    LQ_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    LQ_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    struct Cleanup {
        Lattice& l; double* r; cudaEvent_t* e; cudaStream_t s;
        ~Cleanup() { ws_put(l, r, s); cudaEventDestroy(e[0]); cudaEventDestroy(e[1]); }
    } cleanup{lat, ring, ev, st};
    auto slot = [&](int i) { return ring + (size_t)(i & 1) * SC_N * n; };
    const int gk = graph_iters < 0 ? 0 : (graph_iters == 0 ? 1 : graph_iters);
    Graph graphs[2];
    struct GraphCleanup {
        Graph* g;
        ~GraphCleanup() { graph_destroy(g[0]); graph_destroy(g[1]); }
    } graph_cleanup{graphs};
    bool use_graphs = gk > 0;
    int it = 0, launch_no = 0, pending = -1;  // launch whose scalars are in flight
    while (!all_done() && it < maxiter) {
        const int gi = launch_no & 1;
        int steps = per_call;  // iterations one call of iteration() runs (a persistent kernel: several)
        if (use_graphs && it > 0 && it + gk <= maxiter) {
            Graph& g = graphs[gi];
            if (!g.exec) {
                bool ok = graph_capture_begin(st);
                if (ok) {
                    try {
                        for (int j = 0; j < gk; j++) iteration(j == gk - 1 ? slot(gi) : nullptr);
                    } catch (...) {
                        ok = false;
                    }
                    ok = graph_capture_end(st, g) && ok;
                }
                if (!ok) use_graphs = false;  // run eagerly from here on
            } else {
                graph_collect(g);  // its previous replay finished before the host check of it
            }
            if (g.exec) {
                graph_launch(g, st);
                steps = gk;
            } else {
                iteration(slot(gi));
            }
        } else {
            iteration(slot(gi));
        }
        LQ_CUDA(cudaEventRecord(ev[gi], st));
        for (int k = 0; k < n; k++)
            if (!ks.done[k]) {
                res.iters[k] += steps;
                res.applications[k] += apps_per_iter * steps;
            }
        const int prev = pending;
        pending = launch_no;
        launch_no++;
        it += steps;
        bool upd = it >= maxiter;
        if (prev >= 0) {
            LQ_CUDA(cudaEventSynchronize(ev[prev & 1]));
            const double* hs = slot(prev);
            for (int k = 0; k < n; k++) {
                if (ks.done[k]) continue;
                if (hs[(size_t)k * SC_N + SC_BREAK] >= 2.0)
                    fail(LQ_ECUDA, "a grid barrier of the persistent CG kernel timed out");
                if (hs[(size_t)k * SC_N + SC_BREAK] != 0.0) upd = true;
                double ss = sqrt(hs[(size_t)k * SC_N + SC_SS]);
                check_finite(ss, "iterated residual");
                if (ss < delta * ks.rmax[k] || ss <= tol_abs[k]) upd = true;
            }
        }
        if (!upd) continue;
        pending = -1;
        update();
        sc.pull(st);
        for (int k = 0; k < n; k++) {
            if (ks.done[k]) continue;
            res.updates[k]++;
            double ss = sqrt(sc.h(k, SC_SS));
            check_finite(ss, "true residual");
            ks.rmax[k] = ss;
            if (ss <= tol_abs[k]) {
                ks.done[k] = 1;
                res.status[k] = LQ_OK;
                sc.set(k, SC_FROZEN, 1.0, st);
            } else if (!after_update(k)) {
                ks.done[k] = 1;
            }
        }
    }
}

// first check of the sources: |r|^2 in SC_SS (pulled)
static KrylovState krylov_start(Scalars& sc, CgResult& res, const std::vector<double>& tol_abs, cudaStream_t st) {
    KrylovState ks;
    ks.rmax.assign(sc.nrhs, 0.0);
    ks.done.assign(sc.nrhs, 0);
    for (int k = 0; k < sc.nrhs; k++) {
        check_finite(sc.h(k, SC_SS), "source");
        ks.rmax[k] = sqrt(sc.h(k, SC_SS));
        if (ks.rmax[k] <= tol_abs[k]) {
            ks.done[k] = 1;
            res.status[k] = LQ_OK;
            sc.set(k, SC_FROZEN, 1.0, st);
        }
    }
    return ks;
}

// CGNR on Mhat for all right-hand sides of bhat at once (FP64, even sites).
// x_hi receives the solution; tol_abs[k] is the target of |bhat - Mhat x|.
// Each reduction is finalised by the last block of the kernel producing it
// (alpha and beta stay on the device). A reliable update folds the sloppy
// solution into x_hi, recomputes s = bhat - Mhat x_hi in FP64 accuracy, keeps
// p and restarts the norm recurrence from the new r = Mhat^+ s.
// f32_below > 0: a reliable update whose previous true residual is below f32_below |bhat|
// (every right-hand side) forms s = s_prev - Mhat dx in correction form with the FP32
// operator, dx = x_lo the sloppy solution since the previous update (exact in FP32).
static CgResult cgnr_mixed(Lattice& lat, const OpDesc& ops, const OpDesc& op64, Field& bhat, Field& x_hi,
                           const std::vector<double>& tol_abs, double delta, int maxiter, int graph_iters,
                           cudaStream_t st, bool guess = false, int persistent = 0, double f32_below = 0.0) {
    const int n = bhat.nrhs;
    const int ps = ops.prec;
    // the sloppy solution x_lo in the sloppy precision (FP16 storage halves the bytes of its
    // update in every iteration; the reliable update folds it into x_hi, which absorbs its
    // rounding: the iteration count and the true residual stay those of FP32 storage);
    // the persistent kernel keeps it in FP32
    const int px = ps == LQ_F16 && persistent > 0 ? LQ_F32 : ps;
    const int WF = LQ_WILSON_FIELD;
    Pool pool(lat, st);
    const int ph = op64.prec;  // FP64, or double-float for the mixed solvers
    Field s_hi = pool.get(WF, ph, n), q64 = pool.get(WF, ph, n), t64 = pool.get(WF, ph, n);
    Field x_lo = pool.get(WF, px, n);
    Field s_lo = pool.get(WF, ps, n), r = pool.get(WF, ps, n), p = pool.get(WF, ps, n);
    Field q = pool.get(WF, ps, n), t = pool.get(WF, ps, n);
    Scalars sc;
    sc.init(lat, n, st);
    CgResult res(n);
    std::vector<double> ones(n, 1.0);

    if (guess) {  // x_hi holds the initial guess: s = bhat - Mhat x_hi in FP64 accuracy
        schur_residual(lat, op64, x_hi, bhat, s_hi, s_lo, q64, t64, sc.part, st, sc.f(SC_SS, FIN_SET));
    } else {
        blas_zero(x_hi, st);
        blas_copy(s_hi, bhat, st);
        blas_norm2(bhat, sc.part, st, sc.f(SC_SS, FIN_SET));
        blas_copy(s_lo, s_hi, st);
    }
    // partial sums of |q|^2 and |r|^2 that the CG vector kernels finalise themselves
    const size_t nper = std::max<size_t>((size_t)(lat.vh + 7) / 8, (size_t)3 * RED_BLOCKS) * n;
    df* part_q = (df*)ws_get(lat, sizeof(df) * nper, false, st);
    df* part_r = (df*)ws_get(lat, sizeof(df) * nper, false, st);
    struct PartCleanup {
        Lattice& l; void* a; void* b; cudaStream_t s;
        ~PartCleanup() { ws_put(l, a, s); ws_put(l, b, s); }
    } part_cleanup{lat, part_q, part_r, st};
    blas_zero(x_lo, st);
    int nr = schur_wilson(lat, ops, 1, s_lo, r, t, part_r, st, sc.f(SC_RR, FIN_SET));
    blas_copy(p, r, st);
    sc.pull(st);
    KrylovState ks = krylov_start(sc, res, tol_abs, st);
    const std::vector<double> r_start = ks.rmax;  // |bhat - Mhat x_0| per right-hand side
    // the correction-form updates: the FP32 operator and its fields
    OpDesc op32 = ops;
    op32.prec = LQ_F32;
    const bool corr_ok = f32_below > 0 && (ps == LQ_F16 || ps == LQ_F32);
    Field x32, q32, t32;
    if (corr_ok) {
        x32 = pool.get(WF, LQ_F32, n);
        q32 = pool.get(WF, LQ_F32, n);
        t32 = pool.get(WF, LQ_F32, n);
    }
    // persistent: that many iterations per launch of one cooperative kernel (persistent.cu)
    const bool pers = persistent > 0 && persistent_cg_supported(lat, ops, n);
    unsigned* bar = nullptr;
    df* ppart = nullptr;
    if (pers) {
        bar = (unsigned*)ws_get(lat, 16, false, st);
        LQ_CUDA(cudaMemsetAsync(bar, 0, 16, st));
        ppart = (df*)ws_get(lat, sizeof(df) * 2 * persistent_cg_blocks(lat), false, st);
    }
    struct PersistCleanup {
        Lattice& l; void* a; void* b; cudaStream_t s;
        ~PersistCleanup() { if (a) ws_put(l, a, s); if (b) ws_put(l, b, s); }
    } pcleanup{lat, bar, ppart, st};
    auto iteration = [&](double* dst) {
        if (pers) {
            const double th = std::max(delta * ks.rmax[0], tol_abs[0]);
            persistent_cg_run(lat, ops, x_lo, p, s_lo, q, r, t, sc.dev, ppart, bar, persistent, th * th, st);
        } else {
            // the reductions of the two operator applications are finalised by one small
            // kernel each (a finalising last block would make every block of the operator
            // wait for a memory fence and an atomic at its end)
            const int nq = schur_wilson(lat, ops, 0, p, q, t, part_q, st);
            blas_finalize(part_q, nq, n, sc.dev, 0, FIN_ALPHA, st);
            blas_cg_s(s_lo, q, sc.dev, sc.part, st, sc.f(SC_SS, FIN_SET));
            nr = schur_wilson(lat, ops, 1, s_lo, r, t, part_r, st);
            blas_finalize(part_r, nr, n, sc.dev, 0, FIN_BETA, st);
            blas_cg_xp(x_lo, p, r, sc.dev, st);  // x += alpha p with the p of this step, then p
        }
        if (dst) LQ_CUDA(cudaMemcpyAsync(dst, sc.dev, sizeof(double) * SC_N * n, cudaMemcpyDeviceToHost, st));
    };
    auto update = [&]() {
        bool corr = corr_ok;
        for (int k = 0; k < n && corr; k++)
            if (!ks.done[k] && !(ks.rmax[k] <= f32_below * r_start[k])) corr = false;
        if (corr) {  // s = s_prev - Mhat_32 x_lo, then x_hi += x_lo
            blas_copy(x32, x_lo, st);
            blas_axpy_h_zero(x_hi, ones.data(), x_lo, st);
            schur_wilson(lat, op32, 0, x32, q32, t32, nullptr, st);
            blas_copy(q64, q32, st);
            blas_xmy_norm(s_hi, s_hi, q64, sc.part, st, sc.f(SC_SS, FIN_SET));
            blas_copy(s_lo, s_hi, st);
        } else {
            blas_axpy_h_zero(x_hi, ones.data(), x_lo, st);
            schur_residual(lat, op64, x_hi, bhat, s_hi, s_lo, q64, t64, sc.part, st, sc.f(SC_SS, FIN_SET));
        }
        nr = schur_wilson(lat, ops, 1, s_lo, r, t, part_r, st, sc.f(SC_RR, FIN_SET));
        for (int k = 0; k < n; k++)
            if (!ks.done[k]) res.applications[k] += 2;
    };
    krylov_loop(lat, sc, res, ks, tol_abs, delta, maxiter, pers ? -1 : graph_iters, 2, st, iteration, update,
                [](int) { return true; }, pers ? persistent : 1);
    if (pers) {  // the loop counted whole launches; the kernel counted the iterations it did
        sc.pull(st);
        res.iters[0] = (int)sc.h(0, SC_ITERS);
        res.applications[0] = 2 * res.iters[0] + 2 * res.updates[0];
    }
    return res;
}

// Mixed-precision BiCGStab (van der Vorst) on Mhat for all right-hand sides of
// bhat, with complex device scalars finalised in the producing kernels. A
// reliable update folds x_lo into x_hi, recomputes r = bhat - Mhat x_hi in FP64
// accuracy and rho = (r0, r), and keeps p and the shadow residual r0; a
// vanishing denominator restarts that rhs from its true residual (r0 = p = r).
static CgResult bicgstab_mixed(Lattice& lat, const OpDesc& ops, const OpDesc& op64, Field& bhat, Field& x_hi,
                               const std::vector<double>& tol_abs, double delta, int maxiter, int graph_iters,
                               cudaStream_t st) {
    const int n = bhat.nrhs;
    const int ps = ops.prec;
    const int px = ps == LQ_F16 ? LQ_F32 : ps;
    const int WF = LQ_WILSON_FIELD;
    Pool pool(lat, st);
    const int ph = op64.prec;
    Field r_hi = pool.get(WF, ph, n), q64 = pool.get(WF, ph, n), t64 = pool.get(WF, ph, n);
    Field x_lo = pool.get(WF, px, n);
    Field r = pool.get(WF, ps, n), r0 = pool.get(WF, ps, n), p = pool.get(WF, ps, n);
    Field v = pool.get(WF, ps, n), t = pool.get(WF, ps, n), tmp = pool.get(WF, ps, n);
    Scalars sc;
    sc.init(lat, n, st);
    CgResult res(n);
    std::vector<double> ones(n, 1.0);
    std::vector<int> restarts(n, 0);

    blas_zero(x_hi, st);
    blas_zero(x_lo, st);
    blas_norm2(bhat, sc.part, st, sc.f(SC_SS, FIN_SET));
    blas_copy(r, bhat, st);
    blas_copy(r0, r, st);
    blas_copy(p, r, st);
    blas_bicg_rho(r, r0, sc.part, st, sc.f(0, FIN_BICG_RHO));  // rho = (r0, r)
    sc.pull(st);
    KrylovState ks = krylov_start(sc, res, tol_abs, st);
    auto iteration = [&](double* dst) {
        schur_wilson(lat, ops, 0, p, v, tmp, nullptr, st);                     // v = Mhat p
        blas_bicg_cdot(r0, v, sc.part, st, sc.f(0, FIN_BICG_ALPHA));            // alpha = rho / (r0, v)
        blas_bicg_s(r, v, sc.dev, st);                                         // s = r - alpha v
        schur_wilson(lat, ops, 0, r, t, tmp, nullptr, st);                     // t = Mhat s
        blas_bicg_tdot(t, r, sc.part, st, sc.f(0, FIN_BICG_OMEGA));            // omega = (t, s) / |t|^2
        blas_bicg_xr(x_lo, p, r, t, r0, sc.dev, sc.part, st, sc.f(0, FIN_BICG_BETA));  // x, r, rho', beta
        blas_bicg_p(p, r, v, sc.dev, st);                                      // p = r + beta (p - omega v)
        if (dst) LQ_CUDA(cudaMemcpyAsync(dst, sc.dev, sizeof(double) * SC_N * n, cudaMemcpyDeviceToHost, st));
    };
    auto update = [&]() {
        blas_axpy_h_zero(x_hi, ones.data(), x_lo, st);
        schur_residual(lat, op64, x_hi, bhat, r_hi, r, q64, t64, sc.part, st, sc.f(SC_SS, FIN_SET));
        blas_bicg_rho(r, r0, sc.part, st, sc.f(0, FIN_BICG_RHO));
        for (int k = 0; k < n; k++)
            if (!ks.done[k]) res.applications[k] += 2;
    };
    auto after_update = [&](int k) {
        if (sc.h(k, SC_BREAK) == 0.0) return true;
        // a vanishing denominator: restart this right-hand side from its true residual
        if (++restarts[k] > 8) {
            res.status[k] = LQ_EBREAKDOWN;
            return false;
        }
        Field r0k = r0.sub(k, 1), pk = p.sub(k, 1), rk = r.sub(k, 1);
        blas_copy(r0k, rk, st);
        blas_copy(pk, rk, st);
        sc.set(k, SC_BREAK, 0.0, st);
        sc.set(k, SC_FROZEN, 0.0, st);
        FinArgs fk = sc.f(0, FIN_BICG_RHO);
        fk.sc += (size_t)k * SC_N;  // the sub-field's rhs 0 is rhs k
        blas_bicg_rho(rk, r0k, sc.part, st, fk);
        return true;
    };
    krylov_loop(lat, sc, res, ks, tol_abs, delta, maxiter, graph_iters, 2, st, iteration, update, after_update);
    return res;
}

// Restarted GCR (generalised conjugate residual) directly on Mhat for all
// right-hand sides of bhat, in the sloppy precision, inside a defect correction
// in FP64 accuracy. Step j takes the current residual as the new direction p_j,
// forms q_j = Mhat p_j, makes q_j orthogonal to the earlier q_i by classical
// Gram-Schmidt (the same combination applied to p_j keeps q_j = Mhat p_j), and
// moves x along p_j and r along q_j by alpha = <q_j, r>/|q_j|^2, which makes |r|
// minimal over the kept directions. After kmax directions, or once |r| is below
// delta times its value at the restart (or below the target), x_lo is folded into
// x_hi, r = bhat - Mhat x_hi is recomputed in FP64 accuracy and the directions are
// dropped. The scalars of every step are summed on the host from per-block
// double-float partials (fixed order).
static CgResult gcr_mixed(Lattice& lat, const OpDesc& ops, const OpDesc& op64, Field& bhat, Field& x_hi,
                          const std::vector<double>& tol_abs, double delta, int maxiter, int kmax, cudaStream_t st) {
    const int n = bhat.nrhs;
    const int ps = ops.prec;
    const int px = ps == LQ_F16 ? LQ_F32 : ps;
    const int WF = LQ_WILSON_FIELD;
    const int RB = RED_BLOCKS;
    Pool pool(lat, st);
    const int ph = op64.prec;
    Field r_hi = pool.get(WF, ph, n), q64 = pool.get(WF, ph, n), t64 = pool.get(WF, ph, n);
    Field x_lo = pool.get(WF, px, n);
    Field r = pool.get(WF, ps, n), tmp = pool.get(WF, ps, n);
    std::vector<Field> P, Q;
    for (int i = 0; i < kmax; i++) {
        P.push_back(pool.get(WF, ps, n));
        Q.push_back(pool.get(WF, ps, n));
    }
    // device lists of field views: q_0..q_{kmax-1}, p_0..p_{kmax-1}, and (q_j, r) per j
    std::vector<FieldV> lists;
    for (int i = 0; i < kmax; i++) lists.push_back(Q[i].view());
    for (int i = 0; i < kmax; i++) lists.push_back(P[i].view());
    for (int i = 0; i < kmax; i++) {
        lists.push_back(Q[i].view());
        lists.push_back(r.view());
    }
    const size_t part_n = (size_t)n * std::max(kmax, 2) * 2 * RB;
    struct Buffers {
        Lattice& l; cudaStream_t s; std::vector<void*> ptrs;
        void* get(size_t bytes, bool pinned) {
            ptrs.push_back(ws_get(l, bytes, pinned, s));
            return ptrs.back();
        }
        ~Buffers() { for (void* p : ptrs) ws_put(l, p, s); }
    } buf{lat, st, {}};
    FieldV* lists_dev = (FieldV*)buf.get(sizeof(FieldV) * lists.size(), false);
    df* part = (df*)buf.get(sizeof(df) * part_n, false);
    df* hpart = (df*)buf.get(sizeof(df) * part_n, true);
    double* coef_dev = (double*)buf.get(sizeof(double) * 2 * n * kmax, false);
    double* alpha_dev = (double*)buf.get(sizeof(double) * 2 * n, false);
    std::vector<double> coef_h((size_t)2 * n * kmax), alpha_h((size_t)2 * n);
    // pageable sources: each copy is staged before the call returns
    LQ_CUDA(cudaMemcpyAsync(lists_dev, lists.data(), sizeof(FieldV) * lists.size(), cudaMemcpyHostToDevice, st));
    const FieldV* qlist = lists_dev;
    const FieldV* plist = lists_dev + kmax;
    auto pull = [&](size_t count) {
        LQ_CUDA(cudaMemcpyAsync(hpart, part, sizeof(df) * count, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
    };
    auto total = [&](size_t row) {  // sum of the RB partials of one row, fixed order
        double s = 0.0;
        for (int b = 0; b < RB; b++) s += (double)hpart[row * RB + b].hi + (double)hpart[row * RB + b].lo;
        return s;
    };

    CgResult res(n);
    std::vector<char> done(n, 0);
    std::vector<double> rref(n), nq((size_t)n * kmax, 0.0);
    std::vector<double> ones(n, 1.0);
    std::vector<int> stuck(n, 0);
    blas_zero(x_hi, st);
    blas_zero(x_lo, st);
    blas_copy(r_hi, bhat, st);
    blas_norm2(r_hi, part, st);
    blas_copy(r, r_hi, st);
    pull((size_t)n * RB);
    for (int k = 0; k < n; k++) {
        rref[k] = sqrt(total(k));
        check_finite(rref[k], "source");
        if (rref[k] <= tol_abs[k]) {
            done[k] = 1;
            res.status[k] = LQ_OK;
        }
    }
    auto all_done = [&]() {
        for (int k = 0; k < n; k++)
            if (!done[k]) return false;
        return true;
    };
    int it = 0;
    while (!all_done() && it < maxiter) {
        std::vector<char> broke(n, 0);
        for (int j = 0;; j++) {
            blas_copy(P[j], r, st);
            schur_wilson(lat, ops, 0, P[j], Q[j], tmp, nullptr, st);
            if (j > 0) {  // c_i = <q_i, q_j> / |q_i|^2, then q_j -= sum c_i q_i (and p_j alike)
                blas_cdot_multi(qlist, j, Q[j], part, st);
                pull((size_t)n * j * 2 * RB);
                for (int k = 0; k < n; k++)
                    for (int i = 0; i < j; i++) {
                        const size_t row = ((size_t)k * j + i) * 2;
                        const double d = nq[(size_t)k * kmax + i];
                        const bool use = !done[k] && d > 0.0;
                        coef_h[((size_t)k * kmax + i) * 2] = use ? total(row) / d : 0.0;
                        coef_h[((size_t)k * kmax + i) * 2 + 1] = use ? total(row + 1) / d : 0.0;
                    }
                LQ_CUDA(cudaMemcpyAsync(coef_dev, coef_h.data(), sizeof(double) * coef_h.size(), cudaMemcpyHostToDevice,
                                        st));
                blas_gcr_orth(qlist, plist, j, coef_dev, kmax, Q[j], st);
            }
            // |q_j|^2 and <r, q_j>: alpha = <q_j, r> / |q_j|^2 = conj(<r, q_j>) / |q_j|^2
            blas_cdot_multi(lists_dev + 2 * kmax + 2 * j, 2, Q[j], part, st);
            pull((size_t)n * 4 * RB);
            bool restart = false;
            for (int k = 0; k < n; k++) {
                const double qq = total((size_t)k * 4), rq_re = total((size_t)k * 4 + 2),
                             rq_im = total((size_t)k * 4 + 3);
                nq[(size_t)k * kmax + j] = qq;
                const bool ok = !done[k] && qq > 0.0 && std::isfinite(qq);
                if (!done[k] && !ok) {
                    check_finite(qq, "GCR direction");
                    broke[k] = 1;
                    restart = true;
                }
                alpha_h[2 * k] = ok ? rq_re / qq : 0.0;
                alpha_h[2 * k + 1] = ok ? -rq_im / qq : 0.0;
            }
            LQ_CUDA(cudaMemcpyAsync(alpha_dev, alpha_h.data(), sizeof(double) * alpha_h.size(), cudaMemcpyHostToDevice,
                                    st));
            blas_gcr_xr(x_lo, P[j], r, Q[j], alpha_dev, part, st);
            pull((size_t)n * RB);
            it++;
            for (int k = 0; k < n; k++) {
                if (done[k]) continue;
                res.iters[k]++;
                res.applications[k]++;
                const double rn = sqrt(total(k));
                check_finite(rn, "iterated residual");
                if (rn <= tol_abs[k] || rn < delta * rref[k]) restart = true;
            }
            if (restart || j + 1 == kmax || it >= maxiter) break;
        }
        // defect correction: x_hi += x_lo, r = bhat - Mhat x_hi in FP64 accuracy
        blas_axpy_h_zero(x_hi, ones.data(), x_lo, st);
        schur_wilson(lat, op64, 0, x_hi, q64, t64, nullptr, st);
        blas_xmy_norm(r_hi, bhat, q64, part, st);
        blas_copy(r, r_hi, st);
        pull((size_t)n * RB);
        for (int k = 0; k < n; k++) {
            if (done[k]) continue;
            res.updates[k]++;
            res.applications[k]++;
            const double rn = sqrt(total(k));
            check_finite(rn, "true residual");
            // a breakdown that recurs with no progress ends this right-hand side
            stuck[k] = (broke[k] && !(rn < 0.999 * rref[k])) ? stuck[k] + 1 : 0;
            rref[k] = rn;
            if (rn <= tol_abs[k]) {
                done[k] = 1;
                res.status[k] = LQ_OK;
            } else if (stuck[k] > 4) {
                done[k] = 1;
                res.status[k] = LQ_EBREAKDOWN;
            }
        }
    }
    return res;
}

int solve_wilson(Lattice& lat, const lq_op_params& opp, const lq_solve_params& sp, int nrhs, const double* const* b,
                 double* const* x, lq_solve_info* info, cudaStream_t st, const double* const* x0,
                 const SolutionReady* ready) {
    if (opp.action == LQ_WILSON_TM_CLOVER && !lat.has_clover) fail(LQ_EINVAL, "clover action without clover term");
    if (!lat.canon[LQ_THIN]) fail(LQ_EINVAL, "thin gauge field not loaded");
    if (nrhs < 1 || nrhs > 64) fail(LQ_EINVAL, "nrhs must be in [1, 64]");
    int ps = sp.prec_sloppy;
    if (ps < LQ_F64 || ps > LQ_F16) fail(LQ_EINVAL, "prec_sloppy");
    if (sp.solver != LQ_CGNR && sp.solver != LQ_MIXED_CGNR && sp.solver != LQ_BICGSTAB && sp.solver != LQ_GCR)
        fail(LQ_EINVAL, "solver kind for a Wilson action");
    if (sp.restart < 0 || sp.restart > GCR_MAX) fail(LQ_EINVAL, "restart must be in [0, 16]");
    if (!(sp.tol > 0)) fail(LQ_EINVAL, "tol must be positive");
    const int recon = sloppy_recon(sp);
    // the FP64-accuracy steps: native FP64 for the plain FP64 solver, double-float
    // (FP32 pipes) when the iterations run in FP32 / FP16
    const int ph = ps == LQ_F64 ? LQ_F64 : LQ_F32X2;
    const OpDesc op64 = wilson_desc(opp, ph, 18);
    const OpDesc ops = wilson_desc(opp, ps, recon);
    double delta = sp.solver != LQ_CGNR ? (sp.delta > 0 ? sp.delta : 0.1) : 0.0;
    if (ps == LQ_F64) delta = 0.0;
    const int maxiter = sp.maxiter > 0 ? sp.maxiter : 100000;

    // the clover inverse of this (m, mu) stays resident for the whole solve
    struct Pin {
        Lattice& l; double m, mu0, mu1; bool on;
        Pin(Lattice& l_, double m_, double mu0_, double mu1_, bool on_) : l(l_), m(m_), mu0(mu0_), mu1(mu1_), on(on_) {
            if (on) pin_ainv(l, m, mu0, mu1, true);
        }
        ~Pin() { if (on) pin_ainv(l, m, mu0, mu1, false); }
    } pin(lat, opp.m, ops.mu, mu_block1(ops), opp.action == LQ_WILSON_TM_CLOVER);
    cudaEvent_t e0, e1;
    LQ_CUDA(cudaEventCreate(&e0));
    LQ_CUDA(cudaEventCreate(&e1));
    LQ_CUDA(cudaEventRecord(e0, st));
    Pool pool(lat, st);
    Field be = pool.get(LQ_WILSON_FIELD, ph, nrhs), bo = pool.get(LQ_WILSON_FIELD, ph, nrhs);
    Field bhat = pool.get(LQ_WILSON_FIELD, ph, nrhs), xe = pool.get(LQ_WILSON_FIELD, ph, nrhs);
    Field xo = pool.get(LQ_WILSON_FIELD, ph, nrhs), te = pool.get(LQ_WILSON_FIELD, ph, nrhs);
    Field to = pool.get(LQ_WILSON_FIELD, ph, nrhs);
    Scalars sc;
    sc.init(lat, nrhs, st);
    std::vector<double> ones(nrhs, 1.0);
    int ret = LQ_OK;
    try {
        for (int k = 0; k < nrhs; k++) {
            import_field(lat, be, k, 0, b[k], st);
            import_field(lat, bo, k, 1, b[k], st);
        }
        blas_norm2(be, sc.part, st);
        sc.fin(RED_BLOCKS, SC_B2, st);
        blas_norm2(bo, sc.part, st);
        sc.fin(RED_BLOCKS, SC_SS, st);
        sc.pull(st);
        std::vector<double> bn(nrhs), tol_abs(nrhs);
        for (int k = 0; k < nrhs; k++) {
            double b2 = sc.h(k, SC_B2) + sc.h(k, SC_SS);
            check_finite(b2, "source");
            bn[k] = sqrt(b2);
            tol_abs[k] = 0.5 * sp.tol * bn[k];
        }
        // bhat = b_e + H_eo A_oo^{-1} b_o
        wilson_ainv_site(lat, op64, 1, 0, bo, to, st);
        wilson_dslash(lat, op64, 0, 0, EPI_HOP, to, te, nullptr, nullptr, st);
        blas_copy(bhat, be, st);
        blas_axpy_h(bhat, ones.data(), te, st);

        if (x0)
            for (int k = 0; k < nrhs; k++) import_field(lat, xe, k, 0, x0[k], st);
        CgResult cr = sp.solver == LQ_BICGSTAB
                          ? bicgstab_mixed(lat, ops, op64, bhat, xe, tol_abs, delta, maxiter, sp.graph_iters, st)
                      : sp.solver == LQ_GCR
                          ? gcr_mixed(lat, ops, op64, bhat, xe, tol_abs, delta, maxiter,
                                      sp.restart > 0 ? sp.restart : GCR_DEFAULT, st)
                          : cgnr_mixed(lat, ops, op64, bhat, xe, tol_abs, delta, maxiter, sp.graph_iters, st,
                                       x0 != nullptr, sp.solver == LQ_MIXED_CGNR ? sp.persistent : 0,
                                       sp.solver == LQ_MIXED_CGNR ? sp.update_f32_below : 0.0);

        // x_o = A_oo^{-1} (b_o + H_oe x_e)
        wilson_dslash(lat, op64, 1, 0, EPI_HOP, xe, to, nullptr, nullptr, st);
        blas_axpy_h(to, ones.data(), bo, st);
        wilson_ainv_site(lat, op64, 1, 0, to, xo, st);
        for (int k = 0; k < nrhs; k++) {
            export_field(lat, xe, k, 0, x[k], st);
            export_field(lat, xo, k, 1, x[k], st);
            if (ready) (*ready)(k, st);
        }
        // FP64 true residual of the full system: r_p = b_p - (A_pp x_p - H_{p,1-p} x_{1-p})
        // (formed in the double-float kernel's epilogue, or by a subtraction after it)
        if (op64.prec == LQ_F32X2) {
            wilson_dslash(lat, op64, 0, 0, EPI_XPAY, xo, te, &xe, sc.part, st, sc.f(SC_RR, FIN_SET), &be);
            wilson_dslash(lat, op64, 1, 0, EPI_XPAY, xe, to, &xo, sc.part, st, sc.f(SC_QQ, FIN_SET), &bo);
        } else {
            wilson_dslash(lat, op64, 0, 0, EPI_XPAY, xo, te, &xe, nullptr, st);
            blas_xmy_norm(te, be, te, sc.part, st);
            sc.fin(RED_BLOCKS, SC_RR, st);
            wilson_dslash(lat, op64, 1, 0, EPI_XPAY, xe, to, &xo, nullptr, st);
            blas_xmy_norm(to, bo, to, sc.part, st);
            sc.fin(RED_BLOCKS, SC_QQ, st);
        }
        LQ_CUDA(cudaEventRecord(e1, st));
        sc.pull(st);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        for (int k = 0; k < nrhs; k++) {
            double rr = sqrt(sc.h(k, SC_RR) + sc.h(k, SC_QQ)) / bn[k];
            int stt = cr.status[k];
            if (stt == LQ_OK && !(rr <= sp.tol)) stt = LQ_ENOTCONV;
            if (!std::isfinite(rr)) stt = LQ_ENAN;
            if (stt != LQ_OK && ret == LQ_OK) ret = stt;
            if (info) {
                info[k].status = stt;
                info[k].iters = cr.iters[k];
                info[k].reliable_updates = cr.updates[k];
                info[k].operator_applications = cr.applications[k];
                info[k].true_rel_residual = rr;
                info[k].seconds = ms * 1e-3;
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ret != LQ_OK) set_last_error("solve: not every right-hand side reached the tolerance");
    return ret;
}

// Twisted-mass multi-mass solve (no clover). M(mu) = M0 + i mu g5 and M0^+ = g5 M0 g5
// make the cross terms of the normal operator cancel: M(mu)^+ M(mu) = A + mu^2 with
// A = M0^+ M0. So
//   x(mu_i) = (A + mu_i^2)^{-1} M(mu_i)^+ b = y1_i - i mu_i y2_i,
//   y1_i = (A + mu_i^2)^{-1} M0^+ b,   y2_i = (A + mu_i^2)^{-1} g5 b,
// two right-hand sides per source for one multi-shift CG (the multi-mass solver of
// Sec. 2.3) on the full lattice: the even-odd Schur complement is not a shift in mu.
// The multi-shift stage runs in the sloppy precision; each x(mu_i) then starts the
// mixed-precision even-odd CGNR of its own system, which brings it to the tolerance.
int solve_wilson_multishift(Lattice& lat, const lq_op_params& opp, const lq_solve_params& sp, int nrhs,
                            const double* const* b, double* const* x, lq_solve_info* info, cudaStream_t st,
                            const SolutionReady* ready) {
    if (opp.action != LQ_WILSON_TM) fail(LQ_EINVAL, "Wilson multi-shift: twisted mass without clover only");
    if (opp.twist_mode != LQ_TWIST_GAMMA5)
        fail(LQ_EINVAL, "Wilson multi-shift: M^+ M = M0^+ M0 + mu^2 holds for the i mu g5 twist only");
    if (!lat.canon[LQ_THIN]) fail(LQ_EINVAL, "thin gauge field not loaded");
    if (nrhs < 1 || nrhs > 16) fail(LQ_EINVAL, "nrhs must be in [1, 16] for the Wilson multi-shift solve");
    const int ns = sp.nshift;
    if (ns < 1 || ns > 16 || !sp.masses) fail(LQ_EINVAL, "multi-shift solve needs 1..16 twisted masses");
    std::vector<double> mus(sp.masses, sp.masses + ns);
    for (int i = 0; i < ns; i++) {
        if (!std::isfinite(mus[i]) || mus[i] < 0.0) fail(LQ_EINVAL, "twisted masses must be finite and >= 0");
        if (i > 0 && mus[i] <= mus[i - 1]) fail(LQ_EINVAL, "twisted masses must be ascending");
    }
    const int ps = sp.prec_sloppy;
    if (ps < LQ_F64 || ps > LQ_F16) fail(LQ_EINVAL, "prec_sloppy");
    if (!(sp.tol > 0)) fail(LQ_EINVAL, "tol must be positive");
    const int maxiter = sp.maxiter > 0 ? sp.maxiter : 100000;
    lq_op_params op0 = opp;
    op0.mu = 0.0;
    const OpDesc d = wilson_desc(op0, ps, sloppy_recon(sp));
    const int WF = LQ_WILSON_FIELD, nsys = 2 * nrhs, nf = 2 * nsys;
    std::vector<double> sigma(ns);
    for (int i = 0; i < ns; i++) sigma[i] = mus[i] * mus[i];

    int ms_iters = 0;
    {
        Pool pool(lat, st);
        // full-lattice vectors: rhs h * nsys + j is half h (0 even, 1 odd sites) of system j;
        // systems j < nrhs are M0^+ b_j, systems nrhs + j are g5 b_j
        Field B = pool.get(WF, ps, 2 * nrhs);
        for (int k = 0; k < nrhs; k++) {
            import_field(lat, B, k, 0, b[k], st);
            import_field(lat, B, nrhs + k, 1, b[k], st);
        }
        Field R = pool.get(WF, ps, nf), Q = pool.get(WF, ps, nf), T = pool.get(WF, ps, nf);
        for (int h = 0; h < 2; h++) {
            Field bo = B.sub((1 - h) * nrhs, nrhs), bh = B.sub(h * nrhs, nrhs), rh = R.sub(h * nsys, nrhs);
            wilson_dslash(lat, d, h, 1, EPI_XPAY, bo, rh, &bh, nullptr, st);  // (M0^+ b)_h
            Field g = R.sub(h * nsys + nrhs, nrhs);
            blas_gamma5(g, bh, st);
        }
        // x <- M0 in (dag 0) or M0^+ in (dag 1) on all systems
        auto m0 = [&](int dag, const Field& in, Field& out) {
            for (int h = 0; h < 2; h++) {
                const Field same = in.sub(h * nsys, nsys), other = in.sub((1 - h) * nsys, nsys);
                Field o = out.sub(h * nsys, nsys);
                wilson_dslash(lat, d, h, dag, EPI_XPAY, other, o, &same, nullptr, st);
            }
        };
        std::vector<Field> Y, P;
        for (int i = 0; i < ns; i++) {
            Y.push_back(pool.get(WF, ps, nf));
            P.push_back(pool.get(WF, ps, nf));
            blas_zero(Y[i], st);
            blas_copy(P[i], R, st);
        }
        Scalars sc;
        sc.init(lat, nf, st);
        // per-system norm: the halves' partials, added on the host
        auto norms = [&](int slot, std::vector<double>& out) {
            sc.pull(st);
            out.resize(nsys);
            for (int j = 0; j < nsys; j++) out[j] = sc.h(j, slot) + sc.h(nsys + j, slot);
        };
        auto per_rhs = [&](const std::vector<double>& v) {  // system values repeated for both halves
            std::vector<double> o(nf);
            for (int j = 0; j < nsys; j++) o[j] = o[nsys + j] = v[j];
            return o;
        };
        blas_norm2(R, sc.part, st, sc.f(SC_RR, FIN_SET));
        std::vector<double> rr, pp, b2;
        norms(SC_RR, rr);
        pp = rr;
        b2 = rr;
        const double tol_ms = ps == LQ_F64 ? 0.1 * sp.tol : (ps == LQ_F32 ? 1e-6 : 1e-3);
        std::vector<double> alpha(nsys), beta(nsys), alpha_prev(nsys, 1.0), beta_prev(nsys, 0.0);
        std::vector<std::vector<double>> zeta(ns, std::vector<double>(nsys, 1.0)), zeta_prev = zeta, zn = zeta;
        std::vector<std::vector<char>> active(ns, std::vector<char>(nsys, 1));
        for (int j = 0; j < nsys; j++) {
            check_finite(b2[j], "source");
            if (b2[j] == 0.0)
                for (int i = 0; i < ns; i++) active[i][j] = 0;
        }
        auto any_active = [&]() {
            for (int i = 0; i < ns; i++)
                for (int j = 0; j < nsys; j++)
                    if (active[i][j]) return true;
            return false;
        };
        std::vector<double> tt, rrn, ppn, ones(nf, 1.0);
        while (any_active() && ms_iters < maxiter) {
            m0(0, P[0], T);
            blas_norm2(T, sc.part, st, sc.f(SC_QQ, FIN_SET));
            m0(1, T, Q);
            norms(SC_QQ, tt);
            for (int j = 0; j < nsys; j++) {
                const double pap = sigma[0] * pp[j] + tt[j];
                alpha[j] = (pap > 0.0 && b2[j] > 0.0) ? rr[j] / pap : 0.0;
                for (int i = 1; i < ns; i++) {
                    const double dd = sigma[i] - sigma[0];
                    const double den = alpha[j] * beta_prev[j] * (zeta_prev[i][j] - zeta[i][j]) +
                                       zeta_prev[i][j] * alpha_prev[j] * (1.0 + dd * alpha[j]);
                    zn[i][j] = den != 0.0 ? zeta[i][j] * zeta_prev[i][j] * alpha_prev[j] / den : 0.0;
                }
            }
            // Q = (A + sigma_0) P_0
            blas_axpy_h(Q, per_rhs(std::vector<double>(nsys, sigma[0])).data(), P[0], st);
            for (int i = 0; i < ns; i++) {
                std::vector<double> ai(nsys);
                for (int j = 0; j < nsys; j++)
                    ai[j] = !active[i][j] ? 0.0 : (i == 0 ? alpha[j] : alpha[j] * zn[i][j] / zeta[i][j]);
                blas_axpy_h(Y[i], per_rhs(ai).data(), P[i], st);
            }
            std::vector<double> na(nsys);
            for (int j = 0; j < nsys; j++) na[j] = -alpha[j];
            blas_axpby_h(R, per_rhs(na).data(), Q, ones.data(), sc.part, st);
            sc.fin(RED_BLOCKS, SC_RRN, st);
            norms(SC_RRN, rrn);
            for (int j = 0; j < nsys; j++) {
                check_finite(rrn[j], "multi-shift residual");
                beta[j] = rr[j] > 0.0 ? rrn[j] / rr[j] : 0.0;
                rr[j] = rrn[j];
            }
            blas_axpby_h(P[0], ones.data(), R, per_rhs(beta).data(), sc.part, st);
            sc.fin(RED_BLOCKS, SC_PP, st);
            for (int i = 1; i < ns; i++) {
                std::vector<double> zz(nsys), bz(nsys);
                for (int j = 0; j < nsys; j++) {
                    const double zr = zeta[i][j] != 0.0 ? zn[i][j] / zeta[i][j] : 0.0;
                    zz[j] = active[i][j] ? zn[i][j] : 0.0;
                    bz[j] = active[i][j] ? beta[j] * zr * zr : 1.0;
                }
                blas_axpby_h(P[i], per_rhs(zz).data(), R, per_rhs(bz).data(), nullptr, st);
            }
            for (int j = 0; j < nsys; j++) {
                for (int i = 1; i < ns; i++) {
                    zeta_prev[i][j] = zeta[i][j];
                    zeta[i][j] = zn[i][j];
                }
                alpha_prev[j] = alpha[j];
                beta_prev[j] = beta[j];
                for (int i = 0; i < ns; i++) {
                    const double z = i == 0 ? 1.0 : fabs(zeta[i][j]);
                    if (active[i][j] && z * sqrt(rr[j]) <= tol_ms * sqrt(b2[j])) active[i][j] = 0;
                }
            }
            norms(SC_PP, ppn);
            pp = ppn;
            ms_iters++;
        }
        // x(mu_i) = y1_i - i mu_i y2_i, written to the caller's arrays as the refinement's guesses
        Field X = pool.get(WF, ps, 2 * nrhs);
        for (int i = 0; i < ns; i++) {
            std::vector<double> re(nrhs, 0.0), im(nrhs, -mus[i]);
            for (int h = 0; h < 2; h++) {
                Field xh = X.sub(h * nrhs, nrhs);
                blas_copy(xh, Y[i].sub(h * nsys, nrhs), st);
                blas_caxpy_h(xh, re.data(), im.data(), Y[i].sub(h * nsys + nrhs, nrhs), st);
            }
            for (int k = 0; k < nrhs; k++) {
                export_field(lat, X, k, 0, x[k * ns + i], st);
                export_field(lat, X, nrhs + k, 1, x[k * ns + i], st);
            }
        }
        LQ_CUDA(cudaStreamSynchronize(st));
    }

    // refinement of every twisted mass by the mixed-precision even-odd CGNR from its guess
    int ret = LQ_OK;
    std::vector<lq_solve_info> acc(nrhs);
    for (int k = 0; k < nrhs; k++) {
        acc[k] = lq_solve_info{LQ_OK, ms_iters, 0, 2 * ms_iters, 0.0, 0.0};
    }
    for (int i = 0; i < ns; i++) {
        lq_op_params opi = opp;
        opi.mu = mus[i];
        lq_solve_params spi = sp;
        spi.solver = ps == LQ_F64 ? LQ_CGNR : LQ_MIXED_CGNR;
        spi.nshift = 0;
        spi.masses = nullptr;
        std::vector<double*> xi(nrhs);
        std::vector<const double*> x0(nrhs);
        for (int k = 0; k < nrhs; k++) {
            xi[k] = x[k * ns + i];
            x0[k] = x[k * ns + i];
        }
        std::vector<lq_solve_info> inf(nrhs);
        // solution k of this mass is x[k * ns + i] of the caller's array
        SolutionReady ready_i = [&](int k, cudaStream_t s) { (*ready)(k * ns + i, s); };
        int r = solve_wilson(lat, opi, spi, nrhs, b, xi.data(), inf.data(), st, x0.data(),
                             ready ? &ready_i : nullptr);
        if (r != LQ_OK && ret == LQ_OK) ret = r;
        for (int k = 0; k < nrhs; k++) {
            acc[k].iters += inf[k].iters;
            acc[k].reliable_updates += inf[k].reliable_updates;
            acc[k].operator_applications += inf[k].operator_applications;
            acc[k].true_rel_residual = std::max(acc[k].true_rel_residual, inf[k].true_rel_residual);
            acc[k].seconds += inf[k].seconds;
            if (inf[k].status != LQ_OK && acc[k].status == LQ_OK) acc[k].status = inf[k].status;
        }
    }
    if (info)
        for (int k = 0; k < nrhs; k++) info[k] = acc[k];
    if (ret != LQ_OK) set_last_error("solve: not every right-hand side reached the tolerance");
    return ret;
}

// ===================================================================== HISQ
static OpDesc hisq_desc(const lq_op_params& op, int prec, int recon) {
    OpDesc d;
    d.action = LQ_HISQ;
    d.m = op.m;
    d.mu = 0.0;
    d.c_naik = op.c_naik;
    d.prec = prec;
    d.recon = prec == LQ_F64 ? 18 : recon;
    return d;
}

// out = sigma in - H_eo H_oe in; t = H_oe in (odd). part_t receives |t|^2 partials,
// so that (in, out) = sigma |in|^2 + |t|^2 (since -H_eo = H_oe^+).
int schur_hisq(Lattice& lat, const OpDesc& op, double sigma, const Field& in, Field& out, Field& t, df* part_t,
               cudaStream_t st, const FinArgs& fin, const double* sigma_dev) {
    int nb = hisq_dslash(lat, op, 1, 0, EPI_HOP, 0.0, in, t, nullptr, part_t, st, fin);
    hisq_dslash(lat, op, 0, 0, EPI_XPAY, sigma, t, out, &in, nullptr, st, FinArgs(), sigma_dev);
    return nb;
}

// Mixed-precision CG for A x = b, A = sigma - H_eo H_oe = sigma + H_oe^+ H_oe
// (hermitian positive definite), from the initial guess in x_hi, on the Krylov
// driver: (p, A p) = sigma |p|^2 + |H_oe p|^2 with |H_oe p|^2 finalised in the
// kernel that forms H_oe p, alpha and beta on the device; a reliable update
// recomputes r = b - A x_hi in FP64 accuracy and keeps p.
static CgResult cg_hisq(Lattice& lat, const OpDesc& ops, const OpDesc& op64, const std::vector<double>& sigma,
                        const Field& b, Field& x_hi, const std::vector<double>& tol_abs, double delta, int maxiter,
                        int graph_iters, cudaStream_t st) {
    const int n = b.nrhs;
    const int ps = ops.prec, px = ps == LQ_F16 ? LQ_F32 : ps;
    const int SF = LQ_STAGGERED_FIELD;
    Pool pool(lat, st);
    const int ph = op64.prec;
    Field r_hi = pool.get(SF, ph, n), q64 = pool.get(SF, ph, n), t64 = pool.get(SF, ph, n);
    Field x_lo = pool.get(SF, px, n);
    Field r = pool.get(SF, ps, n), p = pool.get(SF, ps, n), q = pool.get(SF, ps, n), t = pool.get(SF, ps, n);
    Scalars sc;
    sc.init(lat, n, st);
    // the shift of every right-hand side (one operator sigma_k - H_eo H_oe per rhs)
    for (int k = 0; k < n; k++) sc.h(k, SC_SIGMA) = sigma[k];
    LQ_CUDA(cudaMemcpyAsync(sc.dev, sc.host, sizeof(double) * SC_N * n, cudaMemcpyHostToDevice, st));
    const double* sig = sc.dev + SC_SIGMA;
    CgResult res(n);
    std::vector<double> ones(n, 1.0);
    FinArgs falpha = sc.f(0, FIN_CG_ALPHA);

    // r = b - A x_hi in FP64 accuracy; |r|^2 -> SC_SS; the sloppy copy's |r|^2 -> SC_RR
    auto true_residual = [&]() {
        schur_hisq(lat, op64, 0.0, x_hi, q64, t64, nullptr, st, FinArgs(), sig);
        blas_xmy_norm(r_hi, b, q64, sc.part, st, sc.f(SC_SS, FIN_SET));
        blas_copy(r, r_hi, st);
        blas_norm2(r, sc.part, st, sc.f(SC_RR, FIN_SET));
    };
    blas_zero(x_lo, st);
    true_residual();
    blas_copy(p, r, st);
    blas_norm2(p, sc.part, st, sc.f(SC_PP, FIN_SET));
    sc.pull(st);
    KrylovState ks = krylov_start(sc, res, tol_abs, st);
    auto iteration = [&](double* dst) {
        // q = A p; alpha from the hop kernel's partials of |H_oe p|^2 by a one-block finalise
        // kernel (a finalising last block would cost every block of the hop a fence and an
        // atomic at its end)
        const int nb = schur_hisq(lat, ops, 0.0, p, q, t, sc.part, st, FinArgs(), sig);
        blas_finalize(sc.part, nb, n, sc.dev, falpha.slot, falpha.op, st);
        blas_cg_s(r, q, sc.dev, sc.part, st, sc.f(0, FIN_CG_BETA));                // r, |r|^2, beta
        blas_cg_xp_norm(x_lo, p, r, sc.dev, sc.part, st, sc.f(SC_PP, FIN_SET));  // x += alpha p, p = r + beta p, |p|^2
        if (dst) LQ_CUDA(cudaMemcpyAsync(dst, sc.dev, sizeof(double) * SC_N * n, cudaMemcpyDeviceToHost, st));
    };
    auto update = [&]() {
        blas_axpy_h_zero(x_hi, ones.data(), x_lo, st);
        true_residual();
        for (int k = 0; k < n; k++)
            if (!ks.done[k]) res.applications[k] += 1;
    };
    auto after_update = [&](int k) {
        if (sc.h(k, SC_BREAK) == 0.0) return true;
        res.status[k] = LQ_EBREAKDOWN;
        return false;
    };
    krylov_loop(lat, sc, res, ks, tol_abs, delta, maxiter, graph_iters, 1, st, iteration, update, after_update);
    return res;
}

// Multi-shift CG in one precision for (sigma_i - H_eo H_oe) y_i = b, shifts
// ascending, one Krylov space. Stops when every shift's iterated residual
// |zeta_i| |r| is below tol_rel |b|. Returns the iterations.
static int multishift_hisq(Lattice& lat, const OpDesc& op, const std::vector<double>& sigma, const Field& b,
                           std::vector<Field>& y, double tol_rel, int maxiter, cudaStream_t st) {
    const int n = b.nrhs, ns = (int)sigma.size();
    Pool pool(lat, st);
    Field r = pool.get(LQ_STAGGERED_FIELD, op.prec, n), q = pool.get(LQ_STAGGERED_FIELD, op.prec, n);
    Field t = pool.get(LQ_STAGGERED_FIELD, op.prec, n);
    std::vector<Field> p;
    for (int i = 0; i < ns; i++) p.push_back(pool.get(LQ_STAGGERED_FIELD, op.prec, n));
    Scalars sc;
    sc.init(lat, n, st);
    blas_copy(r, b, st);
    for (int i = 0; i < ns; i++) {
        blas_copy(p[i], b, st);
        blas_zero(y[i], st);
    }
    blas_norm2(r, sc.part, st);
    sc.fin(RED_BLOCKS, SC_RR, st);
    sc.pull(st);
    std::vector<double> rr(n), pp(n), b2(n), alpha_prev(n, 1.0), beta_prev(n, 0.0), alpha(n), beta(n);
    std::vector<std::vector<double>> zeta(ns, std::vector<double>(n, 1.0)), zeta_prev = zeta, zn = zeta;
    std::vector<std::vector<char>> active(ns, std::vector<char>(n, 1));
    for (int k = 0; k < n; k++) {
        rr[k] = pp[k] = b2[k] = sc.h(k, SC_RR);
        check_finite(b2[k], "source");
        if (b2[k] == 0.0)
            for (int i = 0; i < ns; i++) active[i][k] = 0;
    }
    std::vector<double> a(n), bz(n), zz(n), ones(n, 1.0);
    std::vector<double> ya((size_t)ns * n), pz((size_t)ns * n), pb((size_t)ns * n);  // fused-update coefficients
    auto any_active = [&]() {
        for (int i = 0; i < ns; i++)
            for (int k = 0; k < n; k++)
                if (active[i][k]) return true;
        return false;
    };
    int iters = 0;
    while (any_active() && iters < maxiter) {
        int nb = schur_hisq(lat, op, sigma[0], p[0], q, t, sc.part, st);
        sc.fin(nb, SC_QQ, st);
        sc.pull(st);
        for (int k = 0; k < n; k++) {
            double pap = sigma[0] * pp[k] + sc.h(k, SC_QQ);
            alpha[k] = (pap > 0.0 && b2[k] > 0.0) ? rr[k] / pap : 0.0;
            for (int i = 1; i < ns; i++) {
                double d = sigma[i] - sigma[0];
                double den = alpha[k] * beta_prev[k] * (zeta_prev[i][k] - zeta[i][k]) +
                             zeta_prev[i][k] * alpha_prev[k] * (1.0 + d * alpha[k]);
                zn[i][k] = den != 0.0 ? zeta[i][k] * zeta_prev[i][k] * alpha_prev[k] / den : 0.0;
            }
        }
        // y_i += alpha_i p_i, alpha_i = alpha zeta_i'/zeta_i (fused with the p_i updates below
        // into one pass when the counts allow it)
        const bool fused = ns <= LQ_MS_MAXS && n <= LQ_MS_MAXK;
        for (int i = 0; i < ns; i++) {
            for (int k = 0; k < n; k++)
                a[k] = !active[i][k] ? 0.0 : (i == 0 ? alpha[k] : alpha[k] * zn[i][k] / zeta[i][k]);
            if (fused) std::copy(a.begin(), a.end(), ya.begin() + (size_t)i * n);
            else blas_axpy_h(y[i], a.data(), p[i], st);
        }
        for (int k = 0; k < n; k++) a[k] = -alpha[k];
        blas_axpby_h(r, a.data(), q, ones.data(), sc.part, st);
        sc.fin(RED_BLOCKS, SC_RRN, st);
        sc.pull(st);
        for (int k = 0; k < n; k++) {
            double rn = sc.h(k, SC_RRN);
            check_finite(rn, "multi-shift residual");
            beta[k] = rr[k] > 0.0 ? rn / rr[k] : 0.0;
            rr[k] = rn;
        }
        // p_0 = r + beta p_0 ; p_i = zeta_i' r + beta (zeta_i'/zeta_i)^2 p_i
        if (fused) {
            for (int k = 0; k < n; k++) {
                pz[k] = 1.0;
                pb[k] = beta[k];
            }
            for (int i = 1; i < ns; i++)
                for (int k = 0; k < n; k++) {
                    double zr = zeta[i][k] != 0.0 ? zn[i][k] / zeta[i][k] : 0.0;
                    pz[(size_t)i * n + k] = active[i][k] ? zn[i][k] : 0.0;
                    pb[(size_t)i * n + k] = active[i][k] ? beta[k] * zr * zr : 1.0;
                }
            blas_ms_update(y, p, r, ya.data(), pz.data(), pb.data(), sc.part, st);
            sc.fin(RED_BLOCKS, SC_PP, st);
        } else {
            blas_axpby_h(p[0], ones.data(), r, beta.data(), sc.part, st);
            sc.fin(RED_BLOCKS, SC_PP, st);
            for (int i = 1; i < ns; i++) {
                for (int k = 0; k < n; k++) {
                    double zr = zeta[i][k] != 0.0 ? zn[i][k] / zeta[i][k] : 0.0;
                    zz[k] = active[i][k] ? zn[i][k] : 0.0;
                    bz[k] = active[i][k] ? beta[k] * zr * zr : 1.0;
                }
                blas_axpby_h(p[i], zz.data(), r, bz.data(), nullptr, st);
            }
        }
        for (int k = 0; k < n; k++) {
            for (int i = 1; i < ns; i++) {
                zeta_prev[i][k] = zeta[i][k];
                zeta[i][k] = zn[i][k];
            }
            alpha_prev[k] = alpha[k];
            beta_prev[k] = beta[k];
            for (int i = 0; i < ns; i++) {
                double z = i == 0 ? 1.0 : fabs(zeta[i][k]);
                if (active[i][k] && z * sqrt(rr[k]) <= tol_rel * sqrt(b2[k])) active[i][k] = 0;
            }
        }
        sc.pull(st);
        for (int k = 0; k < n; k++) pp[k] = sc.h(k, SC_PP);
        iters++;
    }
    return iters;
}

int solve_hisq(Lattice& lat, const lq_op_params& opp, const lq_solve_params& sp, int nrhs, const double* const* b,
               double* const* x, lq_solve_info* info, cudaStream_t st, const SolutionReady* ready) {
    if (!lat.canon[LQ_FAT] || !lat.canon[LQ_LONG]) fail(LQ_EINVAL, "HISQ needs fat and long links loaded");
    if (nrhs < 1 || nrhs > 32) fail(LQ_EINVAL, "nrhs must be in [1, 32] for HISQ");
    if (sp.solver == LQ_BICGSTAB || sp.solver == LQ_GCR)
        fail(LQ_EINVAL, "BiCGStab and GCR are for Wilson actions (the HISQ Schur operator is hermitian positive)");
    int ps = sp.prec_sloppy;
    if (ps < LQ_F64 || ps > LQ_F16) fail(LQ_EINVAL, "prec_sloppy");
    if (!(sp.tol > 0)) fail(LQ_EINVAL, "tol must be positive");
    const int recon = sloppy_recon(sp);
    const int ph = ps == LQ_F64 ? LQ_F64 : LQ_F32X2;
    const OpDesc op64 = hisq_desc(opp, ph, 18);
    const OpDesc ops = hisq_desc(opp, ps, recon);
    const double delta = (ps == LQ_F64) ? 0.0 : (sp.delta > 0 ? sp.delta : 0.1);
    const int maxiter = sp.maxiter > 0 ? sp.maxiter : 100000;
    std::vector<double> masses;
    if (sp.solver == LQ_MULTISHIFT_CG) {
        if (sp.nshift < 1 || sp.nshift > 16 || !sp.masses) fail(LQ_EINVAL, "multi-shift solve needs 1..16 masses");
        for (int i = 0; i < sp.nshift; i++) masses.push_back(sp.masses[i]);
        for (int i = 1; i < sp.nshift; i++)
            if (masses[i] < masses[i - 1]) fail(LQ_EINVAL, "multi-shift masses must be ascending");
    } else {
        masses.push_back(opp.m);
    }
    for (double m : masses)
        if (!(m > 0.0)) fail(LQ_EINVAL, "HISQ mass must be positive");
    const int ns = (int)masses.size();

    cudaEvent_t e0, e1;
    LQ_CUDA(cudaEventCreate(&e0));
    LQ_CUDA(cudaEventCreate(&e1));
    LQ_CUDA(cudaEventRecord(e0, st));
    Pool pool(lat, st);
    const int SF = LQ_STAGGERED_FIELD;
    Field be = pool.get(SF, ph, nrhs), bo = pool.get(SF, ph, nrhs), c = pool.get(SF, ph, nrhs);
    Field bh = pool.get(SF, ph, nrhs), xe = pool.get(SF, ph, nrhs), xo = pool.get(SF, ph, nrhs);
    Field te = pool.get(SF, ph, nrhs), to = pool.get(SF, ph, nrhs);
    Scalars sc;
    sc.init(lat, nrhs, st);
    int ret = LQ_OK;
    try {
        for (int k = 0; k < nrhs; k++) {
            import_field(lat, be, k, 0, b[k], st);
            import_field(lat, bo, k, 1, b[k], st);
        }
        blas_norm2(be, sc.part, st);
        sc.fin(RED_BLOCKS, SC_B2, st);
        blas_norm2(bo, sc.part, st);
        sc.fin(RED_BLOCKS, SC_SS, st);
        sc.pull(st);
        std::vector<double> bn(nrhs), tol_abs(nrhs);
        for (int k = 0; k < nrhs; k++) {
            double b2 = sc.h(k, SC_B2) + sc.h(k, SC_SS);
            check_finite(b2, "source");
            bn[k] = sqrt(b2);
        }
        // c = H_eo b_o
        hisq_dslash(lat, op64, 0, 0, EPI_HOP, 0.0, bo, c, nullptr, nullptr, st);

        // sloppy multi-shift stage on the 2*nrhs right-hand sides [b_e, c]:
        // x_e,i = m_i (A + m_i^2)^{-1} b_e - (A + m_i^2)^{-1} c
        std::vector<double> sigma(ns);
        for (int i = 0; i < ns; i++) sigma[i] = masses[i] * masses[i];
        std::vector<Field> ys;
        int ms_iters = 0;
        if (ns > 1) {
            Field b2f = pool.get(SF, ps, 2 * nrhs);
            Field lo = b2f.sub(0, nrhs), hi = b2f.sub(nrhs, nrhs);
            blas_copy(lo, be, st);
            blas_copy(hi, c, st);
            for (int i = 0; i < ns; i++) ys.push_back(pool.get(SF, ps, 2 * nrhs));
            const double tol_ms = ps == LQ_F64 ? 0.1 * sp.tol : (ps == LQ_F32 ? 1e-6 : 1e-3);
            ms_iters = multishift_hisq(lat, ops, sigma, b2f, ys, tol_ms, maxiter, st);
        }

        std::vector<int> tot_iters(nrhs, ms_iters), tot_upd(nrhs, 0), tot_app(nrhs, ms_iters);
        std::vector<double> worst(nrhs, 0.0);
        std::vector<int> status(nrhs, LQ_OK);
        std::vector<double> one(nrhs, 1.0), neg(nrhs, -1.0);
        // Refinement of every mass by the mixed CG from the multi-shift guess, one
        // mass at a time: each stops at its own iteration count. (Solving all
        // masses together as one multi-rhs system with a shift per rhs was measured
        // slower at 48^3x144: the FP16 HISQ kernel is bound by its per-rhs decode
        // and arithmetic, not by the shared link loads, and every mass then runs
        // for the lightest mass's iterations.)
        for (int i = 0; i < ns; i++) {
            const double m = masses[i];
            // bhat_i = m b_e - c; initial guess m y_1 - y_2 from the multi-shift stage, or zero
            std::vector<double> am(nrhs, m);
            blas_copy(bh, c, st);
            blas_axpby_h(bh, am.data(), be, neg.data(), nullptr, st);
            if (ns > 1) {
                Field y1 = ys[i].sub(0, nrhs), y2 = ys[i].sub(nrhs, nrhs);
                blas_copy(xe, y2, st);
                blas_copy(te, y1, st);
                blas_axpby_h(xe, am.data(), te, neg.data(), nullptr, st);
            } else {
                blas_zero(xe, st);
            }
            // the even part of the full residual is (bhat - A x_e) / m
            for (int k = 0; k < nrhs; k++) tol_abs[k] = 0.5 * sp.tol * bn[k] * m;
            CgResult cr = cg_hisq(lat, ops, op64, std::vector<double>(nrhs, sigma[i]), bh, xe, tol_abs, delta,
                                  maxiter, sp.graph_iters, st);
            // x_o = (b_o - H_oe x_e) / m
            hisq_dslash(lat, op64, 1, 0, EPI_HOP, 0.0, xe, to, nullptr, nullptr, st);
            blas_copy(xo, to, st);
            std::vector<double> ai(nrhs, 1.0 / m), bi(nrhs, -1.0 / m);
            blas_axpby_h(xo, ai.data(), bo, bi.data(), nullptr, st);
            for (int k = 0; k < nrhs; k++) {
                export_field(lat, xe, k, 0, x[k * ns + i], st);
                export_field(lat, xo, k, 1, x[k * ns + i], st);
                if (ready) (*ready)(k * ns + i, st);
            }
            // FP64 true residual: r_p = b_p - (m x_p + H x_{1-p}); XPAY gives -(m x_p + H x_{1-p})
            hisq_dslash(lat, op64, 0, 0, EPI_XPAY, -m, xo, te, &xe, nullptr, st);
            blas_axpby_h(te, one.data(), be, one.data(), sc.part, st);
            sc.fin(RED_BLOCKS, SC_RR, st);
            hisq_dslash(lat, op64, 1, 0, EPI_XPAY, -m, xe, to, &xo, nullptr, st);
            blas_axpby_h(to, one.data(), bo, one.data(), sc.part, st);
            sc.fin(RED_BLOCKS, SC_QQ, st);
            sc.pull(st);
            for (int k = 0; k < nrhs; k++) {
                double rr = sqrt(sc.h(k, SC_RR) + sc.h(k, SC_QQ)) / bn[k];
                worst[k] = std::max(worst[k], rr);
                tot_iters[k] += cr.iters[k];
                tot_upd[k] += cr.updates[k];
                tot_app[k] += cr.applications[k];
                int stt = cr.status[k];
                if (stt == LQ_OK && !(rr <= sp.tol)) stt = LQ_ENOTCONV;
                if (!std::isfinite(rr)) stt = LQ_ENAN;
                if (stt != LQ_OK) status[k] = stt;
            }
        }
        LQ_CUDA(cudaEventRecord(e1, st));
        LQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        for (int k = 0; k < nrhs; k++) {
            if (status[k] != LQ_OK && ret == LQ_OK) ret = status[k];
            if (info) {
                info[k].status = status[k];
                info[k].iters = tot_iters[k];
                info[k].reliable_updates = tot_upd[k];
                info[k].operator_applications = tot_app[k];
                info[k].true_rel_residual = worst[k];
                info[k].seconds = ms * 1e-3;
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ret != LQ_OK) set_last_error("solve: not every right-hand side reached the tolerance");
    return ret;
}

}  // namespace lq
