// server.cu -- request server for propagator solves with continuous batching.
//
// Requests wait in a queue in arrival order. When a worker slot is free, the
// first queued request whose estimated device workspace, added to what the
// running requests have reserved, fits in the HBM budget is admitted (the
// resident lattices are counted once, when first used); a request that does not
// fit yet is overtaken by later ones that do, but at most max_bypass() times,
// after which nothing behind it is admitted until it is (so a large request is
// not starved by a stream of small ones). Each worker owns a CUDA stream, so an
// admitted request starts while earlier ones are still on the GPU and their
// kernels overlap. A request that cannot fit even alone is rejected at
// submission.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <new>
#include <set>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using namespace lq;

namespace {

struct Request {
    uint64_t ticket;
    lq_request req;
    std::vector<double> masses;
    std::vector<std::vector<double>> rhs;  // nrhs canonical host arrays, dropped once solved
    std::vector<std::vector<double>> x;    // solutions, allocated when the request is admitted
    int nsol = 0;
    size_t n = 0;                          // reals per canonical field
    std::vector<lq_solve_info> info;
    size_t reserve = 0;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int status = LQ_EAGAIN;
    bool done = false;
    int bypassed = 0;                      // times a later request was admitted first
};

}  // namespace

struct lq_server_s {
    size_t budget;
    int max_slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> all;
    std::set<Lattice*> seen_lattices;
    size_t reserved = 0;
    size_t lattice_bytes = 0;
    int running = 0;
    bool stop = false;
    uint64_t next_ticket = 1;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::vector<std::thread> workers;

    // how often a queued request may be overtaken before it blocks the queue
    int max_bypass() const { return 2 * max_slots; }
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void worker();
};

namespace lq {

size_t solve_workspace_bytes(const Lattice& lat, const lq_op_params& op, const lq_solve_params& sp, int nrhs) {
    const bool hisq = op.action == LQ_HISQ;
    const int kind = hisq ? LQ_STAGGERED_FIELD : LQ_WILSON_FIELD;
    const int ps = sp.prec_sloppy;
    const int px = ps == LQ_F16 ? LQ_F32 : ps;
    const int ns = (hisq && sp.solver == LQ_MULTISHIFT_CG) ? std::max(1, sp.nshift) : 1;
    size_t f64 = field_bytes(kind, LQ_F64, nrhs, lat.vh);
    size_t fs = field_bytes(kind, ps, nrhs, lat.vh);
    size_t fx = field_bytes(kind, px, nrhs, lat.vh);
    size_t canon = (size_t)lat.V * (hisq ? 6 : 24) * sizeof(double) * (size_t)(nrhs + nrhs * ns);
    size_t b;
    if (!hisq) {
        const int kg = sp.restart > 0 ? sp.restart : GCR_DEFAULT;
        b = 7 * f64 + 3 * f64 + fx + (sp.solver == LQ_BICGSTAB ? 6 : sp.solver == LQ_GCR ? 2 + 2 * kg : 5) * fs;
    } else {
        b = 8 * f64 + 3 * f64 + fx + 4 * fs;
        if (ns > 1) b += (size_t)(3 + 2 * ns) * field_bytes(kind, ps, 2 * nrhs, lat.vh);
    }
    // a twisted-clover request may need a new clover inverse (sloppy + double-float
    // copies, and a temporary FP64 one while it is built)
    if (op.action == LQ_WILSON_TM_CLOVER) b += (size_t)144 * 2 * lat.vh * (prec_bytes(ps) + 8 + 8);
    return b + canon + (16u << 20);
}

}  // namespace lq

void lq_server_s::worker() {
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop) break;
                // the first request in arrival order that fits; one that has been
                // overtaken max_bypass() times holds back everything behind it
                auto pick = queue.end();
                size_t extra = 0;
                for (auto it = queue.begin(); it != queue.end(); ++it) {
                    Lattice* L = &(*it)->req.lat->lat;
                    extra = seen_lattices.count(L) ? 0 : L->bytes;
                    if (reserved + lattice_bytes + extra + (*it)->reserve <= budget || running == 0) {
                        pick = it;
                        break;
                    }
                    if ((*it)->bypassed >= max_bypass()) break;
                }
                if (pick != queue.end()) {
                    for (auto it = queue.begin(); it != pick; ++it) (*it)->bypassed++;
                    r = *pick;
                    queue.erase(pick);
                    if (extra) {
                        seen_lattices.insert(&r->req.lat->lat);
                        lattice_bytes += extra;
                    }
                    reserved += r->reserve;
                    running++;
                    r->t_admit = now();
                    break;
                }
                cv_work.wait(lk);
            }
            if (!r) break;
        }
        int status = LQ_OK;
        // host memory of a request: its sources while queued, the solutions from
        // admission until polled
        try {
            r->x.assign(r->nsol, std::vector<double>(r->n));
        } catch (const std::bad_alloc&) {
            std::vector<std::vector<double>>().swap(r->x);
            status = LQ_ENOMEM;
        }
        if (status == LQ_OK) {
            const int nsol = r->nsol;
            std::vector<const double*> b(r->rhs.size());
            std::vector<double*> x(nsol);
            for (size_t k = 0; k < b.size(); k++) b[k] = r->rhs[k].data();
            for (int k = 0; k < nsol; k++) x[k] = r->x[k].data();
            lq_solve_params sp = r->req.solve;
            sp.masses = r->masses.empty() ? nullptr : r->masses.data();
            status = lq_solve(r->req.lat, &r->req.op, &sp, r->req.nrhs, b.data(), x.data(), LQ_HOST,
                              r->info.data(), st);
            // the admission ledger counts a request's work buffers only while it runs
            ws_release(r->req.lat->lat);
        }
        std::vector<std::vector<double>>().swap(r->rhs);
        {
            std::lock_guard<std::mutex> lk(mu);
            r->status = status;
            r->t_finish = now();
            r->done = true;
            reserved -= r->reserve;
            running--;
        }
        cv_work.notify_all();
        cv_done.notify_all();
    }
    cudaStreamDestroy(st);
}

#define LQ_TRY try {
#define LQ_CATCH                                      \
    }                                                 \
    catch (const Error& e) {                          \
        set_last_error(e.msg);                        \
        return e.code;                                \
    }                                                 \
    catch (const std::bad_alloc&) {                   \
        set_last_error("host allocation failed");     \
        return LQ_ENOMEM;                             \
    }                                                 \
    catch (...) {                                     \
        set_last_error("unexpected internal error");  \
        return LQ_EINVAL;                             \
    }

extern "C" int lq_server_create(size_t hbm_budget_bytes, int max_slots, lq_server* out) {
    LQ_TRY
    if (!out || max_slots < 1 || max_slots > 64) fail(LQ_EINVAL, "max_slots must be in [1, 64]");
    lq_server s = new lq_server_s();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    for (int i = 0; i < max_slots; i++) s->workers.emplace_back([s] { s->worker(); });
    *out = s;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_server_destroy(lq_server s) {
    LQ_TRY
    if (!s) return LQ_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->all) delete kv.second;
    delete s;
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_submit(lq_server s, const lq_request* req, const double* const* rhs, uint64_t* ticket) {
    LQ_TRY
    if (!s || !req || !rhs || !ticket || !req->lat) fail(LQ_EINVAL, "null argument");
    if (req->nrhs < 1 || req->nrhs > 64) fail(LQ_EINVAL, "nrhs must be in [1, 64]");
    const Lattice& L = req->lat->lat;
    Request* r = new Request();
    r->req = *req;
    const bool ms = req->op.action == LQ_HISQ && req->solve.solver == LQ_MULTISHIFT_CG;
    if (ms) {
        if (req->solve.nshift < 1 || !req->solve.masses) {
            delete r;
            fail(LQ_EINVAL, "multi-shift request without masses");
        }
        r->masses.assign(req->solve.masses, req->solve.masses + req->solve.nshift);
    }
    const size_t n = (size_t)L.V * (req->op.action == LQ_HISQ ? 6 : 24);
    for (int k = 0; k < req->nrhs; k++) {
        if (!rhs[k]) {
            delete r;
            fail(LQ_EINVAL, "null right-hand side");
        }
        r->rhs.emplace_back(rhs[k], rhs[k] + n);
    }
    r->nsol = req->nrhs * (ms ? req->solve.nshift : 1);
    r->n = n;
    r->info.assign(req->nrhs, lq_solve_info{});
    r->reserve = solve_workspace_bytes(L, req->op, req->solve, req->nrhs);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            fail(LQ_EBUSY, "server is shutting down");
        }
        if (r->reserve + L.bytes > s->budget) {
            delete r;
            fail(LQ_ENOMEM, "request does not fit in the server's HBM budget");
        }
        r->ticket = s->next_ticket++;
        r->t_submit = s->now();
        s->queue.push_back(r);
        s->all[r->ticket] = r;
        *ticket = r->ticket;
    }
    s->cv_work.notify_all();
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_poll(lq_server s, uint64_t ticket, double* const* x, lq_solve_info* info, lq_request_times* times) {
    LQ_TRY
    if (!s) fail(LQ_EINVAL, "null server");
    Request* r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) fail(LQ_EINVAL, "unknown ticket");
        r = it->second;
        if (!r->done) return LQ_EAGAIN;
        s->all.erase(it);
    }
    if (x)
        for (size_t k = 0; k < r->x.size(); k++)
            if (x[k]) memcpy(x[k], r->x[k].data(), r->x[k].size() * sizeof(double));
    if (info) memcpy(info, r->info.data(), r->info.size() * sizeof(lq_solve_info));
    if (times) {
        times->submitted = r->t_submit;
        times->admitted = r->t_admit;
        times->finished = r->t_finish;
    }
    int st = r->status;
    delete r;
    return st;
    LQ_CATCH
}

extern "C" int lq_wait(lq_server s, uint64_t ticket, int timeout_ms) {
    LQ_TRY
    if (!s) fail(LQ_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        auto it = s->all.find(ticket);
        return it == s->all.end() || it->second->done;
    };
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return LQ_ETIMEOUT;
    if (s->all.find(ticket) == s->all.end()) fail(LQ_EINVAL, "unknown ticket");
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_request_bytes(const lq_request* req, size_t* bytes) {
    LQ_TRY
    if (!req || !req->lat || !bytes) fail(LQ_EINVAL, "null argument");
    *bytes = solve_workspace_bytes(req->lat->lat, req->op, req->solve, req->nrhs);
    return LQ_OK;
    LQ_CATCH
}

extern "C" int lq_server_stats(lq_server s, int* queued, int* running, size_t* reserved_bytes) {
    LQ_TRY
    if (!s) fail(LQ_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->queue.size();
    if (running) *running = s->running;
    if (reserved_bytes) *reserved_bytes = s->reserved + s->lattice_bytes;
    return LQ_OK;
    LQ_CATCH
}
