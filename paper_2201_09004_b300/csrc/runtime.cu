// runtime.cu -- errors, launch bookkeeping, profiling events, autotuner, device
// memory and fields.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "runtime.h"

namespace lq {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }
void fail(int code, const std::string& msg) { throw Error{code, msg}; }

// ----------------------------------------------------------------- launches
static std::atomic<int64_t> g_launches{0};
// while this thread captures a graph: its launch count and profile records
static thread_local int64_t* t_cap_kernels = nullptr;
static thread_local std::vector<GraphProf>* t_cap_prof = nullptr;

void count_launch() {
    if (t_cap_kernels) {
        (*t_cap_kernels)++;  // counted once per replay instead
        return;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};
static std::vector<ProfRec> g_prof;                                   // recorded launches since reset
static std::vector<std::pair<std::string, float>> g_prof_done;       // timed graph-replayed launches
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_free;  // reusable event pairs

static std::pair<cudaEvent_t, cudaEvent_t> take_pair() {  // g_prof_mu held
    std::pair<cudaEvent_t, cudaEvent_t> ev;
    if (!g_prof_free.empty()) {
        ev = g_prof_free.back();
        g_prof_free.pop_back();
    } else {
        cudaEventCreate(&ev.first);
        cudaEventCreate(&ev.second);
    }
    return ev;
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// slots: -1 none, >= 0 an eager record, <= -2 a record of the graph being captured
int prof_begin(const char* name, cudaStream_t st) {
    if (!g_prof_on.load()) return -1;
    if (t_cap_prof) {
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        {
            std::lock_guard<std::mutex> lk(g_prof_mu);
            ev = take_pair();
        }
        cudaEventRecordWithFlags(ev.first, st, cudaEventRecordExternal);
        t_cap_prof->push_back(GraphProf{name, ev.first, ev.second});
        return -2 - (int)(t_cap_prof->size() - 1);
    }
    if (stream_capturing(st)) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::pair<cudaEvent_t, cudaEvent_t> ev = take_pair();
    cudaEventRecord(ev.first, st);
    g_prof.push_back(ProfRec{name, ev.first, ev.second});
    return (int)g_prof.size() - 1;
}

void prof_end(int slot, cudaStream_t st) {
    if (slot == -1) return;
    if (slot <= -2) {
        cudaEventRecordWithFlags((*t_cap_prof)[-2 - slot].b, st, cudaEventRecordExternal);
        return;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[slot].b, st);
}

// ------------------------------------------------------------- CUDA graphs
bool graph_capture_begin(cudaStream_t st) {
    // the legacy default stream cannot be captured
    if (st == nullptr || st == cudaStreamLegacy) return false;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    static thread_local int64_t kernels;
    static thread_local std::vector<GraphProf> prof;
    kernels = 0;
    prof.clear();
    t_cap_kernels = &kernels;
    t_cap_prof = &prof;
    return true;
}

bool graph_capture_end(cudaStream_t st, Graph& g) {
    std::vector<GraphProf> prof = *t_cap_prof;
    const int64_t kernels = *t_cap_kernels;
    t_cap_kernels = nullptr;
    t_cap_prof = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !exec) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto& r : prof) g_prof_free.push_back({r.a, r.b});
        return false;
    }
    g.exec = exec;
    g.prof.swap(prof);
    g.kernels = kernels;
    g.uncollected = false;
    return true;
}

void graph_launch(Graph& g, cudaStream_t st) {
    LQ_CUDA(cudaGraphLaunch(g.exec, st));
    g_launches.fetch_add(g.kernels, std::memory_order_relaxed);
    g.uncollected = !g.prof.empty();
}

void graph_collect(Graph& g) {
    if (!g.uncollected) return;
    g.uncollected = false;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g.prof) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
            g_prof_done.push_back({r.name, ms});
        else
            cudaGetLastError();
    }
}

void graph_destroy(Graph& g) {
    if (g.exec) {
        graph_collect(g);
        cudaGraphExecDestroy(g.exec);
    }
    g.exec = nullptr;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g.prof) g_prof_free.push_back({r.a, r.b});
    g.prof.clear();
}

static std::mutex g_smem_mu;
static std::unordered_map<const void*, size_t> g_smem_optin;

void opt_in_smem(const void* kernel, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    size_t& have = g_smem_optin[kernel];
    if (have >= bytes) return;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(LQ_ECUDA, "dynamic shared memory of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    have = bytes;
}

// ------------------------------------------------------------------- tuner
static std::mutex g_tune_mu;
static std::unordered_map<std::string, int> g_tuned;
static std::atomic<int> g_tune_force{0};

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        n = v > 0 ? v : 148;
    }
    return n;
}

// With LQ_TUNE_CACHE=<file>, tuned choices are read from the file on first use
// and every new choice is appended ("key code" per line), so that separate
// processes (a profiler run after a plain run) launch the same configurations.
static void tune_cache_load() {  // g_tune_mu held
    static bool loaded = false;
    if (loaded) return;
    loaded = true;
    const char* path = getenv("LQ_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[512];
    int code;
    while (fscanf(f, "%511s %d", key, &code) == 2) g_tuned[key] = code;
    fclose(f);
}

static void tune_cache_store(const std::string& key, int code) {  // g_tune_mu held
    const char* path = getenv("LQ_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", key.c_str(), code);
    fclose(f);
}

int tuned_block(const std::string& key, cudaStream_t st, const std::function<void(int)>& run,
                const std::vector<int>& candidates) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
    }
    if (stream_capturing(st)) return 128;
    std::vector<int> cand = candidates;
    const int forced = g_tune_force.load();
    if (forced && std::find(cand.begin(), cand.end(), forced) != cand.end()) cand = {forced};
    cudaEvent_t a, b;
    LQ_CUDA(cudaEventCreate(&a));
    LQ_CUDA(cudaEventCreate(&b));
    // tuning launches are not part of the caller's profile
    bool was_on = g_prof_on.exchange(false);
    int best = 128;
    float best_ms = 1e30f;
    try {
        for (int bs : cand) {
            try {
                run(bs);  // warm-up; a configuration that cannot launch is skipped
            } catch (const Error&) {
                continue;
            }
            // three separately timed launches; the median is the candidate's time
            float t3[3];
            for (int r = 0; r < 3; r++) {
                LQ_CUDA(cudaEventRecord(a, st));
                run(bs);
                LQ_CUDA(cudaEventRecord(b, st));
                LQ_CUDA(cudaEventSynchronize(b));
                LQ_CUDA(cudaEventElapsedTime(&t3[r], a, b));
            }
            std::sort(t3, t3 + 3);
            const float ms = t3[1];
            static const bool log = getenv("LQ_TUNE_LOG") != nullptr;  // diagnostics: every candidate's time
            if (log) fprintf(stderr, "lq tune %s candidate %d: %.2f us\n", key.c_str(), bs, ms * 1e3f);
            if (ms < best_ms) {
                best_ms = ms;
                best = bs;
            }
        }
    } catch (...) {
        g_prof_on.store(was_on);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        throw;
    }
    g_prof_on.store(was_on);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    if (!forced) tune_cache_store(key, best);
    return best;
}

// ------------------------------------------------------------------- memory
void* dev_alloc(Lattice* lat, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(LQ_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    if (lat) lat->bytes += bytes;
    return p;
}

void dev_free(Lattice* lat, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    if (lat) lat->bytes -= bytes;
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

static size_t rhs_bytes_of(int kind, int prec, int vh) {
    int nr = kind == LQ_WILSON_FIELD ? 24 : 6;
    return align256((size_t)nr * prec_bytes(prec) * vh);
}

size_t field_bytes(int kind, int prec, int nrhs, int vh) {
    size_t b = rhs_bytes_of(kind, prec, vh) * nrhs;
    if (prec == LQ_F16) b += align256((size_t)vh * 4 * nrhs);
    return b;
}

Field field_alloc(int kind, int prec, int nrhs, int vh) {
    Field f;
    f.kind = kind;
    f.prec = prec;
    f.nrhs = nrhs;
    f.vh = vh;
    f.rhs_bytes = rhs_bytes_of(kind, prec, vh);
    f.data = dev_alloc(nullptr, field_bytes(kind, prec, nrhs, vh));
    if (prec == LQ_F16) f.norm = (float*)((char*)f.data + f.rhs_bytes * nrhs);
    return f;
}

// ---------------------------------------------------------- workspace cache
void* ws_get(Lattice& lat, size_t bytes, bool host, cudaStream_t st) {
    bytes = bytes ? bytes : 16;
    {
        std::lock_guard<std::mutex> lk(lat.mu);
        // best fit among the idle buffers of the same kind, wasting at most a quarter
        int best = -1;
        for (size_t i = 0; i < lat.ws.size(); i++) {
            const auto& b = lat.ws[i];
            if (b.busy || b.host != host || b.bytes < bytes || b.bytes > bytes + bytes / 4) continue;
            if (best < 0 || b.bytes < lat.ws[best].bytes) best = (int)i;
        }
        if (best >= 0) {
            auto& b = lat.ws[best];
            b.busy = true;
            if (host) {
                // the host reads and writes it directly: the last user's copies must be done
                if (b.ev) LQ_CUDA(cudaEventSynchronize(b.ev));
            } else if (b.ev && b.st != st) {
                LQ_CUDA(cudaStreamWaitEvent(st, b.ev, 0));
            }
            return b.p;
        }
    }
    Lattice::WsBlock b;
    b.bytes = bytes;
    b.host = host;
    b.busy = true;
    cudaError_t e = host ? cudaMallocHost(&b.p, bytes) : cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        // idle buffers of other sizes may be what is in the way
        ws_release(lat);
        e = host ? cudaMallocHost(&b.p, bytes) : cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(LQ_ENOMEM, std::string("workspace allocation of ") + std::to_string(bytes) +
                                " bytes failed: " + cudaGetErrorString(e));
        }
    }
    LQ_CUDA(cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming));
    std::lock_guard<std::mutex> lk(lat.mu);
    lat.ws.push_back(b);
    return b.p;
}

static void ws_free_block(Lattice::WsBlock& b) {
    if (b.host) cudaFreeHost(b.p);
    else cudaFree(b.p);
    if (b.ev) cudaEventDestroy(b.ev);
    b.p = nullptr;
}

void ws_put(Lattice& lat, void* p, cudaStream_t st) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(lat.mu);
    for (size_t i = 0; i < lat.ws.size(); i++) {
        auto& b = lat.ws[i];
        if (b.p != p) continue;
        if (!lat.ws_keep) {
            ws_free_block(b);
            lat.ws.erase(lat.ws.begin() + i);
            return;
        }
        cudaEventRecord(b.ev, st);
        b.st = st;
        b.busy = false;
        return;
    }
}

size_t ws_release(Lattice& lat) {
    std::lock_guard<std::mutex> lk(lat.mu);
    size_t freed = 0;
    std::vector<Lattice::WsBlock> keep;
    for (auto& b : lat.ws) {
        if (b.busy) {
            keep.push_back(b);
            continue;
        }
        if (!b.host) freed += b.bytes;
        ws_free_block(b);
    }
    lat.ws.swap(keep);
    return freed;
}

size_t ws_idle_bytes(Lattice& lat) {
    std::lock_guard<std::mutex> lk(lat.mu);
    size_t n = 0;
    for (auto& b : lat.ws)
        if (!b.busy && !b.host) n += b.bytes;
    return n;
}

Field ws_field(Lattice& lat, int kind, int prec, int nrhs, cudaStream_t st) {
    Field f;
    f.kind = kind;
    f.prec = prec;
    f.nrhs = nrhs;
    f.vh = lat.vh;
    f.rhs_bytes = rhs_bytes_of(kind, prec, lat.vh);
    f.data = ws_get(lat, field_bytes(kind, prec, nrhs, lat.vh), false, st);
    if (prec == LQ_F16) f.norm = (float*)((char*)f.data + f.rhs_bytes * nrhs);
    return f;
}

void field_free(Field& f) {
    if (f.data) cudaFree(f.data);
    f.data = nullptr;
    f.norm = nullptr;
}

}  // namespace lq

// ------------------------------------------------------------- C ABI parts
using namespace lq;

extern "C" const char* lq_last_error(void) { return g_last_error.c_str(); }

extern "C" int lq_profile_enable(int on) {
    g_prof_on.store(on != 0);
    return LQ_OK;
}

extern "C" int lq_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) g_prof_free.push_back({r.a, r.b});
    g_prof.clear();
    g_prof_done.clear();
    g_launches.store(0);
    return LQ_OK;
}

extern "C" int lq_profile_query(const char* name, int64_t* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int64_t n = 0;
    double t = 0.0;
    for (auto& r : g_prof) {
        if (name && *name && r.name.find(name) == std::string::npos) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            set_last_error("lq_profile_query: event synchronisation failed");
            return LQ_ECUDA;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            t += ms;
            n++;
        }
    }
    for (auto& r : g_prof_done) {
        if (name && *name && r.first.find(name) == std::string::npos) continue;
        t += r.second;
        n++;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = t;
    return LQ_OK;
}

extern "C" int64_t lq_launch_count(void) { return g_launches.load(); }

extern "C" int lq_tune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    return LQ_OK;
}

extern "C" int lq_tune_force(int code) {
    if (code < 0) return LQ_EINVAL;
    g_tune_force.store(code);
    return LQ_OK;
}
