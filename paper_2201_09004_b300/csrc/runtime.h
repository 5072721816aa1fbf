// runtime.h -- host-side runtime of the library: error handling, kernel launch
// bookkeeping (launch counter, optional per-launch CUDA-event timing), the
// block-size autotuner, and the lattice / field objects behind the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lq.h"
#include "core.cuh"

namespace lq {

// bytes per real of a storage precision (lq_prec values)
inline int prec_bytes(int prec) { return prec == LQ_F32 ? 4 : (prec == LQ_F16 ? 2 : 8); }
inline bool valid_prec(int prec) { return prec >= LQ_F64 && prec <= LQ_F32X2; }

// ------------------------------------------------------------------ errors
struct Error {
    int code;
    std::string msg;
};
void set_last_error(const std::string& msg);
[[noreturn]] void fail(int code, const std::string& msg);

#define LQ_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            ::lq::fail(e_ == cudaErrorMemoryAllocation ? LQ_ENOMEM : LQ_ECUDA,               \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

// ----------------------------------------------------------------- launches
// Every kernel launch of the library goes through launch(): the launch counter
// is always kept; with profiling on, CUDA events bracket the launch on its
// stream (not while the stream is being captured into a graph).
int prof_begin(const char* name, cudaStream_t st);
void prof_end(int slot, cudaStream_t st);
void count_launch();
bool stream_capturing(cudaStream_t st);
// raise a kernel's dynamic shared-memory limit to at least `bytes` (once per size)
void opt_in_smem(const void* kernel, size_t bytes);

template <typename... KArgs, typename... Args>
inline void launch_smem(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                        cudaStream_t st, Args&&... args) {
    if (grid.x == 0 || grid.y == 0) return;
    if (smem > 48 * 1024) opt_in_smem((const void*)kernel, smem);
    int slot = prof_begin(name, st);
    kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(LQ_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    prof_end(slot, st);
    count_launch();
}

template <typename... KArgs, typename... Args>
inline void launch(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                   Args&&... args) {
    if (grid.x == 0 || grid.y == 0) return;
    int slot = prof_begin(name, st);
    kernel<<<grid, block, 0, st>>>(std::forward<Args>(args)...);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(LQ_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    prof_end(slot, st);
    count_launch();
}

// Launch with programmatic stream serialization: the kernel may be scheduled while the
// previous kernel of the stream is finishing, so it must begin with pdl_start()
// (core.cuh), which waits for that kernel's completion before any memory access.
// In a graph capture the dependency becomes a programmatic edge.
template <typename... KArgs, typename... Args>
inline void launch_pdl(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
    if (grid.x == 0 || grid.y == 0) return;
    if (smem > 48 * 1024) opt_in_smem((const void*)kernel, smem);
    int slot = prof_begin(name, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) fail(LQ_ECUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    prof_end(slot, st);
    count_launch();
}

// ------------------------------------------------------------- CUDA graphs
// A captured sequence of launches (solver iterations) replayed by one
// cudaGraphLaunch. If profiling is on while it is captured, every kernel is
// bracketed by event-record nodes; collect() adds the times of the last replay
// to the profile and must run after that replay has finished.
struct GraphProf {
    std::string name;
    cudaEvent_t a, b;
};
struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<GraphProf> prof;
    int64_t kernels = 0;       // kernel launches per replay
    bool uncollected = false;  // a replay whose profile is not yet collected
};
// false (nothing captured) where the stream cannot be captured
bool graph_capture_begin(cudaStream_t st);
// ends the capture; false (and the stream back to normal) if it failed
bool graph_capture_end(cudaStream_t st, Graph& g);
void graph_launch(Graph& g, cudaStream_t st);
void graph_collect(Graph& g);
void graph_destroy(Graph& g);

// Launch autotuner: the first call for a key times each candidate (a block
// size, or a code of the caller's for block size and kernel variant) on the real
// arguments (the launch must be idempotent) and caches the fastest; later calls
// reuse it. While a stream is capturing, an untuned key falls back to 128.
int tuned_block(const std::string& key, cudaStream_t st, const std::function<void(int)>& run,
                const std::vector<int>& candidates = {64, 128, 256});
int num_sms();

// ------------------------------------------------------------------- fields
// A spinor (24 reals/site) or staggered colour vector (6 reals/site) field of
// one parity with nrhs right-hand sides in one allocation.
struct Field {
    int kind = 0;  // LQ_WILSON_FIELD / LQ_STAGGERED_FIELD
    int prec = 0;
    int nrhs = 0;
    int vh = 0;
    void* data = nullptr;
    float* norm = nullptr;
    size_t rhs_bytes = 0;
    int nreals() const { return kind == LQ_WILSON_FIELD ? 24 : 6; }
    FieldV view() const { return FieldV{data, norm, vh, rhs_bytes}; }
    FieldV view_rhs(int k) const {
        return FieldV{(char*)data + (size_t)k * rhs_bytes, norm ? norm + (size_t)k * vh : nullptr, vh, rhs_bytes};
    }
    // non-owning view of right-hand sides [k0, k0 + n)
    Field sub(int k0, int n) const {
        Field f = *this;
        f.nrhs = n;
        f.data = (char*)data + (size_t)k0 * rhs_bytes;
        f.norm = norm ? norm + (size_t)k0 * vh : nullptr;
        return f;
    }
};
Field field_alloc(int kind, int prec, int nrhs, int vh);
void field_free(Field& f);
size_t field_bytes(int kind, int prec, int nrhs, int vh);

// ------------------------------------------------------------------ lattice
struct PackedGauge {
    void* data = nullptr;
    float scale = 1.f;
    size_t bytes = 0;
};

struct Lattice {
    int L[4];
    int bc_t;
    int V, vh;
    Geo geo;
    int device;
    double* canon[3] = {nullptr, nullptr, nullptr};  // canonical FP64 links per kind (device)
    float maxabs[3] = {1.f, 1.f, 1.f};               // max |re|,|im| per kind (FP16 scale)
    std::map<std::tuple<int, int, int>, PackedGauge> packed;  // (kind, prec, recon)
    bool has_clover = false;
    double c_sw = 0.0;
    void* clovC[4] = {nullptr, nullptr, nullptr, nullptr};  // clover C per precision, [2][72 reals][vh]
    float* clovC_norm = nullptr;                     // FP16 norms [2][vh]
    struct Ainv {
        void* data[4] = {nullptr, nullptr, nullptr, nullptr};  // per precision, built on first use
        float* norm = nullptr;
        int pins = 0;           // solves currently using this entry
        uint64_t last_use = 0;  // for least-recently-used eviction
    };
    std::map<std::tuple<double, double, double>, Ainv> ainv;  // (m, mu0, mu1) -> A^{-1}, at most kAinvCache unpinned
    uint64_t ainv_clock = 0;
    // Work buffers of the solvers (device fields, pinned host scalars), kept
    // between solves so that a solve allocates nothing once the lattice is warm.
    struct WsBlock {
        void* p = nullptr;
        size_t bytes = 0;
        bool host = false;
        bool busy = false;
        cudaEvent_t ev = nullptr;   // recorded on the last user's stream when returned
        cudaStream_t st = nullptr;  // that stream
    };
    std::vector<WsBlock> ws;
    bool ws_keep = true;  // false: a returned buffer is freed at once
    // solves issued on the legacy default stream run on this stream (created on
    // first use), which CUDA graphs can capture
    cudaStream_t own_stream = nullptr;
    // device-to-host copies of finished solutions run here, beside the solve's
    // remaining kernels (created on first use)
    cudaStream_t copy_stream = nullptr;
    size_t bytes = 0;                                // device bytes held
    std::mutex mu;  // guards the lazily filled caches when several streams share the lattice
};

GaugeV gauge_view(Lattice& lat, int kind, int prec, int recon);
// pointer to parity block of the clover (C, 72 reals) / inverse (144 reals)
const void* clover_block(Lattice& lat, int prec, int parity, const float** norm);
// mu0 / mu1: the twisted mass on chiral block 0 (spins 0, 1) / 1 (spins 2, 3)
const void* ainv_block(Lattice& lat, double m, double mu0, double mu1, int prec, int parity, const float** norm,
                       cudaStream_t st);
void free_clover(Lattice& lat);
// keep the clover inverse of (m, mu) resident while a solve runs
void pin_ainv(Lattice& lat, double m, double mu0, double mu1, bool pin);
enum { kAinvCache = 8 };

void* dev_alloc(Lattice* lat, size_t bytes);
void dev_free(Lattice* lat, void* p, size_t bytes);

// workspace cache of the lattice: a buffer of at least `bytes` (device, or
// pinned host), ordered after the previous user's work when that ran on
// another stream; put() returns it (the caller's work on `st` may still run).
void* ws_get(Lattice& lat, size_t bytes, bool host, cudaStream_t st);
void ws_put(Lattice& lat, void* p, cudaStream_t st);
size_t ws_release(Lattice& lat);           // frees the idle buffers; returns the device bytes freed
size_t ws_idle_bytes(Lattice& lat);        // device bytes held by idle buffers
Field ws_field(Lattice& lat, int kind, int prec, int nrhs, cudaStream_t st);

// ------------------------------------------------------------ pack / unpack
void pack_gauge(Lattice& lat, int kind, int prec, int recon, PackedGauge& out, cudaStream_t st);
// canonical FP64 (device) <-> field rhs k of parity p
void import_field(const Lattice& lat, Field& f, int k, int parity, const double* canon_dev, cudaStream_t st);
void export_field(const Lattice& lat, const Field& f, int k, int parity, double* canon_dev, cudaStream_t st);
void gauge_maxabs(const double* canon, int V, float* out, cudaStream_t st);

// ------------------------------------------------------------------ clover
void build_clover(Lattice& lat, double c_sw, cudaStream_t st);
void load_clover_canonical(Lattice& lat, const double* canon_dev, cudaStream_t st);
void build_ainv(Lattice& lat, double m, double mu0, double mu1, int prec, Lattice::Ainv& out, cudaStream_t st);

// ------------------------------------------------------------------ dslash
struct OpDesc {
    int action;
    double m, mu, c_naik;
    int prec;
    int recon;       // thin (Wilson) / long (HISQ) link compression
    int gamma5 = 0;  // Wilson: multiply every result by g5 (the hermitian g5 D_w)
    int twist = LQ_TWIST_GAMMA5;  // Wilson: i mu g5 or the scalar i mu
};

// twisted mass on chiral block 1 (spins 2, 3): -mu for i mu g5, +mu for the scalar twist
inline double mu_block1(const OpDesc& d) { return d.twist == LQ_TWIST_SCALAR ? d.mu : -d.mu; }

// out = epilogue(D in) for output parity; `y` used by EPI_XPAY (same parity as out).
// norm_out: optional per-block partials of |out|^2 (nrhs * blocks).
// Returns the number of thread blocks per right-hand side (the partial-sum stride).
// rb, lo (double-float EPI_XPAY only): out = rb - (A y - D in) instead, and its FP16 copy into lo.
int wilson_dslash(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, const Field& in,
                  Field& out, const Field* y, df* norm_out, cudaStream_t st, const FinArgs& fin = FinArgs(),
                  const Field* rb = nullptr, Field* lo = nullptr);
// ak (device, optional): per-rhs XPAY scale at ak[k * SC_N], replacing a
int hisq_dslash(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, double a, const Field& in,
                Field& out, const Field* y, df* norm_out, cudaStream_t st, const FinArgs& fin = FinArgs(),
                const double* ak = nullptr);
// the arguments of a Wilson operator launch (links, fields, clover or A^{-1} block)
struct WilsonArgs;
WilsonArgs wilson_args(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, const Field& in, Field& out,
                       const Field* y, cudaStream_t st);
// the inner iterations of the mixed CGNR in one persistent cooperative kernel (persistent.cu):
// FP16 sloppy operator with R12 links and clover, one right-hand side
bool persistent_cg_supported(const Lattice& lat, const OpDesc& op, int nrhs);
int persistent_cg_blocks(const Lattice& lat);
// up to iters CG iterations on x (FP32), p, s, q, r (FP16, even), t (FP16, odd), stopping
// after the one whose |s|^2 falls below stop2; sc: the scalar block (SC_ITERS counts the
// iterations done); part: 2 * persistent_cg_blocks() partials; bar: 2 zeroed counters
void persistent_cg_run(Lattice& lat, const OpDesc& op, Field& x, Field& p, Field& s, Field& q, Field& r, Field& t,
                       double* sc, df* part, unsigned* bar, int iters, double stop2, cudaStream_t st);
// site-local out = A_pp^{-1} in (Wilson twisted mass / clover), parity of both fields
void wilson_ainv_site(Lattice& lat, const OpDesc& op, int parity, int dagger, const Field& in, Field& out,
                      cudaStream_t st);

// ------------------------------------------------------------------- blas
// All BLAS kernels work on whole fields of one parity, per right-hand side.
// Reductions write per-block partials to `part`, then finalize into dev scalars.
enum { RED_BLOCKS = 148 * 4, RED_THREADS = 256 };
enum { GCR_MAX = 16, GCR_DEFAULT = 12 };  // directions kept by the GCR solver before a restart
void blas_norm2(const Field& x, df* part, cudaStream_t st, const FinArgs& fin = FinArgs());          // part[k*RED_BLOCKS + b]
void blas_copy(Field& dst, const Field& src, cudaStream_t st);           // with precision conversion
void blas_zero(Field& x, cudaStream_t st);
void blas_axpy_h(Field& y, const double* a_host, const Field& x, cudaStream_t st);  // y += a_k x (host scalars)
void blas_axpy_h_zero(Field& y, const double* a_host, Field& x, cudaStream_t st);  // y += a_k x, then x = 0
// the vector updates of a multi-shift CG iteration in one pass (at most LQ_MS_MAXS shifts and
// LQ_MS_MAXK right-hand sides; coefficients [i * nrhs + k]): y_i += a p_i, p_i = z r + b p_i,
// per-block partials of |p_0|^2 in part (RED_BLOCKS per rhs)
#define LQ_MS_MAXS 8
#define LQ_MS_MAXK 8
void blas_ms_update(std::vector<Field>& y, std::vector<Field>& p, const Field& r, const double* a, const double* z,
                    const double* b, df* part, cudaStream_t st);
// y = a_k x + b_k y per right-hand side k (host scalars), optional partial |y|^2
void blas_axpby_h(Field& y, const double* a, const Field& x, const double* b, df* part, cudaStream_t st);
// s = b - q, with partial |s|^2
void blas_xmy_norm(Field& s, const Field& b, const Field& q, df* part, cudaStream_t st,
                   const FinArgs& fin = FinArgs());
// BiCGStab vector steps (complex device scalars in the solver scalar block, see core.cuh):
// (a, b) -> partials (2 per block), s = r - alpha v in place, (t, s) and |t|^2 (3),
// x += alpha p + omega s with r = s - omega t and |r|^2, (r0, r) (3), p = r + beta (p - omega v),
// |r|^2 and (r0, r) (3). Reductions are finalised by the last block (fin.sc non-null).
void blas_bicg_cdot(const Field& a, const Field& b, df* part, cudaStream_t st, const FinArgs& fin);
void blas_bicg_s(Field& r, const Field& v, const double* sc, cudaStream_t st);
void blas_bicg_tdot(const Field& t, const Field& s, df* part, cudaStream_t st, const FinArgs& fin);
void blas_bicg_xr(Field& x, const Field& p, Field& r, const Field& t, const Field& r0, const double* sc, df* part,
                  cudaStream_t st, const FinArgs& fin);
void blas_bicg_p(Field& p, const Field& r, const Field& v, const double* sc, cudaStream_t st);
void blas_bicg_rho(const Field& r, const Field& r0, df* part, cudaStream_t st, const FinArgs& fin);
// out = a0 v + a1 t + a2 w - out (sub_old), or without the last term; per element, all rhs
void blas_lincomb4(Field& out, double a0, const Field& v, double a1, const Field& t, double a2, const Field& w,
                   cudaStream_t st, bool sub_old = true);
// out = g5 in (Wilson fields); y += (a_re_k + i a_im_k) x per rhs (host scalars)
void blas_gamma5(Field& out, const Field& in, cudaStream_t st);
void blas_caxpy_h(Field& y, const double* a_re, const double* a_im, const Field& x, cudaStream_t st);
// The CG vector step (alpha_k = sc[k*SC_N + SC_ALPHA], beta_k = sc[k*SC_N + SC_BETA]) in two
// kernels: s -= alpha q with partial |s|^2, and later x += alpha p, p = r + beta p (one pass
// over p for both)
void blas_cg_s(Field& s, const Field& q, const double* sc, df* part, cudaStream_t st, const FinArgs& fin);
void blas_cg_xp(Field& x, Field& p, const Field& r, const double* sc, cudaStream_t st);
// the same with partial |p|^2 of the new p
void blas_cg_xp_norm(Field& x, Field& p, const Field& r, const double* sc, df* part, cudaStream_t st,
                     const FinArgs& fin);

// GCR and Gram-Schmidt steps. Partials of <v_i, w> (i < nv, fields listed in device
// memory) at part[((k * nv + i) * 2 + re/im) * RED_BLOCKS + block]; q_j -= sum_{i<j} c_i q_i
// and p_j -= sum_{i<j} c_i p_i (ps_dev null: q only) with c_i = coef[(k * cstride + i) * 2 +
// re/im] (device); x += a_k p, r -= a_k q with partial |r|^2 at part[k * RED_BLOCKS + block]
void blas_cdot_multi(const FieldV* vs_dev, int nv, const Field& w, df* part, cudaStream_t st);
void blas_gcr_orth(const FieldV* qs_dev, const FieldV* ps_dev, int j, const double* coef_dev, int cstride,
                   const Field& like, cudaStream_t st);
void blas_gcr_xr(Field& x, const Field& p, Field& r, const Field& q, const double* alpha_dev, df* part,
                 cudaStream_t st);

// sum part[k*nblocks ...] (compensated, fixed order) into sc[k*SC_N + slot], or apply `op`
void blas_finalize(const df* part, int nblocks, int nrhs, double* sc, int slot, int op, cudaStream_t st);

// ----------------------------------------------------------------- solvers
// Schur operators on resident fields (see solver.cu)
int schur_wilson(Lattice& lat, const OpDesc& op, int dagger, const Field& in, Field& out, Field& tmp, df* part,
                 cudaStream_t st, const FinArgs& fin = FinArgs());
// sigma_dev (device, optional): per-rhs shift at sigma_dev[k * SC_N], replacing sigma
int schur_hisq(Lattice& lat, const OpDesc& op, double sigma, const Field& in, Field& out, Field& t, df* part_t,
               cudaStream_t st, const FinArgs& fin = FinArgs(), const double* sigma_dev = nullptr);
// overlap building blocks (overlap.cu): Chebyshev coefficients of 1/sqrt(y) on
// [eps^2, 1] meeting the sign deviation delta; g5 D_w(-rho) and eps(g5 D_w(-rho))
// on full-lattice vectors (fields of 2 rhs: even sites, odd sites)
void sign_coefficients(double eps, double delta, int max_order, std::vector<double>& c, double& dev);
void hw_apply_full(Lattice& lat, double rho, const Field& in, Field& out, cudaStream_t st);
void sign_apply(Lattice& lat, double rho, double lmax, double eps, const std::vector<double>& c, const Field& v,
                Field& out, cudaStream_t st);
// low modes of H_w (eigen.cu): nev eigenvalues (ascending |lambda|) and double-float
// full-lattice eigenvectors in fields from the workspace cache (the caller returns them)
void hw_eigensolve(Lattice& lat, double rho, const lq_eig_params& p, std::vector<double>& evals,
                   std::vector<Field>& evecs, lq_eig_info& info, cudaStream_t st);
// eps(H_w) v with the eigenvectors projected out of the polynomial's argument (double-float fields)
void sign_apply_deflated(Lattice& lat, double rho, double lmax, double eps, const std::vector<double>& c,
                         const std::vector<double>& evals, const std::vector<Field>& evecs, const Field& v, Field& out,
                         cudaStream_t st);
// estimated device bytes of a solve's work fields
size_t solve_workspace_bytes(const Lattice& lat, const lq_op_params& op, const lq_solve_params& sp, int nrhs);
// Called from the solve's host thread once solution x[idx] is final in device
// memory: everything that writes it has been enqueued on st, and nothing enqueued
// later on st touches it. The caller may read it from another stream ordered
// after an event recorded on st.
using SolutionReady = std::function<void(int idx, cudaStream_t st)>;
// x0 (optional, device canonical): initial guesses whose even sites start the even-odd CGNR
int solve_wilson(Lattice& lat, const lq_op_params& op, const lq_solve_params& sp, int nrhs, const double* const* b,
                 double* const* x, lq_solve_info* info, cudaStream_t st, const double* const* x0 = nullptr,
                 const SolutionReady* ready = nullptr);
int solve_wilson_multishift(Lattice& lat, const lq_op_params& op, const lq_solve_params& sp, int nrhs,
                            const double* const* b, double* const* x, lq_solve_info* info, cudaStream_t st,
                            const SolutionReady* ready = nullptr);
int solve_hisq(Lattice& lat, const lq_op_params& op, const lq_solve_params& sp, int nrhs, const double* const* b,
               double* const* x, lq_solve_info* info, cudaStream_t st, const SolutionReady* ready = nullptr);

}  // namespace lq

// the opaque handle of include/lq.h
struct lq_lattice_s {
    lq::Lattice lat;
};
