// noalloc.cu -- lq_dslash_apply_noalloc: the hopping term of lq_dslash_apply for
// callers that must not allocate device memory.
//
// lq_dslash_apply packs its canonical input into the library's even-odd layout
// and unpacks the result through two temporary device fields that it
// allocates per call. Some callers cannot allow that: a host application whose
// memory pool owns the whole GPU and forbids other allocators, code running
// under a fixed device-memory budget that must not fragment, or a real-time
// loop where a cudaMalloc/cudaFree pair (an implicit device synchronisation)
// is not acceptable. This variant keeps those two temporary fields in one
// fixed scratch array compiled into the library instead, and allocates nothing.
//
// The scratch array lives in device memory on every GPU that loads the
// library, until the process exits; its size caps the lattices this entry
// point accepts. Every call shares it: calls that may run at the same time on
// the GPU (different streams or threads) race on it, so the caller must order
// them. A call overwrites every scratch byte it reads, so nothing left by the
// previous call leaks into the next.
#include <mutex>

#include "hisq.cuh"
#include "runtime.h"

namespace lq {
namespace {

// maximum bytes of scratch: the packed input and output fields of one call
constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;

// In host code this name is only a stand-in for the device object: its device
// address comes from cudaGetSymbolAddress (below), once per device.
static __device__ __align__(256) unsigned char lq_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[256] = {nullptr};

// device address of the scratch array on the current device; the first call on
// a device looks it up (this is why the first call must not be inside a stream
// capture)
void* scratch_address() {
    int dev = 0;
    LQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) fail(LQ_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, lq_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(LQ_ECUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

// packed links of a kind already resident in the lattice, or nothing
bool packed_links(Lattice& lat, int kind, int prec, int recon, GaugeV* out) {
    std::lock_guard<std::mutex> lk(lat.mu);
    auto it = lat.packed.find(std::make_tuple(kind, prec, recon));
    if (it == lat.packed.end()) return false;
    *out = GaugeV{it->second.data, lat.vh, it->second.scale};
    return true;
}

template <int P, int NR, int R>
void run_noalloc(Lattice& lat, bool hisq, const GaugeV& g1, const GaugeV& g2, int parity, int dagger, double c_naik,
                 const double* in, double* out, Field& fi, const Field& fo, cudaStream_t st) {
    const int block = 128;
    dim3 grid((lat.vh + block - 1) / block);
    import_field(lat, fi, 0, 1 - parity, in, st);
    if (hisq) {
        HisqArgs a;
        a.g = lat.geo;
        a.fat = g1;
        a.lng = g2;
        a.in = fi.view();
        a.out = fo.view();
        a.y = fo.view();
        a.parity = parity;
        a.dagger = dagger;
        a.c_naik = c_naik;
        a.a = 0.0;
        a.nrhs = 1;
        a.norm_out = nullptr;
        launch("hisq_dslash_noalloc", hisq_dslash_kernel<P, R, EPI_HOP, 1>, grid, dim3(block), st, a);
    } else {
        WilsonArgs a;
        a.g = lat.geo;
        a.U = g1;
        a.in = fi.view();
        a.out = fo.view();
        a.y = fo.view();
        a.clov = nullptr;
        a.clov_norm = nullptr;
        a.parity = parity;
        a.dagger = dagger;
        a.has_clover = 0;
        a.m4 = 4.0;
        a.mu = 0.0;
        a.mu1 = 0.0;
        a.nrhs = 1;
        a.norm_out = nullptr;
        launch("wilson_dslash_noalloc", wilson_dslash_kernel<P, R, EPI_HOP, 1>, grid, dim3(block), st, a);
    }
    LQ_CUDA(cudaMemsetAsync(out, 0, (size_t)lat.V * NR * sizeof(double), st));
    export_field(lat, fo, 0, parity, out, st);
}

}  // namespace
}  // namespace lq

using namespace lq;

extern "C" int lq_dslash_apply_noalloc(lq_lattice h, const lq_op_params* op, int parity, int dagger, int prec,
                                       const double* in, double* out, void* stream) {
    try {
        if (!h || !op || !in || !out) fail(LQ_EINVAL, "null argument");
        if (op->action < LQ_WILSON_TM || op->action > LQ_HISQ) fail(LQ_EINVAL, "unknown action");
        if (prec < LQ_F64 || prec > LQ_F16) fail(LQ_EINVAL, "unknown precision");
        if (op->recon != 0 && op->recon != 8 && op->recon != 12 && op->recon != 18)
            fail(LQ_EINVAL, "recon must be 0, 8, 12 or 18");
        if (parity != 0 && parity != 1) fail(LQ_EINVAL, "parity must be 0 or 1");
        Lattice& lat = h->lat;
        const bool hisq = op->action == LQ_HISQ;
        const int kind = hisq ? LQ_STAGGERED_FIELD : LQ_WILSON_FIELD;
        const size_t per = field_bytes(kind, prec, 1, lat.vh);
        if (2 * per > kNoallocScratchBytes)
            fail(LQ_EINVAL, "lattice too large for lq_dslash_apply_noalloc: needs " + std::to_string(2 * per) +
                                " bytes of scratch, the maximum is " + std::to_string(kNoallocScratchBytes) +
                                " (use lq_dslash_apply)");
        const int recon = (prec == LQ_F64 || prec == LQ_F32X2) ? 18 : (op->recon == 0 ? 12 : op->recon);
        GaugeV g1{}, g2{};
        bool ok = hisq ? (packed_links(lat, LQ_FAT, prec, 18, &g1) && packed_links(lat, LQ_LONG, prec, recon, &g2))
                       : packed_links(lat, LQ_THIN, prec, recon, &g1);
        if (!ok)
            fail(LQ_EINVAL, "links are not packed in this precision yet; one lq_dslash_apply call with the same "
                            "action and precision packs them");
        char* base = (char*)scratch_address();
        // two fields of one right-hand side each, laid out as field_alloc would
        Field fi, fo;
        fi.kind = fo.kind = kind;
        fi.prec = fo.prec = prec;
        fi.nrhs = fo.nrhs = 1;
        fi.vh = fo.vh = lat.vh;
        const int nr = hisq ? 6 : 24;
        fi.rhs_bytes = fo.rhs_bytes = ((size_t)nr * (prec == LQ_F64 ? 8 : (prec == LQ_F32 ? 4 : 2)) * lat.vh + 255) & ~(size_t)255;
        fi.data = base;
        fo.data = base + per;
        fi.norm = prec == LQ_F16 ? (float*)(base + fi.rhs_bytes) : nullptr;
        fo.norm = prec == LQ_F16 ? (float*)(base + per + fo.rhs_bytes) : nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        const double cn = hisq ? op->c_naik : 0.0;
#define LQ_NOALLOC(P, R)                                                                              \
    (hisq ? run_noalloc<P, 6, R>(lat, true, g1, g2, parity, dagger, cn, in, out, fi, fo, st)          \
          : run_noalloc<P, 24, R>(lat, false, g1, g2, parity, dagger, cn, in, out, fi, fo, st))
        if (prec == LQ_F64) LQ_NOALLOC(P64, 18);
        else if (prec == LQ_F32 && recon == 8) LQ_NOALLOC(P32, 8);
        else if (prec == LQ_F32 && recon == 18) LQ_NOALLOC(P32, 18);
        else if (prec == LQ_F32) LQ_NOALLOC(P32, 12);
        else if (recon == 8) LQ_NOALLOC(P16, 8);
        else if (recon == 18) LQ_NOALLOC(P16, 18);
        else LQ_NOALLOC(P16, 12);
#undef LQ_NOALLOC
        LQ_CUDA(cudaStreamSynchronize(st));
        return LQ_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("unexpected internal error");
        return LQ_EINVAL;
    }
}
