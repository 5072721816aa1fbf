// pack.cu -- ingest: canonical FP64 (lexicographic, complex interleaved) to the
// library's even-odd chunked layouts in FP64 / FP32 / FP16, link compression,
// and the reverse for fields.
#include <string.h>

#include "runtime.h"

namespace lq {

__device__ __forceinline__ int lex_of(const Geo& g, const int c[4]) {
    return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// one thread per (site of parity p = blockIdx.y, direction mu = blockIdx.z).
// R = 8 stores u01, u02, u10, arg(u00)/pi * scale, arg(u20)/pi * scale and counts
// the links with |u01|^2 + |u02|^2 below 1e-12 in *singular: their lower 2x2
// block cannot be rebuilt from those eight reals.
template <int P, int R>
__global__ void pack_gauge_kernel(const double* canon, int V, Geo g, void* out, float scale, unsigned* singular) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y, mu = blockIdx.z;
    if (s >= g.vh) return;
    int c[4];
    cb_coords(g, s, p, c);
    const double* u = canon + ((size_t)mu * V + lex_of(g, c)) * 18;
    double v[R];
    if constexpr (R == 8) {
#pragma unroll
        for (int k = 0; k < 6; k++) v[k] = u[2 + k];  // u01, u02, u10
        const double kpi = 0.318309886183790671537767526745;  // 1/pi
        v[6] = atan2(u[1], u[0]) * kpi * scale;
        v[7] = atan2(u[13], u[12]) * kpi * scale;
        if (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3] < 1e-12) atomicAdd(singular, 1u);
    } else {
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = u[k];  // R = 12 keeps rows 0 and 1
    }
    typedef Layout<P, R> Lay;
    char* base = (char*)out + (size_t)(p * 4 + mu) * Lay::NC * g.vh * sizeof(typename Lay::C);
    store_reals<P, R, double>(base, g.vh, s, nullptr, scale, v);
}

template <int P, int R>
static void pack_gauge_t(Lattice& lat, const double* canon, void* out, float scale, cudaStream_t st,
                         unsigned* singular = nullptr) {
    dim3 grid((lat.vh + 127) / 128, 2, 4);
    launch("pack_gauge", pack_gauge_kernel<P, R>, grid, dim3(128), st, canon, lat.V, lat.geo, out, scale, singular);
}

// R = 8 for FP32 / FP16; fails (and frees the packed copy) on a field with a
// link whose |u00| is 1, such as the unit gauge field
static void pack_gauge_r8(Lattice& lat, const double* canon, int prec, PackedGauge& out, cudaStream_t st) {
    unsigned* d = nullptr;
    LQ_CUDA(cudaMalloc(&d, sizeof(unsigned)));
    LQ_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned), st));
    if (prec == LQ_F32) pack_gauge_t<P32, 8>(lat, canon, out.data, out.scale, st, d);
    else pack_gauge_t<P16, 8>(lat, canon, out.data, out.scale, st, d);
    unsigned h = 0;
    LQ_CUDA(cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    LQ_CUDA(cudaStreamSynchronize(st));
    cudaFree(d);
    if (h) {
        dev_free(&lat, out.data, out.bytes);
        out.data = nullptr;
        fail(LQ_EINVAL, "recon 8 cannot represent links with |U_00| = 1 (" + std::to_string(h) +
                            " such links, e.g. a unit gauge field); use recon 12");
    }
}

void pack_gauge(Lattice& lat, int kind, int prec, int recon, PackedGauge& out, cudaStream_t st) {
    const double* canon = lat.canon[kind];
    if (!canon) fail(LQ_EINVAL, "gauge field of this kind is not loaded");
    if (recon != 18 && recon != 12 && recon != 8) fail(LQ_EINVAL, "recon must be 18, 12 or 8");
    if (recon == 8 && prec != LQ_F32 && prec != LQ_F16) fail(LQ_EINVAL, "recon 8 is for LQ_F32 and LQ_F16 links");
    if (recon != 18 && kind == LQ_FAT) fail(LQ_EINVAL, "fat links are not in SU(3): recon 18 only");
    out.bytes = (size_t)2 * 4 * recon * prec_bytes(prec) * lat.vh;
    out.data = dev_alloc(&lat, out.bytes);
    out.scale = prec == LQ_F16 ? lat.maxabs[kind] : 1.f;
    if (recon == 8) {
        pack_gauge_r8(lat, canon, prec, out, st);
    } else if (prec == LQ_F64) {
        if (recon == 18) pack_gauge_t<P64, 18>(lat, canon, out.data, out.scale, st);
        else pack_gauge_t<P64, 12>(lat, canon, out.data, out.scale, st);
    } else if (prec == LQ_F32X2) {
        if (recon == 18) pack_gauge_t<PDF, 18>(lat, canon, out.data, out.scale, st);
        else pack_gauge_t<PDF, 12>(lat, canon, out.data, out.scale, st);
    } else if (prec == LQ_F32) {
        if (recon == 18) pack_gauge_t<P32, 18>(lat, canon, out.data, out.scale, st);
        else pack_gauge_t<P32, 12>(lat, canon, out.data, out.scale, st);
    } else {
        if (recon == 18) pack_gauge_t<P16, 18>(lat, canon, out.data, out.scale, st);
        else pack_gauge_t<P16, 12>(lat, canon, out.data, out.scale, st);
    }
}

GaugeV gauge_view(Lattice& lat, int kind, int prec, int recon) {
    std::lock_guard<std::mutex> lk(lat.mu);
    auto key = std::make_tuple(kind, prec, recon);
    auto it = lat.packed.find(key);
    if (it == lat.packed.end()) {
        PackedGauge pg;
        pack_gauge(lat, kind, prec, recon, pg, 0);
        LQ_CUDA(cudaStreamSynchronize(0));
        it = lat.packed.emplace(key, pg).first;
    }
    return GaugeV{it->second.data, lat.vh, it->second.scale};
}

// ------------------------------------------------------------------ maxabs
__global__ void maxabs_kernel(const double* a, size_t n, unsigned* out) {
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, (float)fabs(a[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

void gauge_maxabs(const double* canon, int V, float* out, cudaStream_t st) {
    unsigned* d = nullptr;
    LQ_CUDA(cudaMalloc(&d, sizeof(unsigned)));
    LQ_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned), st));
    launch("gauge_maxabs", maxabs_kernel, dim3(num_sms() * 4), dim3(256), st, canon, (size_t)V * 4 * 18, d);
    unsigned h = 0;
    LQ_CUDA(cudaMemcpyAsync(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    LQ_CUDA(cudaStreamSynchronize(st));
    cudaFree(d);
    float f;
    memcpy(&f, &h, sizeof(float));
    // round the scale up slightly so that the largest entry maps inside int16
    *out = f > 0.f ? f * (1.f + 1e-6f) : 1.f;
}

// ------------------------------------------------------------------ fields
template <int P, int NR>
__global__ void import_kernel(const double* canon, Geo g, int parity, FieldV f) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vh) return;
    int c[4];
    cb_coords(g, s, parity, c);
    const double* src = canon + (size_t)lex_of(g, c) * NR;
    double v[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) v[k] = src[k];
    fstore<P, NR, double>(f, 0, s, v);
}

template <int P, int NR>
__global__ void export_kernel(double* canon, Geo g, int parity, FieldV f) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.vh) return;
    int c[4];
    cb_coords(g, s, parity, c);
    double* dst = canon + (size_t)lex_of(g, c) * NR;
    double v[NR];
    fload<P, NR, double>(f, 0, s, v);
#pragma unroll
    for (int k = 0; k < NR; k++) dst[k] = v[k];
}

#define FIELD_DISPATCH(NAME, KERNEL, ...)                                                                  \
    do {                                                                                                   \
        dim3 grid_((lat.vh + 127) / 128);                                                                  \
        if (f.kind == LQ_WILSON_FIELD) {                                                                   \
            if (f.prec == LQ_F32X2) launch(NAME, KERNEL<PDF, 24>, grid_, dim3(128), st, __VA_ARGS__);      \
            else if (f.prec == LQ_F64) launch(NAME, KERNEL<P64, 24>, grid_, dim3(128), st, __VA_ARGS__);   \
            else if (f.prec == LQ_F32) launch(NAME, KERNEL<P32, 24>, grid_, dim3(128), st, __VA_ARGS__);   \
            else launch(NAME, KERNEL<P16, 24>, grid_, dim3(128), st, __VA_ARGS__);                         \
        } else {                                                                                           \
            if (f.prec == LQ_F32X2) launch(NAME, KERNEL<PDF, 6>, grid_, dim3(128), st, __VA_ARGS__);       \
            else if (f.prec == LQ_F64) launch(NAME, KERNEL<P64, 6>, grid_, dim3(128), st, __VA_ARGS__);    \
            else if (f.prec == LQ_F32) launch(NAME, KERNEL<P32, 6>, grid_, dim3(128), st, __VA_ARGS__);    \
            else launch(NAME, KERNEL<P16, 6>, grid_, dim3(128), st, __VA_ARGS__);                          \
        }                                                                                                  \
    } while (0)

void import_field(const Lattice& lat, Field& f, int k, int parity, const double* canon, cudaStream_t st) {
    FieldV v = f.view_rhs(k);
    FIELD_DISPATCH("import_field", import_kernel, canon, lat.geo, parity, v);
}

void export_field(const Lattice& lat, const Field& f, int k, int parity, double* canon, cudaStream_t st) {
    FieldV v = f.view_rhs(k);
    FIELD_DISPATCH("export_field", export_kernel, canon, lat.geo, parity, v);
}

}  // namespace lq
