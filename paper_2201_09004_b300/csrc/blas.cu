// blas.cu -- Krylov vector operations on even-odd fields: updates with device
// or host scalars, precision conversion, and reductions. Reductions are
// deterministic and carried in double-float arithmetic (about 2^-44 relative
// per step, on the FP32 pipes): each thread sums its sites in a fixed order,
// blocks reduce by warp shuffles, and one block per right-hand side adds the
// per-block partials in a fixed order.
#include <type_traits>

#include "runtime.h"

namespace lq {

// arithmetic type of an operation between two storage precisions: FP64 if
// either side is FP64, else double-float if either side is double-float, else FP32
template <int PA, int PB> struct MathT {
    typedef typename std::conditional<PA == P64 || PB == P64, double,
            typename std::conditional<PA == PDF || PB == PDF, df, float>::type>::type T;
};

struct HostScalars {
    double a[64];
    double b[64];
};

#define SITE_LOOP(vh) for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < (vh); s += gridDim.x * blockDim.x)

template <int P, int NR>
__global__ void norm2_kernel(FieldV x, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    df acc(0.f);
    SITE_LOOP(x.vh) {
        T v[NR];
        fload<P, NR, T>(x, k, s, v);
        T t = (T)0;
#pragma unroll
        for (int q = 0; q < NR; q++) t = fma(v[q], v[q], t);
        acc = acc + df_of(t);
    }
    df r = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = r;
    fin_tail(part, gridDim.x, gridDim.y, fin);
}

template <int PD, int PS, int NR>
__global__ void copy_kernel(FieldV d, FieldV src) {
    typedef typename MathT<PD, PS>::T T;
    const int k = blockIdx.y;
    SITE_LOOP(d.vh) {
        T v[NR];
        fload<PS, NR, T>(src, k, s, v);
        fstore<PD, NR, T>(d, k, s, v);
    }
}

template <int P, int NR>
__global__ void zero_kernel(FieldV d) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    SITE_LOOP(d.vh) {
        T v[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) v[q] = (T)0;
        fstore<P, NR, T>(d, k, s, v);
    }
}

// y += a_k x  (host scalars)
template <int PY, int PX, int NR>
__global__ void axpy_h_kernel(FieldV y, FieldV x, HostScalars h) {
    typedef typename MathT<PY, PX>::T T;
    const int k = blockIdx.y;
    const T a = (T)h.a[k];
    SITE_LOOP(y.vh) {
        T vy[NR], vx[NR];
        fload<PY, NR, T>(y, k, s, vy);
        fload<PX, NR, T>(x, k, s, vx);
#pragma unroll
        for (int q = 0; q < NR; q++) vy[q] = fma(a, vx[q], vy[q]);
        fstore<PY, NR, T>(y, k, s, vy);
    }
}

// y = a_k x + b_k y, optional partial |y|^2 (host scalars)
template <int P, int NR>
__global__ void axpby_h_kernel(FieldV y, FieldV x, HostScalars h, df* part) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const T a = (T)h.a[k], b = (T)h.b[k];
    df acc(0.f);
    SITE_LOOP(y.vh) {
        T vy[NR], vx[NR];
        fload<P, NR, T>(y, k, s, vy);
        fload<P, NR, T>(x, k, s, vx);
        T t = (T)0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            vy[q] = fma(b, vy[q], a * vx[q]);
            t = fma(vy[q], vy[q], t);
        }
        acc = acc + df_of(t);
        fstore<P, NR, T>(y, k, s, vy);
    }
    if (part) {
        df r = block_sum_df(acc);
        if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = r;
    }
}

// s = b - q, partial |s|^2
template <int P, int NR>
__global__ void xmy_norm_kernel(FieldV sf, FieldV b, FieldV qf, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    df acc(0.f);
    SITE_LOOP(sf.vh) {
        T vb[NR], vq[NR];
        fload<P, NR, T>(b, k, s, vb);
        fload<P, NR, T>(qf, k, s, vq);
        T t = (T)0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            vb[q] -= vq[q];
            t = fma(vb[q], vb[q], t);
        }
        acc = acc + df_of(t);
        fstore<P, NR, T>(sf, k, s, vb);
    }
    df r = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = r;
    fin_tail(part, gridDim.x, gridDim.y, fin);
}

// x += alpha p; s -= alpha q; partial |s|^2; alpha_k = sc[k*SC_N + SC_ALPHA]
template <int PX, int P, int NR>
__global__ void cg_xs_kernel(FieldV x, FieldV p, FieldV sf, FieldV qf, const double* sc, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    typedef typename MathT<PX, P>::T TX;
    const int k = blockIdx.y;
    const double al = sc[(size_t)k * SC_N + SC_ALPHA];
    const T a = (T)al;
    const TX ax = (TX)al;
    df acc(0.f);
    SITE_LOOP(x.vh) {
        T vp[NR], vs[NR], vq[NR];
        TX vx[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<P, NR, T>(sf, k, s, vs);
        fload<P, NR, T>(qf, k, s, vq);
        fload<PX, NR, TX>(x, k, s, vx);
        T t = (T)0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            vx[q] = fma(ax, (TX)vp[q], vx[q]);
            vs[q] = fma(-a, vq[q], vs[q]);
            t = fma(vs[q], vs[q], t);
        }
        acc = acc + df_of(t);
        fstore<PX, NR, TX>(x, k, s, vx);
        fstore<P, NR, T>(sf, k, s, vs);
    }
    df r = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = r;
    fin_tail(part, gridDim.x, gridDim.y, fin);
}

// p = r + beta p
template <int P, int NR>
__global__ void cg_p_kernel(FieldV p, FieldV r, const double* sc) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const T b = (T)sc[(size_t)k * SC_N + SC_BETA];
    SITE_LOOP(p.vh) {
        T vp[NR], vr[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<P, NR, T>(r, k, s, vr);
#pragma unroll
        for (int q = 0; q < NR; q++) vp[q] = fma(b, vp[q], vr[q]);
        fstore<P, NR, T>(p, k, s, vp);
    }
}

// sum the partials of right-hand side blockIdx.x (double-float, fixed order),
// then apply the scalar step in FP64
__global__ void finalize_kernel(const df* part, int nblocks, double* sc, int slot, int op) {
    const int k = blockIdx.x;
    const df* pk = part + (size_t)k * nblocks;
    df sum(0.f);
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) sum = sum + pk[i];
    sum = block_sum_df(sum);
    if (threadIdx.x == 0) fin_apply(sc + (size_t)k * SC_N, df_to_double(sum), slot, op);
}

// ---------------------------------------------------------------- launchers
static dim3 red_grid(int nrhs) { return dim3(RED_BLOCKS, nrhs); }
static dim3 upd_grid(int vh, int nrhs) {
    int b = (vh + RED_THREADS - 1) / RED_THREADS;
    int cap = num_sms() * 8;
    return dim3(b < cap ? b : cap, nrhs);
}

#define DISPATCH_P(prec, MACRO)                    \
    do {                                           \
        if ((prec) == LQ_F64) { MACRO(P64); }       \
        else if ((prec) == LQ_F32) { MACRO(P32); }  \
        else if ((prec) == LQ_F16) { MACRO(P16); }  \
        else { MACRO(PDF); }                        \
    } while (0)

#define BY_KIND(f, NAME, KERNEL, GRID, ...)                                                     \
    do {                                                                                        \
        if ((f).kind == LQ_WILSON_FIELD) launch(NAME, KERNEL(24), GRID, dim3(RED_THREADS), st, __VA_ARGS__); \
        else launch(NAME, KERNEL(6), GRID, dim3(RED_THREADS), st, __VA_ARGS__);                  \
    } while (0)

void blas_norm2(const Field& x, df* part, cudaStream_t st, const FinArgs& fin) {
#define K(NR) norm2_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(x, "blas_norm2", K, red_grid(x.nrhs), x.view(), part, fin); }
    DISPATCH_P(x.prec, L);
#undef L
#undef K
}

template <int PD>
static void copy_from(Field& d, const Field& s, cudaStream_t st) {
    dim3 g = upd_grid(d.vh, d.nrhs);
#define K(NR) copy_kernel<PD, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(d, "blas_copy", K, g, d.view(), s.view()); }
    DISPATCH_P(s.prec, L);
#undef L
#undef K
}

void blas_copy(Field& d, const Field& s, cudaStream_t st) {
    if (d.kind != s.kind || d.nrhs != s.nrhs) fail(LQ_EINVAL, "blas_copy: shape mismatch");
    if (d.prec == LQ_F64) copy_from<P64>(d, s, st);
    else if (d.prec == LQ_F32) copy_from<P32>(d, s, st);
    else if (d.prec == LQ_F16) copy_from<P16>(d, s, st);
    else copy_from<PDF>(d, s, st);
}

void blas_zero(Field& x, cudaStream_t st) {
    dim3 g = upd_grid(x.vh, x.nrhs);
#define K(NR) zero_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(x, "blas_zero", K, g, x.view()); }
    DISPATCH_P(x.prec, L);
#undef L
#undef K
}

static HostScalars hs(const double* a, const double* b, int n) {
    if (n > 64) fail(LQ_EINVAL, "more than 64 right-hand sides in one field");
    HostScalars h;
    for (int i = 0; i < 64; i++) {
        h.a[i] = (a && i < n) ? a[i] : 0.0;
        h.b[i] = (b && i < n) ? b[i] : 0.0;
    }
    return h;
}

template <int PY>
static void axpy_h_from(Field& y, const HostScalars& h, const Field& x, cudaStream_t st) {
    dim3 g = upd_grid(y.vh, y.nrhs);
#define K(NR) axpy_h_kernel<PY, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(y, "blas_axpy", K, g, y.view(), x.view(), h); }
    DISPATCH_P(x.prec, L);
#undef L
#undef K
}

void blas_axpy_h(Field& y, const double* a, const Field& x, cudaStream_t st) {
    if (y.kind != x.kind || y.nrhs != x.nrhs) fail(LQ_EINVAL, "blas_axpy: shape mismatch");
    HostScalars h = hs(a, nullptr, y.nrhs);
    if (y.prec == LQ_F64) axpy_h_from<P64>(y, h, x, st);
    else if (y.prec == LQ_F32) axpy_h_from<P32>(y, h, x, st);
    else if (y.prec == LQ_F16) axpy_h_from<P16>(y, h, x, st);
    else axpy_h_from<PDF>(y, h, x, st);
}

void blas_axpby_h(Field& y, const double* a, const Field& x, const double* b, df* part, cudaStream_t st) {
    if (y.prec != x.prec || y.kind != x.kind || y.nrhs != x.nrhs) fail(LQ_EINVAL, "blas_axpby: field mismatch");
    HostScalars h = hs(a, b, y.nrhs);
    dim3 g = part ? red_grid(y.nrhs) : upd_grid(y.vh, y.nrhs);
#define K(NR) axpby_h_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(y, "blas_axpby", K, g, y.view(), x.view(), h, part); }
    DISPATCH_P(y.prec, L);
#undef L
#undef K
}

void blas_xmy_norm(Field& s, const Field& b, const Field& q, df* part, cudaStream_t st, const FinArgs& fin) {
    if (s.prec != b.prec || s.prec != q.prec) fail(LQ_EINVAL, "blas_xmy_norm: precision mismatch");
#define K(NR) xmy_norm_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(s, "blas_xmy_norm", K, red_grid(s.nrhs), s.view(), b.view(), q.view(), part, fin); }
    DISPATCH_P(s.prec, L);
#undef L
#undef K
}

template <int PX>
static void cg_xs_from(Field& x, const Field& p, Field& s, const Field& q, const double* sc, df* part,
                       cudaStream_t st, const FinArgs& fin) {
#define K(NR) cg_xs_kernel<PX, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(x, "blas_cg_xs", K, red_grid(x.nrhs), x.view(), p.view(), s.view(), q.view(), sc, part, fin); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_cg_xs(Field& x, const Field& p, Field& s, const Field& q, const double* sc, df* part,
                cudaStream_t st, const FinArgs& fin) {
    if (p.prec != s.prec || p.prec != q.prec) fail(LQ_EINVAL, "blas_cg_xs: precision mismatch");
    if (x.prec == LQ_F64) cg_xs_from<P64>(x, p, s, q, sc, part, st, fin);
    else if (x.prec == LQ_F32) cg_xs_from<P32>(x, p, s, q, sc, part, st, fin);
    else if (x.prec == LQ_F16) cg_xs_from<P16>(x, p, s, q, sc, part, st, fin);
    else cg_xs_from<PDF>(x, p, s, q, sc, part, st, fin);
}

void blas_cg_p(Field& p, const Field& r, const double* sc, cudaStream_t st) {
    if (p.prec != r.prec) fail(LQ_EINVAL, "blas_cg_p: precision mismatch");
    dim3 g = upd_grid(p.vh, p.nrhs);
#define K(NR) cg_p_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(p, "blas_cg_p", K, g, p.view(), r.view(), sc); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_finalize(const df* part, int nblocks, int nrhs, double* sc, int slot, int op, cudaStream_t st) {
    launch("blas_finalize", finalize_kernel, dim3(nrhs), dim3(256), st, part, nblocks, sc, slot, op);
}

}  // namespace lq
