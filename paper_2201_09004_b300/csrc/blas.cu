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

// y += a_k x  (host scalars); zero_x: then x = 0 (the reliable update's fold of the
// sloppy solution into the accumulated one)
template <int PY, int PX, int NR>
__global__ void axpy_h_kernel(FieldV y, FieldV x, HostScalars h, int zero_x) {
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
        if (zero_x) {
#pragma unroll
            for (int q = 0; q < NR; q++) vx[q] = (T)0;
            fstore<PX, NR, T>(x, k, s, vx);
        }
    }
}

// The vector updates of one multi-shift CG iteration in one pass, for shifts i < ns and
// right-hand side k (blockIdx.y): y_i += a_ik p_i, then p_i = z_ik r + b_ik p_i (both
// with the old p_i), and the per-block partial of |p_0|^2. Inactive pairs come with
// a = 0, z = 0, b = 1 (nothing changes).
struct MsUpdate {
    FieldV y[LQ_MS_MAXS], p[LQ_MS_MAXS];
    FieldV r;
    int ns;
    double a[LQ_MS_MAXS * LQ_MS_MAXK], z[LQ_MS_MAXS * LQ_MS_MAXK], b[LQ_MS_MAXS * LQ_MS_MAXK];
};

template <int P, int NR>
__global__ void ms_update_kernel(MsUpdate m, df* part) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    df acc(0.f);
    SITE_LOOP(m.r.vh) {
        T vr[NR];
        fload<P, NR, T>(m.r, k, s, vr);
#pragma unroll 1
        for (int i = 0; i < m.ns; i++) {
            const T a = (T)m.a[i * LQ_MS_MAXK + k], z = (T)m.z[i * LQ_MS_MAXK + k], b = (T)m.b[i * LQ_MS_MAXK + k];
            T vp[NR], vy[NR];
            fload<P, NR, T>(m.p[i], k, s, vp);
            fload<P, NR, T>(m.y[i], k, s, vy);
            T t = (T)0;
#pragma unroll
            for (int q = 0; q < NR; q++) {
                vy[q] = fma(a, vp[q], vy[q]);
                vp[q] = fma(b, vp[q], z * vr[q]);
                t = fma(vp[q], vp[q], t);
            }
            if (i == 0) acc = acc + df_of(t);
            fstore<P, NR, T>(m.y[i], k, s, vy);
            fstore<P, NR, T>(m.p[i], k, s, vp);
        }
    }
    df r = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = r;
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

// s -= alpha q; partial |s|^2 (the x update of the same step goes with the next p update)
template <int P, int NR>
__global__ void cg_s_kernel(FieldV sf, FieldV qf, const double* sc, df* part, FinArgs fin) {
    pdl_start();
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const T a = (T)sc[(size_t)k * SC_N + SC_ALPHA];
    df acc(0.f);
    SITE_LOOP(sf.vh) {
        T vs[NR], vq[NR];
        fload<P, NR, T>(sf, k, s, vs);
        fload<P, NR, T>(qf, k, s, vq);
        T t = (T)0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            vs[q] = fma(-a, vq[q], vs[q]);
            t = fma(vs[q], vs[q], t);
        }
        acc = acc + df_of(t);
        fstore<P, NR, T>(sf, k, s, vs);
    }
    df r = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = r;
    fin_tail(part, gridDim.x, gridDim.y, fin);
}

// x += alpha p, then p = r + beta p: one read of p for both updates
template <int PX, int P, int NR>
__global__ void cg_xp_kernel(FieldV x, FieldV p, FieldV r, const double* sc) {
    pdl_start();
    typedef typename RealT<P>::T T;
    typedef typename MathT<PX, P>::T TX;
    const int k = blockIdx.y;
    const TX ax = (TX)sc[(size_t)k * SC_N + SC_ALPHA];
    const T b = (T)sc[(size_t)k * SC_N + SC_BETA];
    SITE_LOOP(p.vh) {
        T vp[NR], vr[NR];
        TX vx[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<PX, NR, TX>(x, k, s, vx);
        fload<P, NR, T>(r, k, s, vr);
#pragma unroll
        for (int q = 0; q < NR; q++) {
            vx[q] = fma(ax, (TX)vp[q], vx[q]);
            vp[q] = fma(b, vp[q], vr[q]);
        }
        fstore<PX, NR, TX>(x, k, s, vx);
        fstore<P, NR, T>(p, k, s, vp);
    }
}

// x += alpha p, then p = r + beta p with partial |p|^2
template <int PX, int P, int NR>
__global__ void cg_xp_norm_kernel(FieldV x, FieldV p, FieldV r, const double* sc, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    typedef typename MathT<PX, P>::T TX;
    const int k = blockIdx.y;
    const TX ax = (TX)sc[(size_t)k * SC_N + SC_ALPHA];
    const T b = (T)sc[(size_t)k * SC_N + SC_BETA];
    df acc(0.f);
    SITE_LOOP(p.vh) {
        T vp[NR], vr[NR];
        TX vx[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<PX, NR, TX>(x, k, s, vx);
        fload<P, NR, T>(r, k, s, vr);
        T t = (T)0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            vx[q] = fma(ax, (TX)vp[q], vx[q]);
            vp[q] = fma(b, vp[q], vr[q]);
            t = fma(vp[q], vp[q], t);
        }
        acc = acc + df_of(t);
        fstore<PX, NR, TX>(x, k, s, vx);
        fstore<P, NR, T>(p, k, s, vp);
    }
    df rr = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = rr;
    fin_tail(part, gridDim.x, gridDim.y, fin);
}

// sum the partials of right-hand side blockIdx.x (double-float, fixed order),
// then apply the scalar step in FP64
__global__ void finalize_kernel(const df* part, int nblocks, double* sc, int slot, int op) {
    pdl_start();
    const int k = blockIdx.x;
    const df* pk = part + (size_t)k * nblocks;
    df sum(0.f);
    // sixteen partials in flight per thread, added in the order of one at a time
    const int B = blockDim.x;
    for (int i0 = threadIdx.x; i0 < nblocks; i0 += 16 * B) {
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; j++)
            v[j] = i0 + j * B < nblocks ? __ldcg((const float2*)(pk + i0 + j * B)) : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 16; j++)
            if (i0 + j * B < nblocks) sum = sum + df(v[j].x, v[j].y);
    }
    sum = block_sum_df(sum);
    if (threadIdx.x == 0) fin_apply(sc + (size_t)k * SC_N, df_to_double(sum), slot, op);
}

// ------------------------------------------------------------- BiCGStab
// complex scalar (re, im) of rhs k from the solver scalar block
template <typename T>
__device__ __forceinline__ cx<T> sc_cx(const double* sc, int k, int slot) {
    return mk((T)sc[(size_t)k * SC_N + slot], (T)sc[(size_t)k * SC_N + slot + 1]);
}
template <typename T>
__device__ __forceinline__ cx<T> ld_c(const T* v, int j) { return mk(v[2 * j], v[2 * j + 1]); }

// write W block partials (thread 0) and finalise in the last block
template <int W>
__device__ __forceinline__ void partials_w(const df (&acc)[W], df* part, int k, const FinArgs& fin) {
#pragma unroll
    for (int w = 0; w < W; w++) {
        const df r = block_sum_df(acc[w]);
        if (threadIdx.x == 0) part[(size_t)(k * W + w) * gridDim.x + blockIdx.x] = r;
    }
    fin_tail_w<W>(part, gridDim.x, gridDim.y, fin);
}

// (a, b) = sum conj(a) b: W = 2 totals (re, im), then FIN_BICG_ALPHA
template <int P, int NR>
__global__ void cdot_kernel(FieldV a, FieldV b, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    df acc[2] = {df(0.f), df(0.f)};
    SITE_LOOP(a.vh) {
        T va[NR], vb[NR];
        fload<P, NR, T>(a, k, s, va);
        fload<P, NR, T>(b, k, s, vb);
        T re = (T)0, im = (T)0;
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            re = fma(va[2 * j], vb[2 * j], re);
            re = fma(va[2 * j + 1], vb[2 * j + 1], re);
            im = fma(va[2 * j], vb[2 * j + 1], im);
            im = fma(-va[2 * j + 1], vb[2 * j], im);
        }
        acc[0] = acc[0] + df_of(re);
        acc[1] = acc[1] + df_of(im);
    }
    partials_w<2>(acc, part, k, fin);
}

// s = r - alpha v (in place in r)
template <int P, int NR>
__global__ void bicg_s_kernel(FieldV r, FieldV v, const double* sc) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const cx<T> al = sc_cx<T>(sc, k, SC_AL_R);
    SITE_LOOP(r.vh) {
        T vr[NR], vv[NR];
        fload<P, NR, T>(r, k, s, vr);
        fload<P, NR, T>(v, k, s, vv);
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            const cx<T> o = ld_c(vr, j) - al * ld_c(vv, j);
            vr[2 * j] = o.r;
            vr[2 * j + 1] = o.i;
        }
        fstore<P, NR, T>(r, k, s, vr);
    }
}

// (t, s) and |t|^2: W = 3 totals, then FIN_BICG_OMEGA
template <int P, int NR>
__global__ void tdot_kernel(FieldV t, FieldV sf, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    df acc[3] = {df(0.f), df(0.f), df(0.f)};
    SITE_LOOP(t.vh) {
        T vt[NR], vs[NR];
        fload<P, NR, T>(t, k, s, vt);
        fload<P, NR, T>(sf, k, s, vs);
        T re = (T)0, im = (T)0, tt = (T)0;
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            re = fma(vt[2 * j], vs[2 * j], re);
            re = fma(vt[2 * j + 1], vs[2 * j + 1], re);
            im = fma(vt[2 * j], vs[2 * j + 1], im);
            im = fma(-vt[2 * j + 1], vs[2 * j], im);
            tt = fma(vt[2 * j], vt[2 * j], tt);
            tt = fma(vt[2 * j + 1], vt[2 * j + 1], tt);
        }
        acc[0] = acc[0] + df_of(re);
        acc[1] = acc[1] + df_of(im);
        acc[2] = acc[2] + df_of(tt);
    }
    partials_w<3>(acc, part, k, fin);
}

// x += alpha p + omega s; r = s - omega t (s held in r); |r|^2, (r0, r): W = 3, then FIN_BICG_BETA
template <int PX, int P, int NR>
__global__ void bicg_xr_kernel(FieldV x, FieldV p, FieldV r, FieldV t, FieldV r0, const double* sc, df* part,
                               FinArgs fin) {
    typedef typename RealT<P>::T T;
    typedef typename MathT<PX, P>::T TX;
    const int k = blockIdx.y;
    const cx<TX> al = sc_cx<TX>(sc, k, SC_AL_R), om = sc_cx<TX>(sc, k, SC_OM_R);
    const cx<T> omt = sc_cx<T>(sc, k, SC_OM_R);
    df acc[3] = {df(0.f), df(0.f), df(0.f)};
    SITE_LOOP(x.vh) {
        T vp[NR], vs[NR], vt[NR], v0[NR];
        TX vx[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<P, NR, T>(r, k, s, vs);
        fload<P, NR, T>(t, k, s, vt);
        fload<P, NR, T>(r0, k, s, v0);
        fload<PX, NR, TX>(x, k, s, vx);
        T rr = (T)0, re = (T)0, im = (T)0;
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            const cx<TX> pj = mk((TX)vp[2 * j], (TX)vp[2 * j + 1]), sj = mk((TX)vs[2 * j], (TX)vs[2 * j + 1]);
            const cx<TX> xn = ld_c(vx, j) + al * pj + om * sj;
            vx[2 * j] = xn.r;
            vx[2 * j + 1] = xn.i;
            const cx<T> rn = ld_c(vs, j) - omt * ld_c(vt, j);
            vs[2 * j] = rn.r;
            vs[2 * j + 1] = rn.i;
            rr = fma(rn.r, rn.r, rr);
            rr = fma(rn.i, rn.i, rr);
            re = fma(v0[2 * j], rn.r, re);
            re = fma(v0[2 * j + 1], rn.i, re);
            im = fma(v0[2 * j], rn.i, im);
            im = fma(-v0[2 * j + 1], rn.r, im);
        }
        acc[0] = acc[0] + df_of(rr);
        acc[1] = acc[1] + df_of(re);
        acc[2] = acc[2] + df_of(im);
        fstore<PX, NR, TX>(x, k, s, vx);
        fstore<P, NR, T>(r, k, s, vs);
    }
    partials_w<3>(acc, part, k, fin);
}

// p = r + beta (p - omega v)
template <int P, int NR>
__global__ void bicg_p_kernel(FieldV p, FieldV r, FieldV v, const double* sc) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const cx<T> be = sc_cx<T>(sc, k, SC_BE_R), om = sc_cx<T>(sc, k, SC_OM_R);
    SITE_LOOP(p.vh) {
        T vp[NR], vr[NR], vv[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<P, NR, T>(r, k, s, vr);
        fload<P, NR, T>(v, k, s, vv);
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            const cx<T> o = ld_c(vr, j) + be * (ld_c(vp, j) - om * ld_c(vv, j));
            vp[2 * j] = o.r;
            vp[2 * j + 1] = o.i;
        }
        fstore<P, NR, T>(p, k, s, vp);
    }
}

// |r|^2 and (r0, r): W = 3, then FIN_BICG_RHO
template <int P, int NR>
__global__ void rho_kernel(FieldV r, FieldV r0, df* part, FinArgs fin) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    df acc[3] = {df(0.f), df(0.f), df(0.f)};
    SITE_LOOP(r.vh) {
        T vr[NR], v0[NR];
        fload<P, NR, T>(r, k, s, vr);
        fload<P, NR, T>(r0, k, s, v0);
        T rr = (T)0, re = (T)0, im = (T)0;
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            rr = fma(vr[2 * j], vr[2 * j], rr);
            rr = fma(vr[2 * j + 1], vr[2 * j + 1], rr);
            re = fma(v0[2 * j], vr[2 * j], re);
            re = fma(v0[2 * j + 1], vr[2 * j + 1], re);
            im = fma(v0[2 * j], vr[2 * j + 1], im);
            im = fma(-v0[2 * j + 1], vr[2 * j], im);
        }
        acc[0] = acc[0] + df_of(rr);
        acc[1] = acc[1] + df_of(re);
        acc[2] = acc[2] + df_of(im);
    }
    partials_w<3>(acc, part, k, fin);
}

// out = a0 v + a1 t + a2 w - out_old (sub_old) or a0 v + a1 t + a2 w
template <int P, int NR>
__global__ void lincomb4_kernel(FieldV out, double a0, FieldV v, double a1, FieldV t, double a2, FieldV w, int sub_old) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const T c0 = (T)a0, c1 = (T)a1, c2 = (T)a2;
    SITE_LOOP(out.vh) {
        T vo[NR], vv[NR], vt[NR], vw[NR];
        fload<P, NR, T>(v, k, s, vv);
        fload<P, NR, T>(t, k, s, vt);
        fload<P, NR, T>(w, k, s, vw);
        if (sub_old) fload<P, NR, T>(out, k, s, vo);
#pragma unroll
        for (int q = 0; q < NR; q++) {
            T r = c0 * vv[q] + c1 * vt[q] + c2 * vw[q];
            vo[q] = sub_old ? r - vo[q] : r;
        }
        fstore<P, NR, T>(out, k, s, vo);
    }
}

// out = g5 in (Wilson fields: negate spins 2 and 3, the reals 12..23)
template <int P>
__global__ void gamma5_kernel(FieldV out, FieldV in) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    SITE_LOOP(out.vh) {
        T v[24];
        fload<P, 24, T>(in, k, s, v);
#pragma unroll
        for (int q = 12; q < 24; q++) v[q] = -v[q];
        fstore<P, 24, T>(out, k, s, v);
    }
}

// y += (a_k + i b_k) x per right-hand side k (host scalars)
template <int P, int NR>
__global__ void caxpy_h_kernel(FieldV y, FieldV x, HostScalars h) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const cx<T> c = mk((T)h.a[k], (T)h.b[k]);
    SITE_LOOP(y.vh) {
        T vy[NR], vx[NR];
        fload<P, NR, T>(y, k, s, vy);
        fload<P, NR, T>(x, k, s, vx);
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            const cx<T> o = mk(vy[2 * j], vy[2 * j + 1]) + c * mk(vx[2 * j], vx[2 * j + 1]);
            vy[2 * j] = o.r;
            vy[2 * j + 1] = o.i;
        }
        fstore<P, NR, T>(y, k, s, vy);
    }
}

// ------------------------------------------------------- GCR and Gram-Schmidt
// partial (re, im) of <v_i, w> = sum conj(v_i) w for i = blockIdx.z; the fields v_i
// are listed in device memory; part[((k * nv + i) * 2 + c) * gridDim.x + block]
template <int P, int NR>
__global__ void cdot_multi_kernel(const FieldV* vs, FieldV w, df* part) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y, i = blockIdx.z;
    const FieldV a = vs[i];
    df acc[2] = {df(0.f), df(0.f)};
    SITE_LOOP(w.vh) {
        T va[NR], vw[NR];
        fload<P, NR, T>(a, k, s, va);
        fload<P, NR, T>(w, k, s, vw);
        T re = (T)0, im = (T)0;
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            re = fma(va[2 * j], vw[2 * j], re);
            re = fma(va[2 * j + 1], vw[2 * j + 1], re);
            im = fma(va[2 * j], vw[2 * j + 1], im);
            im = fma(-va[2 * j + 1], vw[2 * j], im);
        }
        acc[0] = acc[0] + df_of(re);
        acc[1] = acc[1] + df_of(im);
    }
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const df r = block_sum_df(acc[c]);
        if (threadIdx.x == 0) part[((size_t)(k * gridDim.z + i) * 2 + c) * gridDim.x + blockIdx.x] = r;
    }
}

// q_j -= sum_{i<j} c_i q_i and p_j -= sum_{i<j} c_i p_i (ps may be null: q only),
// c_i = coef[(k * cstride + i) * 2 + {0, 1}]
template <int P, int NR>
__global__ void gcr_orth_kernel(const FieldV* qs, const FieldV* ps, int j, const double* coef, int cstride) {
    typedef typename RealT<P>::T T;
    const int k = blockIdx.y;
    const FieldV qj = qs[j];
    const FieldV pj = ps ? ps[j] : qj;
    SITE_LOOP(qj.vh) {
        T vq[NR], vp[NR];
        fload<P, NR, T>(qj, k, s, vq);
        if (ps) fload<P, NR, T>(pj, k, s, vp);
        for (int i = 0; i < j; i++) {
            const double* ci = coef + ((size_t)k * cstride + i) * 2;
            const cx<T> c = mk((T)__ldg(ci), (T)__ldg(ci + 1));
            T a[NR];
            fload<P, NR, T>(qs[i], k, s, a);
#pragma unroll
            for (int q = 0; q < NR / 2; q++) {
                const cx<T> o = ld_c(vq, q) - c * ld_c(a, q);
                vq[2 * q] = o.r;
                vq[2 * q + 1] = o.i;
            }
            if (!ps) continue;
            fload<P, NR, T>(ps[i], k, s, a);
#pragma unroll
            for (int q = 0; q < NR / 2; q++) {
                const cx<T> o = ld_c(vp, q) - c * ld_c(a, q);
                vp[2 * q] = o.r;
                vp[2 * q + 1] = o.i;
            }
        }
        fstore<P, NR, T>(qj, k, s, vq);
        if (ps) fstore<P, NR, T>(pj, k, s, vp);
    }
}

// x += a p, r -= a q, partial |r|^2 (part[k * gridDim.x + block]); a = alpha[2k] + i alpha[2k+1]
template <int PX, int P, int NR>
__global__ void gcr_xr_kernel(FieldV x, FieldV p, FieldV r, FieldV q, const double* alpha, df* part) {
    typedef typename RealT<P>::T T;
    typedef typename MathT<PX, P>::T TX;
    const int k = blockIdx.y;
    const cx<TX> ax = mk((TX)__ldg(alpha + 2 * k), (TX)__ldg(alpha + 2 * k + 1));
    const cx<T> a = mk((T)__ldg(alpha + 2 * k), (T)__ldg(alpha + 2 * k + 1));
    df acc(0.f);
    SITE_LOOP(x.vh) {
        T vp[NR], vr[NR], vq[NR];
        TX vx[NR];
        fload<P, NR, T>(p, k, s, vp);
        fload<P, NR, T>(r, k, s, vr);
        fload<P, NR, T>(q, k, s, vq);
        fload<PX, NR, TX>(x, k, s, vx);
        T rr = (T)0;
#pragma unroll
        for (int j = 0; j < NR / 2; j++) {
            const cx<TX> ox = mk(vx[2 * j], vx[2 * j + 1]) + ax * mk((TX)vp[2 * j], (TX)vp[2 * j + 1]);
            vx[2 * j] = ox.r;
            vx[2 * j + 1] = ox.i;
            const cx<T> orr = ld_c(vr, j) - a * ld_c(vq, j);
            vr[2 * j] = orr.r;
            vr[2 * j + 1] = orr.i;
            rr = fma(orr.r, orr.r, rr);
            rr = fma(orr.i, orr.i, rr);
        }
        fstore<PX, NR, TX>(x, k, s, vx);
        fstore<P, NR, T>(r, k, s, vr);
        acc = acc + df_of(rr);
    }
    const df t = block_sum_df(acc);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = t;
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

#define BY_KIND_PDL(f, NAME, KERNEL, GRID, ...)                                                                 \
    do {                                                                                                        \
        if ((f).kind == LQ_WILSON_FIELD) launch_pdl(NAME, KERNEL(24), GRID, dim3(RED_THREADS), 0, st, __VA_ARGS__); \
        else launch_pdl(NAME, KERNEL(6), GRID, dim3(RED_THREADS), 0, st, __VA_ARGS__);                          \
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
static void axpy_h_from(Field& y, const HostScalars& h, const Field& x, int zero_x, cudaStream_t st) {
    dim3 g = upd_grid(y.vh, y.nrhs);
#define K(NR) axpy_h_kernel<PY, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(y, "blas_axpy", K, g, y.view(), x.view(), h, zero_x); }
    DISPATCH_P(x.prec, L);
#undef L
#undef K
}

static void axpy_h_any(Field& y, const double* a, const Field& x, int zero_x, cudaStream_t st) {
    if (y.kind != x.kind || y.nrhs != x.nrhs) fail(LQ_EINVAL, "blas_axpy: shape mismatch");
    HostScalars h = hs(a, nullptr, y.nrhs);
    if (y.prec == LQ_F64) axpy_h_from<P64>(y, h, x, zero_x, st);
    else if (y.prec == LQ_F32) axpy_h_from<P32>(y, h, x, zero_x, st);
    else if (y.prec == LQ_F16) axpy_h_from<P16>(y, h, x, zero_x, st);
    else axpy_h_from<PDF>(y, h, x, zero_x, st);
}

void blas_axpy_h(Field& y, const double* a, const Field& x, cudaStream_t st) { axpy_h_any(y, a, x, 0, st); }

void blas_axpy_h_zero(Field& y, const double* a, Field& x, cudaStream_t st) { axpy_h_any(y, a, x, 1, st); }

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

void blas_cg_s(Field& s, const Field& q, const double* sc, df* part, cudaStream_t st, const FinArgs& fin) {
    if (s.prec != q.prec) fail(LQ_EINVAL, "blas_cg_s: precision mismatch");
#define K(NR) cg_s_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND_PDL(s, "blas_cg_s", K, red_grid(s.nrhs), s.view(), q.view(), sc, part, fin); }
    DISPATCH_P(s.prec, L);
#undef L
#undef K
}

template <int PX>
static void cg_xp_from(Field& x, Field& p, const Field& r, const double* sc, cudaStream_t st) {
    dim3 g = upd_grid(p.vh, p.nrhs);
#define K(NR) cg_xp_kernel<PX, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND_PDL(p, "blas_cg_xp", K, g, x.view(), p.view(), r.view(), sc); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_cg_xp(Field& x, Field& p, const Field& r, const double* sc, cudaStream_t st) {
    if (p.prec != r.prec) fail(LQ_EINVAL, "blas_cg_xp: precision mismatch");
    if (x.prec == LQ_F64) cg_xp_from<P64>(x, p, r, sc, st);
    else if (x.prec == LQ_F32) cg_xp_from<P32>(x, p, r, sc, st);
    else if (x.prec == LQ_F16) cg_xp_from<P16>(x, p, r, sc, st);
    else cg_xp_from<PDF>(x, p, r, sc, st);
}

template <int PX>
static void cg_xp_norm_from(Field& x, Field& p, const Field& r, const double* sc, df* part, cudaStream_t st,
                            const FinArgs& fin) {
#define K(NR) cg_xp_norm_kernel<PX, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(p, "blas_cg_xp", K, red_grid(p.nrhs), x.view(), p.view(), r.view(), sc, part, fin); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_cg_xp_norm(Field& x, Field& p, const Field& r, const double* sc, df* part, cudaStream_t st,
                     const FinArgs& fin) {
    if (p.prec != r.prec) fail(LQ_EINVAL, "blas_cg_xp_norm: precision mismatch");
    if (x.prec == LQ_F64) cg_xp_norm_from<P64>(x, p, r, sc, part, st, fin);
    else if (x.prec == LQ_F32) cg_xp_norm_from<P32>(x, p, r, sc, part, st, fin);
    else if (x.prec == LQ_F16) cg_xp_norm_from<P16>(x, p, r, sc, part, st, fin);
    else cg_xp_norm_from<PDF>(x, p, r, sc, part, st, fin);
}

void blas_bicg_cdot(const Field& a, const Field& b, df* part, cudaStream_t st, const FinArgs& fin) {
    if (a.prec != b.prec) fail(LQ_EINVAL, "blas_bicg_cdot: precision mismatch");
#define K(NR) cdot_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(a, "blas_bicg_cdot", K, red_grid(a.nrhs), a.view(), b.view(), part, fin); }
    DISPATCH_P(a.prec, L);
#undef L
#undef K
}

void blas_bicg_s(Field& r, const Field& v, const double* sc, cudaStream_t st) {
    if (r.prec != v.prec) fail(LQ_EINVAL, "blas_bicg_s: precision mismatch");
    dim3 g = upd_grid(r.vh, r.nrhs);
#define K(NR) bicg_s_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(r, "blas_bicg_s", K, g, r.view(), v.view(), sc); }
    DISPATCH_P(r.prec, L);
#undef L
#undef K
}

void blas_bicg_tdot(const Field& t, const Field& s, df* part, cudaStream_t st, const FinArgs& fin) {
    if (t.prec != s.prec) fail(LQ_EINVAL, "blas_bicg_tdot: precision mismatch");
#define K(NR) tdot_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(t, "blas_bicg_tdot", K, red_grid(t.nrhs), t.view(), s.view(), part, fin); }
    DISPATCH_P(t.prec, L);
#undef L
#undef K
}

template <int PX>
static void bicg_xr_from(Field& x, const Field& p, Field& r, const Field& t, const Field& r0, const double* sc,
                         df* part, cudaStream_t st, const FinArgs& fin) {
#define K(NR) bicg_xr_kernel<PX, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(x, "blas_bicg_xr", K, red_grid(x.nrhs), x.view(), p.view(), r.view(), t.view(), r0.view(), sc, part, fin); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_bicg_xr(Field& x, const Field& p, Field& r, const Field& t, const Field& r0, const double* sc, df* part,
                  cudaStream_t st, const FinArgs& fin) {
    if (p.prec != r.prec || p.prec != t.prec || p.prec != r0.prec) fail(LQ_EINVAL, "blas_bicg_xr: precision mismatch");
    if (x.prec == LQ_F64) bicg_xr_from<P64>(x, p, r, t, r0, sc, part, st, fin);
    else if (x.prec == LQ_F32) bicg_xr_from<P32>(x, p, r, t, r0, sc, part, st, fin);
    else if (x.prec == LQ_F16) bicg_xr_from<P16>(x, p, r, t, r0, sc, part, st, fin);
    else bicg_xr_from<PDF>(x, p, r, t, r0, sc, part, st, fin);
}

void blas_bicg_p(Field& p, const Field& r, const Field& v, const double* sc, cudaStream_t st) {
    if (p.prec != r.prec || p.prec != v.prec) fail(LQ_EINVAL, "blas_bicg_p: precision mismatch");
    dim3 g = upd_grid(p.vh, p.nrhs);
#define K(NR) bicg_p_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(p, "blas_bicg_p", K, g, p.view(), r.view(), v.view(), sc); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_bicg_rho(const Field& r, const Field& r0, df* part, cudaStream_t st, const FinArgs& fin) {
    if (r.prec != r0.prec) fail(LQ_EINVAL, "blas_bicg_rho: precision mismatch");
#define K(NR) rho_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(r, "blas_bicg_rho", K, red_grid(r.nrhs), r.view(), r0.view(), part, fin); }
    DISPATCH_P(r.prec, L);
#undef L
#undef K
}

void blas_lincomb4(Field& out, double a0, const Field& v, double a1, const Field& t, double a2, const Field& w,
                   cudaStream_t st, bool sub_old) {
    if (out.prec != v.prec || out.prec != t.prec || out.prec != w.prec) fail(LQ_EINVAL, "blas_lincomb4: precision mismatch");
    dim3 g = upd_grid(out.vh, out.nrhs);
#define K(NR) lincomb4_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(out, "blas_lincomb4", K, g, out.view(), a0, v.view(), a1, t.view(), a2, w.view(), (int)sub_old); }
    DISPATCH_P(out.prec, L);
#undef L
#undef K
}

void blas_gamma5(Field& out, const Field& in, cudaStream_t st) {
    if (out.prec != in.prec || out.kind != LQ_WILSON_FIELD || in.kind != LQ_WILSON_FIELD || out.nrhs != in.nrhs)
        fail(LQ_EINVAL, "blas_gamma5: Wilson fields of one precision and shape");
    dim3 g = upd_grid(out.vh, out.nrhs);
#define L(P) { launch("blas_gamma5", gamma5_kernel<P>, g, dim3(RED_THREADS), st, out.view(), in.view()); }
    DISPATCH_P(out.prec, L);
#undef L
}

void blas_caxpy_h(Field& y, const double* a_re, const double* a_im, const Field& x, cudaStream_t st) {
    if (y.prec != x.prec || y.nrhs != x.nrhs) fail(LQ_EINVAL, "blas_caxpy_h: field mismatch");
    HostScalars h = hs(a_re, a_im, y.nrhs);
    dim3 g = upd_grid(y.vh, y.nrhs);
#define K(NR) caxpy_h_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(y, "blas_caxpy", K, g, y.view(), x.view(), h); }
    DISPATCH_P(y.prec, L);
#undef L
#undef K
}

void blas_finalize(const df* part, int nblocks, int nrhs, double* sc, int slot, int op, cudaStream_t st) {
    launch_pdl("blas_finalize", finalize_kernel, dim3(nrhs), dim3(512), 0, st, part, nblocks, sc, slot, op);
}

void blas_cdot_multi(const FieldV* vs_dev, int nv, const Field& w, df* part, cudaStream_t st) {
    dim3 g(RED_BLOCKS, w.nrhs, nv);
#define K(NR) cdot_multi_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(w, "blas_multi_dots", K, g, vs_dev, w.view(), part); }
    DISPATCH_P(w.prec, L);
#undef L
#undef K
}

void blas_gcr_orth(const FieldV* qs_dev, const FieldV* ps_dev, int j, const double* coef_dev, int cstride,
                   const Field& like, cudaStream_t st) {
    dim3 g = upd_grid(like.vh, like.nrhs);
#define K(NR) gcr_orth_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(like, "blas_orth", K, g, qs_dev, ps_dev, j, coef_dev, cstride); }
    DISPATCH_P(like.prec, L);
#undef L
#undef K
}

template <int PX>
static void gcr_xr_from(Field& x, const Field& p, Field& r, const Field& q, const double* alpha, df* part,
                        cudaStream_t st) {
#define K(NR) gcr_xr_kernel<PX, P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(x, "blas_gcr_xr", K, red_grid(x.nrhs), x.view(), p.view(), r.view(), q.view(), alpha, part); }
    DISPATCH_P(p.prec, L);
#undef L
#undef K
}

void blas_gcr_xr(Field& x, const Field& p, Field& r, const Field& q, const double* alpha_dev, df* part,
                 cudaStream_t st) {
    if (p.prec != r.prec || p.prec != q.prec) fail(LQ_EINVAL, "blas_gcr_xr: precision mismatch");
    if (x.prec == LQ_F64) gcr_xr_from<P64>(x, p, r, q, alpha_dev, part, st);
    else if (x.prec == LQ_F32) gcr_xr_from<P32>(x, p, r, q, alpha_dev, part, st);
    else if (x.prec == LQ_F16) gcr_xr_from<P16>(x, p, r, q, alpha_dev, part, st);
    else gcr_xr_from<PDF>(x, p, r, q, alpha_dev, part, st);
}


void blas_ms_update(std::vector<Field>& y, std::vector<Field>& p, const Field& r, const double* a, const double* z,
                    const double* b, df* part, cudaStream_t st) {
    const int ns = (int)p.size(), n = r.nrhs;
    if (ns < 1 || ns > LQ_MS_MAXS || n > LQ_MS_MAXK || (int)y.size() != ns)
        fail(LQ_EINVAL, "blas_ms_update: shift or right-hand-side count");
    MsUpdate m;
    m.ns = ns;
    m.r = r.view();
    for (int i = 0; i < ns; i++) {
        if (y[i].prec != r.prec || p[i].prec != r.prec || y[i].nrhs != n || p[i].nrhs != n || p[i].kind != r.kind)
            fail(LQ_EINVAL, "blas_ms_update: field mismatch");
        m.y[i] = y[i].view();
        m.p[i] = p[i].view();
    }
    for (int i = 0; i < LQ_MS_MAXS; i++)
        for (int k = 0; k < LQ_MS_MAXK; k++) {
            const bool in = i < ns && k < n;
            m.a[i * LQ_MS_MAXK + k] = in ? a[i * n + k] : 0.0;
            m.z[i * LQ_MS_MAXK + k] = in ? z[i * n + k] : 0.0;
            m.b[i * LQ_MS_MAXK + k] = in ? b[i * n + k] : 1.0;
        }
#define K(NR) ms_update_kernel<P_, NR>
#define L(P) { constexpr int P_ = P; BY_KIND(r, "blas_ms_update", K, red_grid(n), m, part); }
    DISPATCH_P(r.prec, L);
#undef L
#undef K
}

}  // namespace lq
