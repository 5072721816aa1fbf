// core.cuh -- device-side building blocks shared by the kernels of the library:
// complex arithmetic, the even-odd site geometry, and the storage formats of
// spinors, colour vectors, links and clover fields in FP64 / FP32 / FP16.
//
// Storage: every field is an array of per-site records of NR reals, stored as
// "chunk-major" structure of arrays so that a warp reading chunk k of 32
// consecutive sites touches one contiguous segment:
//     chunk k of site s lives at  base[k * stride + s]   (in units of a chunk).
// Chunk types: FP64 double2 (2 reals); FP32 float4 (4 reals) when NR % 4 == 0,
// else float2; FP16 = 16-bit fixed point, 8 / 4 / 2 values per 16 / 8 / 4-byte
// chunk, value = q * scale / 32767 with scale either a per-site norm (spinors,
// clover) or one constant (links). q in [-32767, 32767] is stored offset-binary
// (u = q + 32768), so that decoding is a byte permute that places u in the
// mantissa of 2^23 and one exact subtraction, both on full-rate pipes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lq {

// P64: IEEE double. P32: float. P16: 16-bit fixed point with FP32 arithmetic.
// PDF: "double-float", a real stored and computed as an unevaluated sum of two
// floats hi + lo (about 48 significant bits). B300 runs FP64 at 1/64 of its
// FP32 rate, so the FP64-accuracy work of the mixed-precision solvers (reliable
// updates, source preparation, reconstruction, true residual) uses PDF and
// runs on the FP32 pipes.
enum Prec { P64 = 0, P32 = 1, P16 = 2, PDF = 3 };

// site-local epilogues fused into the hopping kernels (see wilson.cuh, hisq.cuh)
enum Epi { EPI_HOP = 0, EPI_AINV = 1, EPI_XPAY = 2 };

// ------------------------------------------------------------ double-float
// Error-free transformations of Knuth (two-sum) and Dekker/FMA (two-product);
// every step uses the _rn intrinsics so the compiler cannot contract or
// reassociate them. Relative error of one operation is about 2^-44.
struct df {
    float hi, lo;
    __host__ __device__ df() {}
    __host__ __device__ df(float h) : hi(h), lo(0.f) {}
    __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
    __device__ explicit df(int i) : hi((float)i), lo(0.f) {}
    __device__ explicit df(double d) {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
    }
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df(s, e);
}
__device__ __forceinline__ df operator+(df x, df y) {
    float s = __fadd_rn(x.hi, y.hi);
    float bb = __fsub_rn(s, x.hi);
    float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    return df_fast_two_sum(s, e);
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df operator/(df x, df y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    df r = x - df(q1) * y;
    float q2 = __fdiv_rn(r.hi, y.hi);
    return df_fast_two_sum(q1, q2);
}
__device__ __forceinline__ df& operator+=(df& x, df y) { x = x + y; return x; }
__device__ __forceinline__ df& operator-=(df& x, df y) { x = x - y; return x; }
__device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }
using ::fma;

// Reductions carry their partial sums as double-float values: B300 runs FP64
// at 1/64 of its FP32 rate, and even a block-level FP64 tree reduction on one
// SM costs microseconds. Every sum is formed in a fixed order (deterministic).
__device__ __forceinline__ df df_of(float v) { return df(v); }
__device__ __forceinline__ df df_of(double v) { return df(v); }
__device__ __forceinline__ df df_of(df v) { return v; }
__device__ __forceinline__ df shfl_down_df(df v, int o) {
    return df(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// block-wide double-float sum (valid in thread 0)
__device__ __forceinline__ df block_sum_df(df v) {
    __shared__ float2 red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_down_df(v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = make_float2(v.hi, v.lo);
    __syncthreads();
    v = df(0.f);
    if (wid == 0) {
        if (lane < (int)(blockDim.x >> 5)) v = df(red[lane].x, red[lane].y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = v + shfl_down_df(v, o);
    }
    return v;
}

// ------------------------------------------------------- scalar steps of CG
// scalar slots per right-hand side in the solver scalar block
// (the BiCGStab scalars are complex: rho = (r0, r), alpha, omega, beta as re/im pairs;
// SC_BREAK is set when a BiCGStab denominator vanishes)
enum {
    SC_RR = 0, SC_QQ, SC_SS, SC_RRN, SC_ALPHA, SC_BETA, SC_B2, SC_FROZEN, SC_PP,
    SC_RHO_R, SC_RHO_I, SC_AL_R, SC_AL_I, SC_OM_R, SC_OM_I, SC_BE_R, SC_BE_I, SC_BREAK,
    SC_SIGMA,  // the rhs's shift sigma of a hermitian operator sigma + K^+ K
    SC_ITERS,  // iterations done by the persistent CG kernel (running total)
    SC_N
};
enum { FIN_SET = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_BICG_ALPHA = 3, FIN_BICG_OMEGA = 4, FIN_BICG_BETA = 5,
       FIN_BICG_RHO = 6, FIN_CG_ALPHA = 7, FIN_CG_BETA = 8 };

// apply the scalar step to the total of a reduction (S: the rhs's scalar block).
// FIN_ALPHA / FIN_BETA: CG on the normal equations; FIN_CG_ALPHA / FIN_CG_BETA:
// CG on a hermitian operator sigma + K^+ K applied as |K p|^2 (tot) + sigma |p|^2
// (SC_PP), sigma per rhs in SC_SIGMA.
__device__ __forceinline__ void fin_apply(double* S, double tot, int slot, int op) {
    if (op == FIN_CG_ALPHA) {  // tot = |K p|^2: alpha = rr / (p, A p)
        S[SC_QQ] = tot;
        const double pap = S[SC_SIGMA] * S[SC_PP] + tot;
        if (S[SC_FROZEN] != 0.0) {
            S[SC_ALPHA] = 0.0;
        } else if (!(pap > 0.0)) {
            S[SC_ALPHA] = 0.0;
            S[SC_BREAK] = 1.0;
            S[SC_FROZEN] = 1.0;
        } else {
            S[SC_ALPHA] = S[SC_RR] / pap;
        }
        return;
    }
    if (op == FIN_CG_BETA) {  // tot = |r'|^2, the iterated residual: beta = rr'/rr
        S[SC_SS] = tot;
        S[SC_RRN] = tot;
        S[SC_BETA] = (S[SC_RR] > 0.0 && S[SC_FROZEN] == 0.0) ? tot / S[SC_RR] : 0.0;
        S[SC_RR] = tot;
        return;
    }
    if (op == FIN_SET) {
        S[slot] = tot;
    } else if (op == FIN_ALPHA) {  // tot = |q|^2: alpha = rr / qq
        S[SC_QQ] = tot;
        S[SC_ALPHA] = (tot > 0.0 && S[SC_FROZEN] == 0.0) ? S[SC_RR] / tot : 0.0;
    } else if (op == FIN_BETA) {   // tot = |r'|^2: beta = rr'/rr, rr = rr'
        S[SC_RRN] = tot;
        S[SC_BETA] = (S[SC_RR] > 0.0 && S[SC_FROZEN] == 0.0) ? tot / S[SC_RR] : 0.0;
        S[SC_RR] = tot;
    }
}

// BiCGStab steps (van der Vorst) on W = 2 or 3 totals of one right-hand side:
//   FIN_BICG_ALPHA  t = (r0, v):          alpha = rho / (r0, v)
//   FIN_BICG_OMEGA  t = (t, s), |t|^2:    omega = (t, s) / |t|^2
//   FIN_BICG_BETA   t = |r|^2, (r0, r):   beta = (rho' / rho)(alpha / omega), rho = rho'
//   FIN_BICG_RHO    t = |r|^2, (r0, r):   rho = (r0, r) (start, after a reliable update or restart)
// A frozen right-hand side gets zero steps; a vanishing denominator freezes it and sets SC_BREAK.
__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
    const double d = br * br + bi * bi;
    cr = (ar * br + ai * bi) / d;
    ci = (ai * br - ar * bi) / d;
}
__device__ __forceinline__ void fin_apply_bicg(double* S, const double* t, int op) {
    const bool frozen = S[SC_FROZEN] != 0.0;
    if (op == FIN_BICG_ALPHA) {
        if (frozen || (t[0] == 0.0 && t[1] == 0.0)) {
            if (!frozen) { S[SC_BREAK] = 1.0; S[SC_FROZEN] = 1.0; }
            S[SC_AL_R] = S[SC_AL_I] = 0.0;
        } else {
            cdiv(S[SC_RHO_R], S[SC_RHO_I], t[0], t[1], S[SC_AL_R], S[SC_AL_I]);
        }
    } else if (op == FIN_BICG_OMEGA) {
        if (frozen || !(t[2] > 0.0)) {
            if (!frozen) { S[SC_BREAK] = 1.0; S[SC_FROZEN] = 1.0; }
            S[SC_OM_R] = S[SC_OM_I] = 0.0;
        } else {
            S[SC_OM_R] = t[0] / t[2];
            S[SC_OM_I] = t[1] / t[2];
        }
    } else if (op == FIN_BICG_BETA) {
        S[SC_SS] = t[0];
        double qr = 0.0, qi = 0.0, br = 0.0, bi = 0.0;
        const bool ok = !frozen && (S[SC_RHO_R] != 0.0 || S[SC_RHO_I] != 0.0) && (S[SC_OM_R] != 0.0 || S[SC_OM_I] != 0.0);
        if (ok) {
            cdiv(t[1], t[2], S[SC_RHO_R], S[SC_RHO_I], qr, qi);  // rho' / rho
            double ar, ai;
            cdiv(S[SC_AL_R], S[SC_AL_I], S[SC_OM_R], S[SC_OM_I], ar, ai);  // alpha / omega
            br = qr * ar - qi * ai;
            bi = qr * ai + qi * ar;
        }
        S[SC_BE_R] = br;
        S[SC_BE_I] = bi;
        S[SC_RHO_R] = t[1];
        S[SC_RHO_I] = t[2];
    } else if (op == FIN_BICG_RHO) {  // |r|^2 of the sloppy copy goes to SC_RRN
        S[SC_RRN] = t[0];
        S[SC_RHO_R] = t[1];
        S[SC_RHO_I] = t[2];
    }
}

// A reduction finalised inside the kernel that produces its partials: the last
// block to finish (atomic ticket) sums every rhs's partials in index order and
// applies the scalar step, then re-arms the ticket. sc == nullptr: no fusion.
struct FinArgs {
    double* sc = nullptr;
    int slot = 0;
    int op = 0;
    unsigned* count = nullptr;
};

// W totals per right-hand side: partial w of rhs k from block b at part[(k * W + w) * nparts + b]
template <int W>
__device__ __forceinline__ void fin_tail_w(const df* part, int nparts, int nrhs, const FinArgs& f) {
    if (!f.sc) return;
    __shared__ int last_w;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y * gridDim.z;
        last_w = atomicAdd(f.count, 1u) == total - 1;
    }
    __syncthreads();
    if (!last_w) return;
    __threadfence();
    for (int k = 0; k < nrhs; k++) {
        double tot[W];
#pragma unroll
        for (int w = 0; w < W; w++) {
            const df* pk = part + (size_t)(k * W + w) * nparts;
            df sum(0.f);
            const int B = blockDim.x;
            int i = threadIdx.x;
            for (; i + 7 * B < nparts; i += 8 * B) {  // eight in flight, same order of additions
                float2 v[8];
#pragma unroll
                for (int j = 0; j < 8; j++) v[j] = __ldcg((const float2*)(pk + i + j * B));
#pragma unroll
                for (int j = 0; j < 8; j++) sum = sum + df(v[j].x, v[j].y);
            }
            for (; i < nparts; i += B) {
                const float2 v = __ldcg((const float2*)(pk + i));
                sum = sum + df(v.x, v.y);
            }
            tot[w] = df_to_double(block_sum_df(sum));
        }
        if (threadIdx.x == 0) fin_apply_bicg(f.sc + (size_t)k * SC_N, tot, f.op);
    }
    if (threadIdx.x == 0) *f.count = 0u;
}

// called by every thread of every block after thread 0 wrote the block's partials
__device__ __forceinline__ void fin_tail(const df* part, int nparts, int nrhs, const FinArgs& f) {
    if (!f.sc) return;
    __shared__ int last;
    if (threadIdx.x == 0) {
        __threadfence();  // this block's partials before its ticket
        const unsigned total = gridDim.x * gridDim.y * gridDim.z;
        last = atomicAdd(f.count, 1u) == total - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int k = 0; k < nrhs; k++) {
        const df* pk = part + (size_t)k * nparts;
        df sum(0.f);
        // sixteen partials in flight per thread (missing ones read as zero, which adds
        // nothing), added in the same order as one at a time
        const int B = blockDim.x;
        for (int i0 = threadIdx.x; i0 < nparts; i0 += 16 * B) {
            float2 v[16];
#pragma unroll
            for (int j = 0; j < 16; j++)
                v[j] = i0 + j * B < nparts ? __ldcg((const float2*)(pk + i0 + j * B)) : make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (i0 + j * B < nparts) sum = sum + df(v[j].x, v[j].y);
        }
        sum = block_sum_df(sum);
        if (threadIdx.x == 0) fin_apply(f.sc + (size_t)k * SC_N, df_to_double(sum), f.slot, f.op);
    }
    if (threadIdx.x == 0) *f.count = 0u;
}

// conversions between the arithmetic types of the kernels
template <typename T> __device__ __forceinline__ T from_df(df d);
template <> __device__ __forceinline__ df from_df<df>(df d) { return d; }
template <> __device__ __forceinline__ double from_df<double>(df d) { return (double)d.hi + (double)d.lo; }
template <> __device__ __forceinline__ float from_df<float>(df d) { return __fadd_rn(d.hi, d.lo); }
__device__ __forceinline__ df to_df(df v) { return v; }
__device__ __forceinline__ df to_df(double v) { return df(v); }
__device__ __forceinline__ df to_df(float v) { return df(v); }

template <int P> struct RealT { typedef float T; };
template <> struct RealT<P64> { typedef double T; };
template <> struct RealT<PDF> { typedef df T; };

// ------------------------------------------------------------------ complex
template <typename T> struct cx {
    T r, i;
};

template <typename T> __device__ __forceinline__ cx<T> mk(T r, T i) { cx<T> c; c.r = r; c.i = i; return c; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.r + b.r, a.i + b.i); }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.r - b.r, a.i - b.i); }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk(a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r);
}
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(s * a.r, s * a.i); }
template <typename T> __device__ __forceinline__ cx<T> cj(cx<T> a) { return mk(a.r, -a.i); }
// i * a
template <typename T> __device__ __forceinline__ cx<T> ti(cx<T> a) { return mk(-a.i, a.r); }
// acc += a * b
template <typename T> __device__ __forceinline__ void cmac(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, acc.r); acc.r = fma(-a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i); acc.i = fma(a.i, b.r, acc.i);
}
// acc += conj(a) * b
template <typename T> __device__ __forceinline__ void cjmac(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.r = fma(a.r, b.r, acc.r); acc.r = fma(a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i); acc.i = fma(-a.i, b.r, acc.i);
}

// ---------------------------------------------------------------- geometry
// Even-odd ("checkerboard") order: within parity p, site cb = lex / 2 with
// lex = x + Lx*(y + Ly*(z + Lz*t)); Lx is even, so x = 2*(cb % (Lx/2)) + ((y+z+t+p) & 1).
struct Geo {
    int L[4];
    int lxh;      // Lx / 2
    int vh;       // V / 2 (sites per parity)
    int bc_t;     // time boundary sign, +1 or -1
    // multiply-high divisors by lxh, L[1], L[2]: n / d = umulhi(n, ceil(2^32 / d)),
    // exact while n d < 2^32 (0 stands for d = 1); fast = 0 where that fails
    unsigned fdiv[3];
    int fast;
};

__device__ __forceinline__ void cb_coords(const Geo& g, int cb, int p, int c[4]) {
    int xh = cb % g.lxh;
    int r = cb / g.lxh;
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

__device__ __forceinline__ int cb_index(const Geo& g, const int c[4]) {
    return (c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]))) >> 1;
}

// checkerboard index of x + k mu (wrapping several times for tiny extents) and
// the boundary sign picked up on the straight path
__device__ __forceinline__ int cb_hop(const Geo& g, const int c[4], int mu, int k, float& sign) {
    int n[4] = {c[0], c[1], c[2], c[3]};
    int L = g.L[mu];
    int v = c[mu] + k;
    int wraps = 0;
    while (v >= L) { v -= L; wraps++; }
    while (v < 0) { v += L; wraps++; }
    n[mu] = v;
    sign = (mu == 3 && g.bc_t < 0 && (wraps & 1)) ? -1.f : 1.f;
    return cb_index(g, n);
}

// ----------------------------------------------------------------- storage
template <int P, int NR> struct Chunk;
template <int NR> struct Chunk<P64, NR> { typedef double2 C; enum { RPC = 2 }; };
// double-float: two reals v0, v1 as (v0.hi, v1.hi, v0.lo, v1.lo), so that for a complex
// number the high parts (re, im) and the low parts are aligned register pairs
template <int NR> struct Chunk<PDF, NR> { typedef float4 C; enum { RPC = 2 }; };
template <int NR> struct Chunk<P32, NR> {
    typedef typename std::conditional<NR % 4 == 0, float4, float2>::type C;
    enum { RPC = (NR % 4 == 0) ? 4 : 2 };
};
template <int NR> struct Chunk<P16, NR> {
    typedef typename std::conditional<NR % 8 == 0, int4, typename std::conditional<NR % 4 == 0, int2, int>::type>::type C;
    enum { RPC = (NR % 8 == 0) ? 8 : ((NR % 4 == 0) ? 4 : 2) };
};

template <int P, int NR> struct Layout {
    typedef typename Chunk<P, NR>::C C;
    enum { RPC = Chunk<P, NR>::RPC, NC = NR / Chunk<P, NR>::RPC };
};

// 2^23 + 32768: the float whose mantissa holds the offset-binary zero
#define LQ_F16_MAGIC 8421376.0f
__device__ __forceinline__ float s16lo(int w) {
    return __int_as_float((int)__byte_perm((unsigned)w, 0x4B000000u, 0x7610)) - LQ_F16_MAGIC;
}
__device__ __forceinline__ float s16hi(int w) {
    return __int_as_float((int)__byte_perm((unsigned)w, 0x4B000000u, 0x7632)) - LQ_F16_MAGIC;
}
// two reals times f, each in [-32767, 32767] after scaling, to offset-binary codes:
// adding 2^23 + 32768 rounds to the nearest integer (ties to even) and leaves
// code + 32768 in the low 16 bits of the float, so no float-to-int conversion is needed
__device__ __forceinline__ int pack16f(float a, float b, float f) {
    const unsigned ua = __float_as_uint(__fmaf_rn(a, f, LQ_F16_MAGIC));
    const unsigned ub = __float_as_uint(__fmaf_rn(b, f, LQ_F16_MAGIC));
    return (int)__byte_perm(ua, ub, 0x5410);
}

// unpack one chunk c into RPC reals (FP16: times f = scale/32767)
template <int P, int NR, typename T>
__device__ __forceinline__ void unpack_chunk(const typename Layout<P, NR>::C& c, float f, T* v) {
    typedef Layout<P, NR> Lay;
    if constexpr (P == P64) {
        v[0] = (T)c.x; v[1] = (T)c.y;
    } else if constexpr (P == PDF) {
        v[0] = from_df<T>(df(c.x, c.z));
        v[1] = from_df<T>(df(c.y, c.w));
    } else if constexpr (P == P32) {
        if constexpr (Lay::RPC == 4) {
            v[0] = (T)c.x; v[1] = (T)c.y; v[2] = (T)c.z; v[3] = (T)c.w;
        } else {
            v[0] = (T)c.x; v[1] = (T)c.y;
        }
    } else {
        if constexpr (Lay::RPC == 8) {
            v[0] = (T)(s16lo(c.x) * f); v[1] = (T)(s16hi(c.x) * f);
            v[2] = (T)(s16lo(c.y) * f); v[3] = (T)(s16hi(c.y) * f);
            v[4] = (T)(s16lo(c.z) * f); v[5] = (T)(s16hi(c.z) * f);
            v[6] = (T)(s16lo(c.w) * f); v[7] = (T)(s16hi(c.w) * f);
        } else if constexpr (Lay::RPC == 4) {
            v[0] = (T)(s16lo(c.x) * f); v[1] = (T)(s16hi(c.x) * f);
            v[2] = (T)(s16lo(c.y) * f); v[3] = (T)(s16hi(c.y) * f);
        } else {
            v[0] = (T)(s16lo(c) * f); v[1] = (T)(s16hi(c) * f);
        }
    }
}

// load NR reals of site s; for P16 multiply by scale/32767
template <int P, int NR, typename T>
__device__ __forceinline__ void load_reals(const void* base, int stride, int s, float scale, T* v) {
    typedef Layout<P, NR> Lay;
    const typename Lay::C* b = (const typename Lay::C*)base;
    const float f = scale * (1.f / 32767.f);
#pragma unroll
    for (int k = 0; k < Lay::NC; k++) {
        typename Lay::C c = __ldg(&b[(size_t)k * stride + s]);
        unpack_chunk<P, NR, T>(c, f, v + k * Lay::RPC);
    }
}

// FP16 chunk to its integer codes (the caller applies the scale)
template <int NR, typename T>
__device__ __forceinline__ void unpack_codes16(const typename Layout<P16, NR>::C& c, T* v) {
    typedef Layout<P16, NR> Lay;
    if constexpr (Lay::RPC == 8) {
        v[0] = (T)s16lo(c.x); v[1] = (T)s16hi(c.x); v[2] = (T)s16lo(c.y); v[3] = (T)s16hi(c.y);
        v[4] = (T)s16lo(c.z); v[5] = (T)s16hi(c.z); v[6] = (T)s16lo(c.w); v[7] = (T)s16hi(c.w);
    } else if constexpr (Lay::RPC == 4) {
        v[0] = (T)s16lo(c.x); v[1] = (T)s16hi(c.x); v[2] = (T)s16lo(c.y); v[3] = (T)s16hi(c.y);
    } else {
        v[0] = (T)s16lo(c); v[1] = (T)s16hi(c);
    }
}

// load the reals of chunk k only (RPC of them); SMEM: base is a shared-memory copy;
// CODES: FP16 entries come back as integer codes, unscaled
template <int P, int NR, typename T, bool SMEM = false, bool CODES = false>
__device__ __forceinline__ void load_chunk(const void* base, int stride, int s, int k, float scale, T* v) {
    typedef Layout<P, NR> Lay;
    const typename Lay::C* b = (const typename Lay::C*)base;
    typename Lay::C c;
    if constexpr (SMEM) c = b[(size_t)k * stride + s];
    else c = __ldg(&b[(size_t)k * stride + s]);
    if constexpr (P == P16 && CODES) unpack_codes16<NR, T>(c, v);
    else unpack_chunk<P, NR, T>(c, scale * (1.f / 32767.f), v);
}

// ------------------------------------------------------- async copies (cp.async)
// Each thread copies its own records into a private slice of shared memory,
// laid out chunk-major like global memory (chunk k of thread t at k*blockDim + t),
// so that reading it back is conflict-free.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Programmatic dependent launch (kernels launched with launch_pdl): pdl_start() first lets
// the next such kernel of the stream be scheduled once all blocks of this one have
// started (its blocks then wait in their own pdl_start), and then waits until the
// previous kernel of the stream has completed and its memory is visible. Without the
// launch attribute both instructions do nothing.
__device__ __forceinline__ void pdl_start() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// copy the NR-real record of site s (chunk-major global array with stride vh)
// into this thread's slice of smem (stride blockDim.x); returns bytes per thread used
template <int P, int NR>
__device__ __forceinline__ void prefetch_record(void* smem, const void* gbase, int vh, int s) {
    typedef Layout<P, NR> Lay;
    typedef typename Lay::C C;
    C* d = (C*)smem;
    const C* g = (const C*)gbase;
#pragma unroll
    for (int k = 0; k < Lay::NC; k++) {
        if constexpr (sizeof(C) == 16) cp_async16(&d[k * blockDim.x + threadIdx.x], &g[(size_t)k * vh + s]);
        else if constexpr (sizeof(C) == 8) cp_async8(&d[k * blockDim.x + threadIdx.x], &g[(size_t)k * vh + s]);
        else cp_async4(&d[k * blockDim.x + threadIdx.x], &g[(size_t)k * vh + s]);
    }
}

// store NR reals of site s. For P16 with a per-site norm the norm is computed
// here (max |v|) and written to norm[s]; with norm == nullptr `scale` is used.
template <int P, int NR, typename T>
__device__ __forceinline__ void store_reals(void* base, int stride, int s, float* norm, float scale, const T* v) {
    typedef Layout<P, NR> Lay;
    typename Lay::C* b = (typename Lay::C*)base;
    if constexpr (P == P16) {
        float nrm = scale;
        if (norm) {
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < NR; k++) m = fmaxf(m, fabsf((float)v[k]));
            nrm = m;
            norm[s] = m;
        }
        // |v| f <= 32767 (1 + 2^-22) rounds to at most 32767
        const float f = nrm > 0.f ? __fdividef(32767.f, nrm) : 0.f;
#pragma unroll
        for (int k = 0; k < Lay::NC; k++) {
            typename Lay::C c;
            if constexpr (Lay::RPC == 8) {
                c.x = pack16f((float)v[8 * k + 0], (float)v[8 * k + 1], f);
                c.y = pack16f((float)v[8 * k + 2], (float)v[8 * k + 3], f);
                c.z = pack16f((float)v[8 * k + 4], (float)v[8 * k + 5], f);
                c.w = pack16f((float)v[8 * k + 6], (float)v[8 * k + 7], f);
            } else if constexpr (Lay::RPC == 4) {
                c.x = pack16f((float)v[4 * k + 0], (float)v[4 * k + 1], f);
                c.y = pack16f((float)v[4 * k + 2], (float)v[4 * k + 3], f);
            } else {
                c = pack16f((float)v[2 * k + 0], (float)v[2 * k + 1], f);
            }
            b[(size_t)k * stride + s] = c;
        }
    } else {
#pragma unroll
        for (int k = 0; k < Lay::NC; k++) {
            typename Lay::C c;
            if constexpr (P == P64) {
                c.x = (double)v[2 * k]; c.y = (double)v[2 * k + 1];
            } else if constexpr (P == PDF) {
                const df a0 = to_df(v[2 * k]), a1 = to_df(v[2 * k + 1]);
                c.x = a0.hi; c.y = a1.hi; c.z = a0.lo; c.w = a1.lo;
            } else if constexpr (Lay::RPC == 4) {
                c.x = (float)v[4 * k]; c.y = (float)v[4 * k + 1]; c.z = (float)v[4 * k + 2]; c.w = (float)v[4 * k + 3];
            } else {
                c.x = (float)v[2 * k]; c.y = (float)v[2 * k + 1];
            }
            b[(size_t)k * stride + s] = c;
        }
    }
}

// A field of one parity with nrhs right-hand sides: rhs k starts at
// data + k * rhs_bytes; norm (FP16 only) at norm + k * vh.
struct FieldV {
    void* data;
    float* norm;
    int vh;
    size_t rhs_bytes;
};

template <int P, int NR, typename T>
__device__ __forceinline__ void fload(const FieldV& f, int k, int s, T* v) {
    const char* base = (const char*)f.data + (size_t)k * f.rhs_bytes;
    float sc = 1.f;
    if constexpr (P == P16) sc = __ldg(f.norm + (size_t)k * f.vh + s);
    load_reals<P, NR, T>(base, f.vh, s, sc, v);
}

template <int P, int NR, typename T>
__device__ __forceinline__ void fstore(const FieldV& f, int k, int s, const T* v) {
    char* base = (char*)f.data + (size_t)k * f.rhs_bytes;
    store_reals<P, NR, T>(base, f.vh, s, P == P16 ? f.norm + (size_t)k * f.vh : nullptr, 1.f, v);
}

// --------------------------------------------------------------- links
// Links of parity p and direction mu: block (p*4 + mu) of NC chunks x vh.
// R = 18: all nine entries. R = 12: rows 0 and 1; row 2 = conj(row0 x row1),
// exact for SU(3). R = 8: u01, u02, u10 and the phases arg(u00)/pi and
// arg(u20)/pi (the phases stored times the field's scale, so that the FP16
// codec treats all eight reals alike); the rest follows from SU(3), see
// su3_recon8. Boundary signs are never stored in links.
struct GaugeV {
    const void* data;
    int vh;
    float scale;  // FP16 fixed-point scale (max |entry| of the field); 1 otherwise
};

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// SU(3) from eight reals. Row 0 and column 0 have unit norm, which gives
// |u00|^2 = 1 - |u01|^2 - |u02|^2 =: 1 - N and |u20|^2 = N - |u10|^2; with the
// stored phases that fixes row 0 and column 0. For a unitary matrix of
// determinant 1 every entry equals the complex conjugate of its cofactor, so
//   u10 w1 - u20 v1 = conj(u02),   u20 v2 - u10 w2 = conj(u01)
// (rows v = row 1, w = row 2), and column 0 is orthogonal to columns 1 and 2:
//   conj(u10) v1 + conj(u20) w1 = -conj(u00) u01,
//   conj(u10) v2 + conj(u20) w2 = -conj(u00) u02.
// Each pair is a 2x2 linear system of determinant -+(|u10|^2 + |u20|^2) = -+N,
// solved by Cramer's rule below. N = 0 (|u00| = 1) is singular: the packing
// step refuses such fields. FAST (FP16 links, whose entries carry 2^-15
// absolute error anyway) takes the hardware approximations of sin, cos,
// 1/sqrt and 1/x (absolute errors near 1e-6 and below) instead of the
// correctly rounded library functions.
template <typename T, bool FAST = false>
__device__ __forceinline__ void su3_recon8(const T v[8], cx<T> U[3][3]) {
    const cx<T> u1 = mk(v[0], v[1]), u2 = mk(v[2], v[3]), v0 = mk(v[4], v[5]);
    const T n = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
    const T q0 = fmax((T)1 - n, (T)0);
    const T q2 = fmax(n - v[4] * v[4] - v[5] * v[5], (T)0);
    T a0, a2, s0, c0, s2, c2, inv;
    if constexpr (FAST && std::is_same<T, float>::value) {
        a0 = q0 > 0.f ? q0 * rsqrtf(q0) : 0.f;
        a2 = q2 > 0.f ? q2 * rsqrtf(q2) : 0.f;
        const float pi = 3.14159265358979f;
        __sincosf(pi * v[6], &s0, &c0);
        __sincosf(pi * v[7], &s2, &c2);
        inv = __fdividef(1.f, n);
    } else {
        a0 = sqrt(q0);
        a2 = sqrt(q2);
        sincospi_t(v[6], &s0, &c0);
        sincospi_t(v[7], &s2, &c2);
        inv = (T)1 / n;
    }
    const cx<T> u0 = mk(a0 * c0, a0 * s0), w0 = mk(a2 * c2, a2 * s2);
    const cx<T> p1 = cj(u0) * u1, p2 = cj(u0) * u2;
    U[0][0] = u0; U[0][1] = u1; U[0][2] = u2;
    U[1][0] = v0;
    U[2][0] = w0;
    U[1][1] = -inv * (cj(u2 * w0) + p1 * v0);
    U[2][1] = inv * (cj(u2 * v0) - p1 * w0);
    U[1][2] = inv * (cj(u1 * w0) - p2 * v0);
    U[2][2] = -inv * (p2 * w0 + cj(u1 * v0));
}

template <int P, int R, typename T>
__device__ __forceinline__ void load_link(const GaugeV& g, int p, int mu, int s, cx<T> U[3][3]) {
    typedef Layout<P, R> Lay;
    const char* base = (const char*)g.data + (size_t)(p * 4 + mu) * Lay::NC * g.vh * sizeof(typename Lay::C);
    T v[R];
    load_reals<P, R, T>(base, g.vh, s, g.scale, v);
    if constexpr (R == 8) {
        const T is = (T)1 / (T)g.scale;
        v[6] *= is;
        v[7] *= is;
        su3_recon8<T, P == P16>(v, U);
        return;
    } else {
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) U[a][b] = mk(v[(a * 3 + b) * 2], v[(a * 3 + b) * 2 + 1]);
        if constexpr (R == 18) {
#pragma unroll
            for (int b = 0; b < 3; b++) U[2][b] = mk(v[(6 + b) * 2], v[(6 + b) * 2 + 1]);
        } else {
            // row2 = conj(row0 x row1)
            U[2][0] = cj(U[0][1] * U[1][2] - U[0][2] * U[1][1]);
            U[2][1] = cj(U[0][2] * U[1][0] - U[0][0] * U[1][2]);
            U[2][2] = cj(U[0][0] * U[1][1] - U[0][1] * U[1][0]);
        }
    }
}

// A link from its raw chunks (software-pipelined hops). FP32: U is the link.
// FP16 with R = 18 / 12: U holds the link divided by scale/32767 (integer codes;
// R12's third row is rescaled once here), and the caller folds scale/32767 into
// its per-hop factor. FP16 with R = 8: U is the link (the reconstruction needs
// true values), so the caller folds in nothing.
template <int P, int R, typename T>
__device__ __forceinline__ void decode_link(const typename Layout<P, R>::C* u, float scale, cx<T> U[3][3]) {
    typedef Layout<P, R> LU;
    T lv[R];
#pragma unroll
    for (int k = 0; k < LU::NC; k++) {
        if constexpr (P == P16) unpack_codes16<R, T>(u[k], lv + k * LU::RPC);
        else unpack_chunk<P, R, T>(u[k], 1.f, lv + k * LU::RPC);
    }
    if constexpr (R == 8) {
        // FP16: entries are codes * scale/32767 and the phases codes/32767; FP32: scale = 1
        const T fe = P == P16 ? (T)(scale * (1.f / 32767.f)) : (T)1;
        const T fp = P == P16 ? (T)(1.f / 32767.f) : (T)1;
#pragma unroll
        for (int k = 0; k < 6; k++) lv[k] *= fe;
        lv[6] *= fp;
        lv[7] *= fp;
        su3_recon8<T, P == P16>(lv, U);
    } else {
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int q = 0; q < 3; q++) U[r][q] = mk(lv[(r * 3 + q) * 2], lv[(r * 3 + q) * 2 + 1]);
        if constexpr (R == 18) {
#pragma unroll
            for (int q = 0; q < 3; q++) U[2][q] = mk(lv[(6 + q) * 2], lv[(6 + q) * 2 + 1]);
        } else {
            U[2][0] = cj(U[0][1] * U[1][2] - U[0][2] * U[1][1]);
            U[2][1] = cj(U[0][2] * U[1][0] - U[0][0] * U[1][2]);
            U[2][2] = cj(U[0][0] * U[1][1] - U[0][1] * U[1][0]);
            if constexpr (P == P16) {  // conj(row0 x row1) of codes carries the scale twice
                const T fu = (T)(scale * (1.f / 32767.f));
#pragma unroll
                for (int q = 0; q < 3; q++) U[2][q] = fu * U[2][q];
            }
        }
    }
}

// the factor that decode_link leaves to its caller
template <int P, int R>
__device__ __forceinline__ float link_factor(float scale) {
    return (P == P16 && R != 8) ? scale * (1.f / 32767.f) : 1.f;
}

// out = U v, out = U^+ v
template <typename T>
__device__ __forceinline__ void su3_mv(const cx<T> U[3][3], const cx<T> v[3], cx<T> out[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx<T> acc = U[a][0] * v[0];
        cmac(acc, U[a][1], v[1]);
        cmac(acc, U[a][2], v[2]);
        out[a] = acc;
    }
}
template <typename T>
__device__ __forceinline__ void su3_dmv(const cx<T> U[3][3], const cx<T> v[3], cx<T> out[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        cx<T> acc = mk((T)0, (T)0);
        cjmac(acc, U[0][a], v[0]);
        cjmac(acc, U[1][a], v[1]);
        cjmac(acc, U[2][a], v[2]);
        out[a] = acc;
    }
}

}  // namespace lq
