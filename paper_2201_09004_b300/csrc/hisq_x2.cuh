// hisq_x2.cuh -- FP16-storage HISQ hopping kernel on packed FP32 pairs.
//
// The operator of hisq.cuh (Sec. 2.2 Eq. 4 with the HISQ fat one-hop links V and
// long three-hop links W, MILC phases, time-boundary sign per crossing), for one
// right-hand side per thread with FP16 colour vectors, fat links at R18 and long
// links at R12. The fat and the long hop of one direction and orientation,
//   V_mu(x) psi(x + mu)   and   W_mu(x) psi(x + 3 mu)   (or the backward pair),
// are computed together as one 3x3 complex product on (fat, long) lane pairs
// (fma.rn.f32x2: two multiply-adds per instruction), with the per-hop factors
// (phase, boundary sign, FP16 scales, and c_naik on the long lane) applied to the
// pair; the two lanes are added at the end. Site coordinates come from
// multiply-high divisions and the neighbour indices at distance 1 and 3 from the
// coordinates without loops; the gathers of the next pair of hops are in flight
// while a pair is computed. The result agrees with hisq.cuh to FP32 rounding.
#pragma once
#include "hisq.cuh"
#include "wilson_x2.cuh"

namespace lq {

// checkerboard index of x + K mu (K = +-1 or +-3) and the time-boundary sign of the
// path (one factor per crossing; a three-hop path may wrap twice on an extent of 2)
template <int MU, int K>
__device__ __forceinline__ int stag_nb(const Geo& g, int s, const int c[4], int xh, float& bs) {
    const int L = g.L[MU];
    int v = c[MU] + K, wraps = 0;
    if constexpr (K > 0) {
        if (v >= L) { v -= L; wraps++; }
        if (v >= L) { v -= L; wraps++; }
    } else {
        if (v < 0) { v += L; wraps++; }
        if (v < 0) { v += L; wraps++; }
    }
    bs = (MU == 3 && (wraps & 1)) ? (float)g.bc_t : 1.f;
    if constexpr (MU == 0) return s - xh + (v >> 1);
    const int stride = MU == 1 ? g.lxh : (MU == 2 ? g.lxh * g.L[1] : g.lxh * g.L[1] * g.L[2]);
    return s + (v - c[MU]) * stride;
}

// raw chunks of a (fat, long) pair of hops: the two neighbour vectors (3 words each:
// one complex per colour) with their norms, the fat link (9 words) and the long link
// (3 double words, R12)
struct HPairRaw {
    int spf[3], spl[3];
    float nf, nl, bsf, bsl;
    int uf[9];
    int2 ul[3];
};

// pair Q (0..7): direction Q >> 1, forward for even Q
template <int Q>
__device__ __forceinline__ void hisq_fetch(const HisqArgs& a, int s, const int c[4], int xh, HPairRaw& r) {
    constexpr int MU = Q >> 1;
    constexpr bool FWD = (Q & 1) == 0;
    const int nf = stag_nb<MU, FWD ? 1 : -1>(a.g, s, c, xh, r.bsf);
    const int nl = stag_nb<MU, FWD ? 3 : -3>(a.g, s, c, xh, r.bsl);
    const size_t vh = (size_t)a.g.vh;
    const int* sb = (const int*)a.in.data;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        r.spf[k] = __ldg(&sb[k * vh + nf]);
        r.spl[k] = __ldg(&sb[k * vh + nl]);
    }
    r.nf = __ldg(a.in.norm + nf);
    r.nl = __ldg(a.in.norm + nl);
    const int lp = FWD ? a.parity : 1 - a.parity;
    const int* ub = (const int*)a.fat.data + (size_t)(lp * 4 + MU) * 9 * vh;
    const int2* wb = (const int2*)a.lng.data + (size_t)(lp * 4 + MU) * 3 * vh;
    const int lf = FWD ? s : nf, ll = FWD ? s : nl;
#pragma unroll
    for (int k = 0; k < 9; k++) r.uf[k] = __ldg(&ub[k * vh + lf]);
#pragma unroll
    for (int k = 0; k < 3; k++) r.ul[k] = __ldg(&wb[k * vh + ll]);
}

// acc (per colour: real and imaginary (fat, long) pairs) += f (L_fat psi_1, L_long psi_3),
// L the link or its adjoint, f the pair of per-hop factors
template <int Q>
__device__ __forceinline__ void hisq_process(const HisqArgs& a, const HPairRaw& r, float eta, float cn, float2 accr[3],
                                             float2 acci[3]) {
    constexpr bool FWD = (Q & 1) == 0;
    cx<float> F[3][3], W[3][3];
    decode_link<P16, 18, float>(r.uf, a.fat.scale, F);
    decode_r12_codes(r.ul, W);  // row 2 one factor scale/32767 short (applied on the long lane below)
    const float2 f2l = make_float2(1.f, a.lng.scale * (1.f / 32767.f));
    float2 Vr[3], Vi[3], NV[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
        Vr[b] = make_float2(s16lo(r.spf[b]), s16lo(r.spl[b]));
        Vi[b] = make_float2(s16hi(r.spf[b]), s16hi(r.spl[b]));
        if (!FWD && b == 2) {  // conj(W[2][i]) multiplies component 2 of the long hop
            Vr[b] = __fmul2_rn(Vr[b], f2l);
            Vi[b] = __fmul2_rn(Vi[b], f2l);
        }
        NV[b] = __fmul2_rn(FWD ? Vi[b] : Vr[b], bc2(-1.f));
    }
    float2 Rr[3], Ri[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Rr[i] = bc2(0.f);
        Ri[i] = bc2(0.f);
#pragma unroll
        for (int b = 0; b < 3; b++) {
            // forward: U[i][b] psi[b]; backward: conj(U[b][i]) psi[b]
            const cx<float> f = FWD ? F[i][b] : F[b][i];
            const cx<float> w = FWD ? W[i][b] : W[b][i];
            const float2 Ur = make_float2(f.r, w.r), Ui = make_float2(f.i, w.i);
            Rr[i] = __ffma2_rn(Ur, Vr[b], Rr[i]);
            Ri[i] = __ffma2_rn(Ur, Vi[b], Ri[i]);
            if constexpr (FWD) {  // re -= Ui Vi, im += Ui Vr
                Rr[i] = __ffma2_rn(Ui, NV[b], Rr[i]);
                Ri[i] = __ffma2_rn(Ui, Vr[b], Ri[i]);
            } else {              // re += Ui Vi, im -= Ui Vr
                Rr[i] = __ffma2_rn(Ui, Vi[b], Rr[i]);
                Ri[i] = __ffma2_rn(Ui, NV[b], Ri[i]);
            }
        }
    }
    if constexpr (FWD) {  // row 2 of W
        Rr[2] = __fmul2_rn(Rr[2], f2l);
        Ri[2] = __fmul2_rn(Ri[2], f2l);
    }
    // forward hops add, backward hops subtract; FP16 scales, boundary signs and c_naik
    const float sg = FWD ? 1.f : -1.f;
    const float ff = eta * sg * r.bsf * r.nf * (1.f / 32767.f) * a.fat.scale * (1.f / 32767.f);
    const float fl = eta * cn * sg * r.bsl * r.nl * (1.f / 32767.f) * a.lng.scale * (1.f / 32767.f);
    const float2 fp = make_float2(ff, fl);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        accr[i] = __ffma2_rn(fp, Rr[i], accr[i]);
        acci[i] = __ffma2_rn(fp, Ri[i], acci[i]);
    }
}

// XPAY: out = a y - D psi; the scale a from a.ak[0] (device) when set. MINB: resident
// blocks of 128 threads the registers must allow.
template <int EPI, int MINB>
__global__ void __launch_bounds__(128, MINB) hisq_f16x2_kernel(HisqArgs a) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    df nrm = df(0.f);
    if (s < a.g.vh) {
        int c[4], xh;
        cb_coords_fast(a.g, s, a.parity, c, xh);
        const float eta[4] = {(c[3] & 1) ? -1.f : 1.f, ((c[3] + c[0]) & 1) ? -1.f : 1.f,
                              ((c[3] + c[0] + c[1]) & 1) ? -1.f : 1.f, 1.f};
        const float cn = (float)a.c_naik;
        float2 accr[3], acci[3];
#pragma unroll
        for (int i = 0; i < 3; i++) accr[i] = acci[i] = bc2(0.f);
        HPairRaw P, Q;
        hisq_fetch<0>(a, s, c, xh, P);
        hisq_fetch<1>(a, s, c, xh, Q); hisq_process<0>(a, P, eta[0], cn, accr, acci);
        hisq_fetch<2>(a, s, c, xh, P); hisq_process<1>(a, Q, eta[0], cn, accr, acci);
        hisq_fetch<3>(a, s, c, xh, Q); hisq_process<2>(a, P, eta[1], cn, accr, acci);
        hisq_fetch<4>(a, s, c, xh, P); hisq_process<3>(a, Q, eta[1], cn, accr, acci);
        hisq_fetch<5>(a, s, c, xh, Q); hisq_process<4>(a, P, eta[2], cn, accr, acci);
        hisq_fetch<6>(a, s, c, xh, P); hisq_process<5>(a, Q, eta[2], cn, accr, acci);
        hisq_fetch<7>(a, s, c, xh, Q); hisq_process<6>(a, P, eta[3], cn, accr, acci);
        hisq_process<7>(a, Q, eta[3], cn, accr, acci);
        const float half = a.dagger ? -0.5f : 0.5f;
        float v[6];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            v[2 * i] = half * (accr[i].x + accr[i].y);
            v[2 * i + 1] = half * (acci[i].x + acci[i].y);
        }
        if constexpr (EPI == EPI_XPAY) {
            float y[6];
            fload<P16, 6, float>(a.y, 0, s, y);
            const float sa = a.ak ? (float)__ldg(a.ak) : (float)a.a;
#pragma unroll
            for (int k = 0; k < 6; k++) v[k] = sa * y[k] - v[k];
        }
        if (a.norm_out) {
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < 6; q++) t = fmaf(v[q], v[q], t);
            nrm = df_of(t);
        }
        fstore<P16, 6, float>(a.out, 0, s, v);
    }
    if (a.norm_out) {
        reduce_norms_rg<1, 1>(&nrm, a.norm_out, 0, blockIdx.x, gridDim.x, 1);
        fin_tail(a.norm_out, gridDim.x, 1, a.fin);
    }
}

}  // namespace lq
