// wilson_x2.cuh -- FP16-storage Wilson hopping kernel on packed FP32 pairs.
//
// The same operator as wilson.cuh (Sec. 2.1 Eq. 2 with M = -D_w; H for dagger = 0,
// H^+ for dagger = 1) and the same fused epilogues (EPI_HOP: D psi, EPI_AINV:
// A^{-1} D psi, EPI_XPAY: A y - D psi), for one right-hand side per thread with
// FP16 fixed-point spinors and R12 links, written for the issue rate rather than
// the byte count. Three changes against the scalar kernel:
//
//  * Pairs. B300 executes two FP32 multiply-adds per instruction on register
//    pairs (fma.rn.f32x2). The two half-spinor components of a hop, h0 and h1,
//    are multiplied by the same link, so every product is formed on the pair
//    (h0, h1) with the link entry in both lanes; the spin reconstruction adds
//    pairs into the accumulators of spins (0, 1), (2, 3) and (3, 2). The clover
//    and A^{-1} epilogues act on the two chiral blocks (spins {0, 1} and {2, 3})
//    with the same 6x6 index pattern, so they run on (block 0, block 1) pairs.
//  * FP16 decode. A 16-bit code u (offset binary) becomes the float 2^23 + u
//    with one byte permute; instead of subtracting 2^23 + 32768 from every
//    decoded spinor entry, the spin projection forms P + k Q (k = +-1) from the
//    raw values and subtracts the combined offset once: exactly, because
//    (2^23 + u_Q) - 2(2^23 + 32768) is representable and the final sum is a
//    small integer.
//  * Geometry. Site coordinates come from three multiply-high divisions and the
//    eight neighbour indices from the coordinates by one compare and select
//    each, without loops or general integer division.
//
// Everything else (chunk-major storage, the FP16 codec, the per-site norms and
// the link scale folded into a per-hop factor, cp.async prefetch of the epilogue
// record and of y, two hops of gathers in flight, the block reduction of |out|^2
// finalised by the last block) is as in wilson.cuh, and the result agrees with
// it to FP32 rounding.
#pragma once
#include "wilson.cuh"

namespace lq {

#define LQ_MAG2 16842752.0f  // 2 (2^23 + 32768): two offsets of the FP16 decode

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float raw_lo(int w) { return __int_as_float((int)__byte_perm((unsigned)w, 0x4B000000u, 0x7610)); }
__device__ __forceinline__ float raw_hi(int w) { return __int_as_float((int)__byte_perm((unsigned)w, 0x4B000000u, 0x7632)); }

// q_P + k q_Q per lane from raw decodes FP, FQ (k = +-1, compile-time): FQ minus the
// offset of the lanes with k = +1 first, so that every step is exact
template <int K0, int K1>
__device__ __forceinline__ float2 proj2(float2 FP, float2 FQ) {
    const float2 off = make_float2(K0 > 0 ? -LQ_MAG2 : 0.f, K1 > 0 ? -LQ_MAG2 : 0.f);
    const float2 k = make_float2((float)K0, (float)K1);
    return __ffma2_rn(__fadd2_rn(FQ, off), k, FP);
}

// coordinates of site cb of parity p by multiply-high divisions (Geo::fdiv)
__device__ __forceinline__ int fdiv_u(int n, unsigned m) { return m ? (int)__umulhi((unsigned)n, m) : n; }
__device__ __forceinline__ void cb_coords_fast(const Geo& g, int cb, int p, int c[4], int& xh) {
    const int q1 = fdiv_u(cb, g.fdiv[0]);
    xh = cb - q1 * g.lxh;
    const int q2 = fdiv_u(q1, g.fdiv[1]);
    c[1] = q1 - q2 * g.L[1];
    c[3] = fdiv_u(q2, g.fdiv[2]);
    c[2] = q2 - c[3] * g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

// checkerboard index of the neighbour x +- mu (one hop) and its time-boundary sign
template <int MU, bool FWD>
__device__ __forceinline__ int cb_nb(const Geo& g, int s, const int c[4], int xh, float& bs) {
    bs = 1.f;
    if constexpr (MU == 0) {
        const int b = c[0] & 1;  // x = 2 xh + b
        if constexpr (FWD) return b == 0 ? s : (xh == g.lxh - 1 ? s - (g.lxh - 1) : s + 1);
        else return b == 1 ? s : (xh == 0 ? s + (g.lxh - 1) : s - 1);
    } else {
        const int stride = MU == 1 ? g.lxh : (MU == 2 ? g.lxh * g.L[1] : g.lxh * g.L[1] * g.L[2]);
        const int L = g.L[MU];
        if constexpr (FWD) {
            const bool wrap = c[MU] == L - 1;
            if (MU == 3 && wrap) bs = (float)g.bc_t;
            return wrap ? s - (L - 1) * stride : s + stride;
        } else {
            const bool wrap = c[MU] == 0;
            if (MU == 3 && wrap) bs = (float)g.bc_t;
            return wrap ? s + (L - 1) * stride : s - stride;
        }
    }
}

// raw chunks of one hop: neighbour spinor (3 x int4) + its norm, link (3 x int2)
struct HopRaw16 {
    int4 sp[3];
    int2 u[3];
    float n;
    float bs;
};

// CG: spinor loads through L2 only (ld.global.cg) instead of the read-only path, for a
// kernel that also writes the field it reads (the persistent CG kernel)
template <int H, bool CG = false>
__device__ __forceinline__ void fetch16(const WilsonArgs& a, int s, const int c[4], int xh, HopRaw16& h) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    const int n = cb_nb<MU, FWD>(a.g, s, c, xh, h.bs);
    const int4* sb = (const int4*)a.in.data;
    const size_t vh = (size_t)a.g.vh;
#pragma unroll
    if constexpr (CG) {
#pragma unroll
        for (int k = 0; k < 3; k++) h.sp[k] = __ldcg(&sb[k * vh + n]);
        h.n = __ldcg(a.in.norm + n);
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) h.sp[k] = __ldg(&sb[k * vh + n]);
        h.n = __ldg(a.in.norm + n);
    }
    const int lp = FWD ? a.parity : 1 - a.parity;
    const int2* ub = (const int2*)a.U.data + (size_t)(lp * 4 + MU) * 3 * vh;
    const int ls = FWD ? s : n;
#pragma unroll
    for (int k = 0; k < 3; k++) h.u[k] = __ldg(&ub[k * vh + ls]);
}

// accumulators: spins (0, 1), (2, 3) and (3, 2) as pairs, per colour, real and imaginary parts
struct Acc2 {
    float2 a01r[3], a01i[3], a23r[3], a23i[3], a32r[3], a32i[3];
};

// the word (spin s, colour c) of a spinor's 12 words (re in the low half, im in the high half)
__device__ __forceinline__ int spw(const int4 sp[3], int s, int c) {
    const int w = 3 * s + c;
    const int4 q = sp[w >> 2];
    const int r = w & 3;
    return r == 0 ? q.x : (r == 1 ? q.y : (r == 2 ? q.z : q.w));
}

// An R12 FP16 link as integer codes: rows 0 and 1 as stored, row 2 = conj(row 0 x row 1)
// of the codes, which is one factor scale/32767 short of the other rows' units (the
// caller applies it to the row-2 result, or to the component row 2 multiplies)
__device__ __forceinline__ void decode_r12_codes(const int2 u[3], cx<float> U[3][3]) {
    float lv[12];
#pragma unroll
    for (int k = 0; k < 3; k++) unpack_codes16<12, float>(u[k], lv + 4 * k);
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 3; q++) U[r][q] = mk(lv[(r * 3 + q) * 2], lv[(r * 3 + q) * 2 + 1]);
    U[2][0] = cj(U[0][1] * U[1][2] - U[0][2] * U[1][1]);
    U[2][1] = cj(U[0][2] * U[1][0] - U[0][0] * U[1][2]);
    U[2][2] = cj(U[0][0] * U[1][1] - U[0][1] * U[1][0]);
}

template <int H, bool DAG>
__device__ __forceinline__ void process16(const WilsonArgs& a, const HopRaw16& h, Acc2& A) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    constexpr int SF = DAG ? -1 : 1;
    constexpr int SP = FWD ? SF : -SF;  // projector (1 + SP g_mu)
    // spins paired with 0 and 1 in the projection, and the lane coefficients
    constexpr int QA = MU < 2 ? 3 : 2, QB = MU < 2 ? 2 : 3;
    constexpr bool ISI = (MU == 0 || MU == 2);
    constexpr int C0 = MU == 0 ? SP : (MU == 1 ? -SP : SP);
    constexpr int C1 = MU == 0 ? SP : (MU == 1 ? SP : (MU == 2 ? -SP : SP));
    // h = P + c Q (real c) or P + i c Q:  re = P.re - c Q.im,  im = P.im + c Q.re
    float2 Hr[3], Hi[3];
#pragma unroll
    for (int col = 0; col < 3; col++) {
        const int w0 = spw(h.sp, 0, col), w1 = spw(h.sp, 1, col);
        const int wa = spw(h.sp, QA, col), wb = spw(h.sp, QB, col);
        const float2 Pr = make_float2(raw_lo(w0), raw_lo(w1)), Pi = make_float2(raw_hi(w0), raw_hi(w1));
        const float2 Qr = make_float2(raw_lo(wa), raw_lo(wb)), Qi = make_float2(raw_hi(wa), raw_hi(wb));
        if constexpr (ISI) {
            Hr[col] = proj2<-C0, -C1>(Pr, Qi);
            Hi[col] = proj2<C0, C1>(Pi, Qr);
        } else {
            Hr[col] = proj2<C0, C1>(Pr, Qr);
            Hi[col] = proj2<C0, C1>(Pi, Qi);
        }
    }
    // per-hop factor: spinor norm / 32767, link scale / 32767, time-boundary sign
    const float fu = a.U.scale * (1.f / 32767.f);
    const float sg = h.n * (1.f / 32767.f) * fu * (MU == 3 ? h.bs : 1.f);
#pragma unroll
    for (int col = 0; col < 3; col++) {
        Hr[col] = __fmul2_rn(Hr[col], bc2(sg));
        Hi[col] = __fmul2_rn(Hi[col], bc2(sg));
    }
    // link (integer codes; the third row's missing factor goes on row 2 of U h, or on
    // component 2 of h for U^+ h)
    cx<float> U[3][3];
    decode_r12_codes(h.u, U);
    float2 Rr[3], Ri[3];
    if constexpr (!FWD) {
        Hr[2] = __fmul2_rn(Hr[2], bc2(fu));
        Hi[2] = __fmul2_rn(Hi[2], bc2(fu));
    }
    if constexpr (FWD) {  // r = U h
        float2 NHi[3];
#pragma unroll
        for (int b = 0; b < 3; b++) NHi[b] = __fmul2_rn(Hi[b], bc2(-1.f));
#pragma unroll
        for (int r = 0; r < 3; r++) {
            Rr[r] = __fmul2_rn(bc2(U[r][0].r), Hr[0]);
            Ri[r] = __fmul2_rn(bc2(U[r][0].r), Hi[0]);
            Rr[r] = __ffma2_rn(bc2(U[r][0].i), NHi[0], Rr[r]);
            Ri[r] = __ffma2_rn(bc2(U[r][0].i), Hr[0], Ri[r]);
#pragma unroll
            for (int b = 1; b < 3; b++) {
                Rr[r] = __ffma2_rn(bc2(U[r][b].r), Hr[b], Rr[r]);
                Ri[r] = __ffma2_rn(bc2(U[r][b].r), Hi[b], Ri[r]);
                Rr[r] = __ffma2_rn(bc2(U[r][b].i), NHi[b], Rr[r]);
                Ri[r] = __ffma2_rn(bc2(U[r][b].i), Hr[b], Ri[r]);
            }
        }
        Rr[2] = __fmul2_rn(Rr[2], bc2(fu));
        Ri[2] = __fmul2_rn(Ri[2], bc2(fu));
    } else {  // r = U^+ h
        float2 NHr[3];
#pragma unroll
        for (int b = 0; b < 3; b++) NHr[b] = __fmul2_rn(Hr[b], bc2(-1.f));
#pragma unroll
        for (int r = 0; r < 3; r++) {
            Rr[r] = __fmul2_rn(bc2(U[0][r].r), Hr[0]);
            Ri[r] = __fmul2_rn(bc2(U[0][r].r), Hi[0]);
            Rr[r] = __ffma2_rn(bc2(U[0][r].i), Hi[0], Rr[r]);
            Ri[r] = __ffma2_rn(bc2(U[0][r].i), NHr[0], Ri[r]);
#pragma unroll
            for (int b = 1; b < 3; b++) {
                Rr[r] = __ffma2_rn(bc2(U[b][r].r), Hr[b], Rr[r]);
                Ri[r] = __ffma2_rn(bc2(U[b][r].r), Hi[b], Ri[r]);
                Rr[r] = __ffma2_rn(bc2(U[b][r].i), Hi[b], Rr[r]);
                Ri[r] = __ffma2_rn(bc2(U[b][r].i), NHr[b], Ri[r]);
            }
        }
    }
    // reconstruction: spins 0, 1 get (r0, r1); the lower spins per mu (see recon_acc)
#pragma unroll
    for (int col = 0; col < 3; col++) {
        A.a01r[col] = __fadd2_rn(A.a01r[col], Rr[col]);
        A.a01i[col] = __fadd2_rn(A.a01i[col], Ri[col]);
        if constexpr (MU == 0) {         // (spin3, spin2) += -SP i (r0, r1)
            A.a32r[col] = __ffma2_rn(bc2((float)SP), Ri[col], A.a32r[col]);
            A.a32i[col] = __ffma2_rn(bc2((float)-SP), Rr[col], A.a32i[col]);
        } else if constexpr (MU == 1) {  // (spin3, spin2) += (-SP r0, SP r1)
            A.a32r[col] = __ffma2_rn(make_float2((float)-SP, (float)SP), Rr[col], A.a32r[col]);
            A.a32i[col] = __ffma2_rn(make_float2((float)-SP, (float)SP), Ri[col], A.a32i[col]);
        } else if constexpr (MU == 2) {  // (spin2, spin3) += i (-SP r0, SP r1)
            A.a23r[col] = __ffma2_rn(make_float2((float)SP, (float)-SP), Ri[col], A.a23r[col]);
            A.a23i[col] = __ffma2_rn(make_float2((float)-SP, (float)SP), Rr[col], A.a23i[col]);
        } else {                         // (spin2, spin3) += SP (r0, r1)
            A.a23r[col] = __ffma2_rn(bc2((float)SP), Rr[col], A.a23r[col]);
            A.a23i[col] = __ffma2_rn(bc2((float)SP), Ri[col], A.a23i[col]);
        }
    }
}

// the eight hops, software-pipelined with DEPTH (1 or 2) hops of gathers in flight
template <bool DAG, bool CG, int DEPTH>
__device__ __forceinline__ void hops16(const WilsonArgs& a, int s, const int c[4], int xh, Acc2& A) {
    if constexpr (DEPTH == 2) {
        HopRaw16 P, Q, R;
        fetch16<0, CG>(a, s, c, xh, P);
        fetch16<1, CG>(a, s, c, xh, Q);
        fetch16<2, CG>(a, s, c, xh, R); process16<0, DAG>(a, P, A);
        fetch16<3, CG>(a, s, c, xh, P); process16<1, DAG>(a, Q, A);
        fetch16<4, CG>(a, s, c, xh, Q); process16<2, DAG>(a, R, A);
        fetch16<5, CG>(a, s, c, xh, R); process16<3, DAG>(a, P, A);
        fetch16<6, CG>(a, s, c, xh, P); process16<4, DAG>(a, Q, A);
        fetch16<7, CG>(a, s, c, xh, Q); process16<5, DAG>(a, R, A);
        process16<6, DAG>(a, P, A);
        process16<7, DAG>(a, Q, A);
    } else {
        HopRaw16 P, Q;
        fetch16<0, CG>(a, s, c, xh, P);
        fetch16<1, CG>(a, s, c, xh, Q); process16<0, DAG>(a, P, A);
        fetch16<2, CG>(a, s, c, xh, P); process16<1, DAG>(a, Q, A);
        fetch16<3, CG>(a, s, c, xh, Q); process16<2, DAG>(a, P, A);
        fetch16<4, CG>(a, s, c, xh, P); process16<3, DAG>(a, Q, A);
        fetch16<5, CG>(a, s, c, xh, Q); process16<4, DAG>(a, P, A);
        fetch16<6, CG>(a, s, c, xh, P); process16<5, DAG>(a, Q, A);
        fetch16<7, CG>(a, s, c, xh, Q); process16<6, DAG>(a, P, A);
        process16<7, DAG>(a, Q, A);
    }
}

// A 24-real record of block pairs: w[j] = (block 0 entry j, block 1 entry j), j = 3 spin' + colour
struct Blk2 {
    float2 r[6], i[6];
};

// the 6x6 complex entry e (0..35) of both blocks of a 144-real A^{-1} record in shared
// memory (18 int4 chunks, chunk k of slot g at k * spb + g), decoded to raw floats
__device__ __forceinline__ void ainv_entry_raw(const int4* rec, int spb, int g, int e, float2& re, float2& im) {
    const int4 c0 = rec[(e >> 2) * spb + g];
    const int4 c1 = rec[((e + 36) >> 2) * spb + g];
    const int r = e & 3;
    const int w0 = r == 0 ? c0.x : (r == 1 ? c0.y : (r == 2 ? c0.z : c0.w));
    const int w1 = r == 0 ? c1.x : (r == 1 ? c1.y : (r == 2 ? c1.z : c1.w));
    re = make_float2(raw_lo(w0), raw_lo(w1));
    im = make_float2(raw_hi(w0), raw_hi(w1));
}

// out = A^{-1} w on both blocks (DAG: (A^{-1})^+ w); w already carries the record's scale
template <bool DAG>
__device__ __forceinline__ void ainv_pairs(const int4* rec, int spb, int g, const Blk2& w, Blk2& out) {
    const float2 mag = bc2(-0.5f * LQ_MAG2);
    Blk2 nw;
#pragma unroll
    for (int j = 0; j < 6; j++) { nw.r[j] = __fmul2_rn(w.r[j], bc2(-1.f)); nw.i[j] = __fmul2_rn(w.i[j], bc2(-1.f)); }
#pragma unroll
    for (int i = 0; i < 6; i++) { out.r[i] = bc2(0.f); out.i[i] = bc2(0.f); }
#pragma unroll
    for (int e = 0; e < 36; e++) {
        float2 mr, mi;
        ainv_entry_raw(rec, spb, g, e, mr, mi);
        mr = __fadd2_rn(mr, mag);
        mi = __fadd2_rn(mi, mag);
        const int i = e / 6, j = e % 6;
        if constexpr (!DAG) {  // out_i += m_ij w_j
            out.r[i] = __ffma2_rn(mr, w.r[j], out.r[i]);
            out.r[i] = __ffma2_rn(mi, nw.i[j], out.r[i]);
            out.i[i] = __ffma2_rn(mr, w.i[j], out.i[i]);
            out.i[i] = __ffma2_rn(mi, w.r[j], out.i[i]);
        } else {               // out_j += conj(m_ij) w_i
            out.r[j] = __ffma2_rn(mr, w.r[i], out.r[j]);
            out.r[j] = __ffma2_rn(mi, w.i[i], out.r[j]);
            out.i[j] = __ffma2_rn(mr, w.i[i], out.i[j]);
            out.i[j] = __ffma2_rn(mi, nw.r[i], out.i[j]);
        }
    }
}

// real r (0..35) of both blocks of a 72-real clover record in shared memory (9 int4 chunks)
__device__ __forceinline__ float2 clov_real_raw(const int4* rec, int spb, int g, int r) {
    const int w0i = r >> 1, w1i = (r + 36) >> 1;
    const int4 c0 = rec[(w0i >> 2) * spb + g];
    const int4 c1 = rec[(w1i >> 2) * spb + g];
    const int q0 = w0i & 3, q1 = w1i & 3;
    const int x0 = q0 == 0 ? c0.x : (q0 == 1 ? c0.y : (q0 == 2 ? c0.z : c0.w));
    const int x1 = q1 == 0 ? c1.x : (q1 == 1 ? c1.y : (q1 == 2 ? c1.z : c1.w));
    return make_float2((r & 1) ? raw_hi(x0) : raw_lo(x0), (r & 1) ? raw_hi(x1) : raw_lo(x1));
}

// out += C y on both blocks: per block 6 real diagonal entries, then the 15 upper entries (i < j)
__device__ __forceinline__ void clover_pairs(const int4* rec, int spb, int g, const Blk2& y, Blk2& out) {
    const float2 mag = bc2(-0.5f * LQ_MAG2);
    Blk2 ny;
#pragma unroll
    for (int j = 0; j < 6; j++) { ny.r[j] = __fmul2_rn(y.r[j], bc2(-1.f)); ny.i[j] = __fmul2_rn(y.i[j], bc2(-1.f)); }
#pragma unroll
    for (int d = 0; d < 6; d++) {
        const float2 cd = __fadd2_rn(clov_real_raw(rec, spb, g, d), mag);
        out.r[d] = __ffma2_rn(cd, y.r[d], out.r[d]);
        out.i[d] = __ffma2_rn(cd, y.i[d], out.i[d]);
    }
#pragma unroll
    for (int q = 0; q < 15; q++) {
        const int i = offd_row(q), j = offd_col(q);
        const float2 er = __fadd2_rn(clov_real_raw(rec, spb, g, 6 + 2 * q), mag);
        const float2 ei = __fadd2_rn(clov_real_raw(rec, spb, g, 7 + 2 * q), mag);
        // out_i += e y_j
        out.r[i] = __ffma2_rn(er, y.r[j], out.r[i]);
        out.r[i] = __ffma2_rn(ei, ny.i[j], out.r[i]);
        out.i[i] = __ffma2_rn(er, y.i[j], out.i[i]);
        out.i[i] = __ffma2_rn(ei, y.r[j], out.i[i]);
        // out_j += conj(e) y_i
        out.r[j] = __ffma2_rn(er, y.r[i], out.r[j]);
        out.r[j] = __ffma2_rn(ei, y.i[i], out.r[j]);
        out.i[j] = __ffma2_rn(er, y.i[i], out.i[j]);
        out.i[j] = __ffma2_rn(ei, ny.r[i], out.i[j]);
    }
}

// FP16 store of 24 reals given as block pairs: per-site norm = max |v|, codes by one FMA each
__device__ __forceinline__ void store16_blk(const WilsonArgs& a, int s, const Blk2& v) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 6; j++)
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.r[j].x), fabsf(v.r[j].y)), fmaxf(fabsf(v.i[j].x), fabsf(v.i[j].y))));
    a.out.norm[s] = m;
    const float f = m > 0.f ? __fdividef(32767.f, m) : 0.f;
    int w[12];  // word (spin, colour): block b = spin / 2, j = 3 (spin % 2) + colour
#pragma unroll
    for (int j = 0; j < 6; j++) {
        const float2 cr = __ffma2_rn(v.r[j], bc2(f), bc2(LQ_F16_MAGIC));
        const float2 ci = __ffma2_rn(v.i[j], bc2(f), bc2(LQ_F16_MAGIC));
        w[j] = (int)__byte_perm(__float_as_uint(cr.x), __float_as_uint(ci.x), 0x5410);      // block 0
        w[6 + j] = (int)__byte_perm(__float_as_uint(cr.y), __float_as_uint(ci.y), 0x5410);  // block 1
    }
    int4* ob = (int4*)a.out.data;
    const size_t vh = (size_t)a.g.vh;
    ob[0 * vh + s] = make_int4(w[0], w[1], w[2], w[3]);
    ob[1 * vh + s] = make_int4(w[4], w[5], w[6], w[7]);
    ob[2 * vh + s] = make_int4(w[8], w[9], w[10], w[11]);
}

// the shared-memory views of x2_site's epilogue records
#define LQ_X2_SMEM_VIEWS \
    constexpr int NREC = EPI == EPI_AINV ? 18 : (EPI == EPI_XPAY ? 9 : 0); /* int4 chunks of the record */ \
    int4* sm_rec = (int4*)smem; \
    int4* sm_y = sm_rec + NREC * spb_rec; \
    float* sm_norm = (float*)(sm_y + (EPI == EPI_XPAY ? 3 : 0) * spb); /* [spb_rec] record, [spb] y norms */ \
    (void)sm_y; (void)sm_norm

// x2_site, step 1: asynchronous copies of the site's epilogue record (and y) into shared memory
template <int EPI, bool CG = false, int RG = 1>
__device__ __forceinline__ void x2_record(const WilsonArgs& a, int s, int g_rec, int spb_rec, int g, int spb, int lane,
                                          unsigned char* smem) {
    LQ_X2_SMEM_VIEWS;
    if constexpr (EPI != EPI_HOP) {
        const int4* gsrc = (const int4*)a.clov;
#pragma unroll
        for (int k = 0; k < NREC; k++)
            if (RG == 1 || k % RG == lane) cp_async16(&sm_rec[k * spb_rec + g_rec], &gsrc[(size_t)k * a.g.vh + s]);
        if (RG == 1 || lane == 0) cp_async4(&sm_norm[g_rec], a.clov_norm + s);
        if constexpr (EPI == EPI_XPAY) {
            const int4* ysrc = (const int4*)a.y.data;
#pragma unroll
            for (int k = 0; k < 3; k++) cp_async16(&sm_y[k * spb + g], &ysrc[(size_t)k * a.g.vh + s]);
            // (the 4-byte asynchronous copy goes through L1, which may hold stale lines of a
            // field written earlier in the same kernel)
            if constexpr (CG) sm_norm[spb_rec + g] = __ldcg(a.y.norm + s);
            else cp_async4(&sm_norm[spb_rec + g], a.y.norm + s);
        }
        cp_async_commit();
    }
}

// x2_site, step 3: the epilogue on the accumulated hops A and the FP16 store
template <int EPI, bool DAG, bool CG = false, int RG = 1>
__device__ __forceinline__ void x2_epilogue(const WilsonArgs& a, int s, int g_rec, int spb_rec, int g, int spb,
                                            unsigned gmask, unsigned char* smem, const Acc2& A, bool want_norm,
                                            bool store, df& nrm) {
    LQ_X2_SMEM_VIEWS;
    // D psi as block pairs, times 1/2: block 0 = spins (0, 1), block 1 = spins (2, 3)
    Blk2 d;
#pragma unroll
    for (int col = 0; col < 3; col++) {
        d.r[col] = make_float2(A.a01r[col].x, A.a23r[col].x + A.a32r[col].y);
        d.i[col] = make_float2(A.a01i[col].x, A.a23i[col].x + A.a32i[col].y);
        d.r[3 + col] = make_float2(A.a01r[col].y, A.a23r[col].y + A.a32r[col].x);
        d.i[3 + col] = make_float2(A.a01i[col].y, A.a23i[col].y + A.a32i[col].x);
    }
    Blk2 res;
    if constexpr (EPI == EPI_HOP) {
#pragma unroll
        for (int j = 0; j < 6; j++) { res.r[j] = __fmul2_rn(d.r[j], bc2(0.5f)); res.i[j] = __fmul2_rn(d.i[j], bc2(0.5f)); }
    } else if constexpr (EPI == EPI_AINV) {
        cp_async_wait_all();
        if constexpr (RG > 1) __syncwarp(gmask);  // the record chunks the other lanes copied
        const float f = 0.5f * sm_norm[g_rec] * (1.f / 32767.f);
#pragma unroll
        for (int j = 0; j < 6; j++) { d.r[j] = __fmul2_rn(d.r[j], bc2(f)); d.i[j] = __fmul2_rn(d.i[j], bc2(f)); }
        ainv_pairs<DAG>(sm_rec, spb_rec, g_rec, d, res);
    } else {  // A y - D psi, A = (4+m) + i mu_b + C
        cp_async_wait_all();
        if constexpr (RG > 1) __syncwarp(gmask);
        Blk2 y;
        const float fy = sm_norm[spb_rec + g] * (1.f / 32767.f);
        const float2 mag = bc2(-0.5f * LQ_MAG2);
#pragma unroll
        for (int col = 0; col < 3; col++) {
#pragma unroll
            for (int sp2 = 0; sp2 < 2; sp2++) {  // spin' within the block
                const int4 yc0 = sm_y[((3 * sp2 + col) >> 2) * spb + g];
                const int4 yc1 = sm_y[((3 * (2 + sp2) + col) >> 2) * spb + g];
                const int r0 = (3 * sp2 + col) & 3, r1 = (3 * (2 + sp2) + col) & 3;
                const int w0 = r0 == 0 ? yc0.x : (r0 == 1 ? yc0.y : (r0 == 2 ? yc0.z : yc0.w));
                const int w1 = r1 == 0 ? yc1.x : (r1 == 1 ? yc1.y : (r1 == 2 ? yc1.z : yc1.w));
                const int j = 3 * sp2 + col;
                y.r[j] = __fmul2_rn(__fadd2_rn(make_float2(raw_lo(w0), raw_lo(w1)), mag), bc2(fy));
                y.i[j] = __fmul2_rn(__fadd2_rn(make_float2(raw_hi(w0), raw_hi(w1)), mag), bc2(fy));
            }
        }
        // res = (4+m) y + i mu_b y - D psi / 2, then + C y
        const float m4 = a.m4f;
        const float2 mub = make_float2(a.muf, a.mu1f);
        const float2 nmub = make_float2(-a.muf, -a.mu1f);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            res.r[j] = __ffma2_rn(bc2(m4), y.r[j], __fmul2_rn(d.r[j], bc2(-0.5f)));
            res.r[j] = __ffma2_rn(nmub, y.i[j], res.r[j]);
            res.i[j] = __ffma2_rn(bc2(m4), y.i[j], __fmul2_rn(d.i[j], bc2(-0.5f)));
            res.i[j] = __ffma2_rn(mub, y.r[j], res.i[j]);
        }
        // the clover record's scale goes on y (C's entries stay integer codes)
        const float fc = sm_norm[g_rec] * (1.f / 32767.f);
#pragma unroll
        for (int j = 0; j < 6; j++) { y.r[j] = __fmul2_rn(y.r[j], bc2(fc)); y.i[j] = __fmul2_rn(y.i[j], bc2(fc)); }
        clover_pairs(sm_rec, spb_rec, g_rec, y, res);
    }
    if (want_norm) {
        float2 t = bc2(0.f);
#pragma unroll
        for (int j = 0; j < 6; j++) { t = __ffma2_rn(res.r[j], res.r[j], t); t = __ffma2_rn(res.i[j], res.i[j], t); }
        nrm = nrm + df_of(t.x + t.y);
    }
    if (store) store16_blk(a, s, res);
}

// One output site s: the hops, the epilogue and the FP16 store (when `store`). The
// fields of `a` are those of one right-hand side. The epilogue record of the site goes
// through record slot g_rec of the block's shared memory (spb_rec slots; with RG > 1
// the RG threads of the site share it, lane L copying the chunks k = L mod RG, and
// gmask names those threads), y through this thread's slot g (spb slots). Adds |out|^2
// to nrm when want_norm is set.
template <int EPI, bool DAG, bool CG = false, int DEPTH = 2, int RG = 1>
__device__ __forceinline__ void x2_site(const WilsonArgs& a, int s, int g_rec, int spb_rec, int g, int spb, int lane,
                                        unsigned gmask, unsigned char* smem, bool want_norm, bool store, df& nrm) {
    x2_record<EPI, CG, RG>(a, s, g_rec, spb_rec, g, spb, lane, smem);
    int c[4], xh;
    cb_coords_fast(a.g, s, a.parity, c, xh);
    Acc2 A;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        A.a01r[k] = A.a01i[k] = A.a23r[k] = A.a23i[k] = A.a32r[k] = A.a32i[k] = bc2(0.f);
    }
    hops16<DAG, CG, DEPTH>(a, s, c, xh, A);
    x2_epilogue<EPI, DAG, CG, RG>(a, s, g_rec, spb_rec, g, spb, gmask, smem, A, want_norm, store, nrm);
}

// Grid: one thread per output site, blocks of consecutive sites. DAG: the adjoint.
// The result times g5 is not provided here (the host uses wilson.cuh for it).
// MINB: resident blocks of BT threads the registers must allow; DEPTH: hops of gathers in
// flight; BT: the largest block size of the build (128 or 256).
template <int EPI, bool DAG, int MINB, int DEPTH, int BT = 128>
__global__ void __launch_bounds__(BT, MINB) wilson_f16x2_kernel(WilsonArgs a) {
    pdl_start();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    extern __shared__ __align__(16) unsigned char lq_smem[];
    df nrm = df(0.f);
    if (s < a.g.vh)
        x2_site<EPI, DAG, false, DEPTH>(a, s, threadIdx.x, blockDim.x, threadIdx.x, blockDim.x, 0, 0u, lq_smem,
                                        a.norm_out != nullptr, true, nrm);
    if (a.norm_out) {
        reduce_norms_rg<1, 1>(&nrm, a.norm_out, 0, blockIdx.x, gridDim.x, 1);
        fin_tail(a.norm_out, gridDim.x, 1, a.fin);
    }
}

// Several right-hand sides: RG consecutive threads take one site and one right-hand
// side each, so that their link loads are the same addresses (served once) and they
// share one copy of the site's clover or A^{-1} record. Blocks are ordered site block
// major, right-hand-side group minor (the groups of a site block run together and
// meet its links in L2). A group's lanes beyond the last right-hand side compute the
// last one again and store nothing, so that the whole group reaches its warp barrier.
template <int EPI, bool DAG, int MINB, int DEPTH, int RG>
__global__ void __launch_bounds__(128, MINB) wilson_f16x2_mrhs_kernel(WilsonArgs a) {
    extern __shared__ __align__(16) unsigned char lq_smem[];
    const int spb = blockDim.x / RG;
    const int ngroups = (a.nrhs + RG - 1) / RG;
    const int sb = blockIdx.x / ngroups, grp = blockIdx.x - sb * ngroups;
    const int nsb = gridDim.x / ngroups;
    const int gs = threadIdx.x / RG, lane = threadIdx.x % RG;
    const int s = sb * spb + gs;
    const int k = grp * RG + lane;
    const int kk = k < a.nrhs ? k : a.nrhs - 1;
    const unsigned gmask = ((1u << RG) - 1u) << ((threadIdx.x & 31) & ~(RG - 1));
    WilsonArgs ak = a;  // the fields of right-hand side kk
    ak.in.data = (char*)a.in.data + (size_t)kk * a.in.rhs_bytes;
    ak.in.norm = a.in.norm + (size_t)kk * a.g.vh;
    ak.out.data = (char*)a.out.data + (size_t)kk * a.out.rhs_bytes;
    ak.out.norm = a.out.norm + (size_t)kk * a.g.vh;
    ak.y.data = (char*)a.y.data + (size_t)kk * a.y.rhs_bytes;
    ak.y.norm = a.y.norm + (size_t)kk * a.g.vh;
    df nrm = df(0.f);
    if (s < a.g.vh)
        x2_site<EPI, DAG, false, DEPTH, RG>(ak, s, gs, spb, threadIdx.x, blockDim.x, lane, gmask, lq_smem,
                                            a.norm_out != nullptr && k < a.nrhs, k < a.nrhs, nrm);
    if (a.norm_out) {
        reduce_norms_rg<1, RG>(&nrm, a.norm_out, grp, sb, nsb, a.nrhs);
        fin_tail(a.norm_out, nsb, a.nrhs, a.fin);
    }
}

// shared memory of a launch with `block` threads, rg threads per site
template <int EPI>
__host__ __device__ constexpr size_t x2_smem_bytes(int block, int rg = 1) {
    return EPI == EPI_AINV   ? (size_t)(block / rg) * (18 * 16 + 4)
           : EPI == EPI_XPAY ? (size_t)(block / rg) * (9 * 16 + 4) + (size_t)block * (3 * 16 + 4)
                             : 0;
}

}  // namespace lq
