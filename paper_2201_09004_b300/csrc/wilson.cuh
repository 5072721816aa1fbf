// wilson.cuh -- Wilson hopping term with fused site-local epilogues.
//
// For output parity p, each thread takes one site x and NB right-hand sides:
//   D psi(x) = 1/2 sum_mu [(1 + s g_mu) U_mu(x) psi(x+mu) + (1 - s g_mu) U_mu(x-mu)^+ psi(x-mu)]
// with s = +1 (H, Sec. 2.1 Eq. 2 with M = -D_w) or s = -1 (H^+). Each
// neighbour is spin-projected to a half spinor (two spin components, since
// (1 +- g_mu) has rank two), multiplied by the link once per half spinor, and
// expanded back, so a hop costs 2 SU(3) mat-vecs instead of 4. The link of a
// direction is loaded once and used for all NB right-hand sides.
//
// Epilogues (A = (4+m) + i mu g5 + C is site-local, or (4+m) + i mu + C with the
// scalar twist: the twisted mass is mu on chiral block 0 and mu1 = -mu or +mu on
// block 1; both signs are flipped by the host for the adjoint, and C is hermitian):
//   EPI_HOP   out = D psi
//   EPI_AINV  out = A^{-1} D psi     (A^{-1} stored per site, or analytic without clover)
//   EPI_XPAY  out = A y - D psi      (y: same-parity input; gives M = A - H and the
//                                     Schur operator A_ee - H_eo (A_oo^{-1} H_oe v))
// Gamma basis DeGrand-Rossi, g5 = diag(1,1,-1,-1): the chiral blocks are spins
// {0,1} and {2,3}; C and A^{-1} are stored as two 6x6 blocks (index 3*spin'+colour).
#pragma once
#include "core.cuh"

namespace lq {

struct WilsonArgs {
    Geo g;
    GaugeV U;
    FieldV in, out, y;
    const void* clov;       // output parity block: C (72 reals) for XPAY, A^{-1} (144) for AINV
    const float* clov_norm; // FP16 per-site norms of that block
    int parity;             // output parity
    int dagger;
    int has_clover;
    int gamma5_out = 0;     // multiply the result by g5 (negate spins 2, 3): the hermitian g5 D_w
    double m4;              // 4 + m
    double mu;              // twisted mass on chiral block 0 (spins 0, 1), already negated for the adjoint
    double mu1;             // the same on block 1 (spins 2, 3): -mu (i mu g5) or mu (scalar twist)
    int nrhs;
    df* norm_out;       // if non-null: per-block partial sums of |out|^2, per rhs
    FinArgs fin;        // with norm_out: the last block finalises the sums
    float m4f, muf, mu1f;  // m4, mu, mu1 rounded to FP32 once on the host (FP32 kernels)
    // double-float A y - D psi only: with rb.data set the kernel writes the residual
    // out = rb - (A y - D psi) (and |out|^2 with norm_out); with lo.data set also its
    // FP16 copy into lo (codes and per-site norm as the FP16 store writes them)
    FieldV rb = {nullptr, nullptr, 0, 0};
    FieldV lo = {nullptr, nullptr, 0, 0};
};

// spin projection h = top two spins of (1 + s g_mu) psi, for psi as cx[4][3]
template <int MU, typename T>
__device__ __forceinline__ void proj(const cx<T> ps[4][3], T s, cx<T> h0[3], cx<T> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if constexpr (MU == 0) {        // g1: h0 = p0 + s i p3, h1 = p1 + s i p2
            h0[c] = ps[0][c] + s * ti(ps[3][c]);
            h1[c] = ps[1][c] + s * ti(ps[2][c]);
        } else if constexpr (MU == 1) { // g2: h0 = p0 - s p3, h1 = p1 + s p2
            h0[c] = ps[0][c] - s * ps[3][c];
            h1[c] = ps[1][c] + s * ps[2][c];
        } else if constexpr (MU == 2) { // g3: h0 = p0 + s i p2, h1 = p1 - s i p3
            h0[c] = ps[0][c] + s * ti(ps[2][c]);
            h1[c] = ps[1][c] - s * ti(ps[3][c]);
        } else {                        // g4: h0 = p0 + s p2, h1 = p1 + s p3
            h0[c] = ps[0][c] + s * ps[2][c];
            h1[c] = ps[1][c] + s * ps[3][c];
        }
    }
}

// acc += full spinor reconstructed from the rotated half spinor r0, r1
template <int MU, typename T>
__device__ __forceinline__ void recon_acc(cx<T> acc[4][3], const cx<T> r0[3], const cx<T> r1[3], T s) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[0][c] = acc[0][c] + r0[c];
        acc[1][c] = acc[1][c] + r1[c];
        if constexpr (MU == 0) {        // comp2 = -s i h1, comp3 = -s i h0
            acc[2][c] = acc[2][c] - s * ti(r1[c]);
            acc[3][c] = acc[3][c] - s * ti(r0[c]);
        } else if constexpr (MU == 1) { // comp2 = s h1, comp3 = -s h0
            acc[2][c] = acc[2][c] + s * r1[c];
            acc[3][c] = acc[3][c] - s * r0[c];
        } else if constexpr (MU == 2) { // comp2 = -s i h0, comp3 = s i h1
            acc[2][c] = acc[2][c] - s * ti(r0[c]);
            acc[3][c] = acc[3][c] + s * ti(r1[c]);
        } else {                        // comp2 = s h0, comp3 = s h1
            acc[2][c] = acc[2][c] + s * r0[c];
            acc[3][c] = acc[3][c] + s * r1[c];
        }
    }
}

template <typename T>
__device__ __forceinline__ void to_spinor(const T* v, cx<T> ps[4][3]) {
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) ps[a][c] = mk(v[(a * 3 + c) * 2], v[(a * 3 + c) * 2 + 1]);
}

template <int MU, int P, int R, int NB, typename T>
__device__ __forceinline__ void hop_dir(const WilsonArgs& a, const int c[4], int s, int kb, T sf,
                                        cx<T> acc[NB][4][3]) {
    // forward: (1 + sf g_mu) U_mu(x) psi(x+mu)
    {
        float bs;
        const int n = cb_hop(a.g, c, MU, +1, bs);
        cx<T> U[3][3];
        load_link<P, R, T>(a.U, a.parity, MU, s, U);
        const T sg = (T)bs;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            if (kb + b >= a.nrhs) break;
            T v[24];
            fload<P, 24, T>(a.in, kb + b, n, v);
            cx<T> ps[4][3], h0[3], h1[3], r0[3], r1[3];
            to_spinor(v, ps);
            proj<MU>(ps, sf, h0, h1);
            su3_mv(U, h0, r0);
            su3_mv(U, h1, r1);
            if constexpr (MU == 3) {
#pragma unroll
                for (int k = 0; k < 3; k++) { r0[k] = sg * r0[k]; r1[k] = sg * r1[k]; }
            }
            recon_acc<MU>(acc[b], r0, r1, sf);
        }
    }
    // backward: (1 - sf g_mu) U_mu(x-mu)^+ psi(x-mu)
    {
        float bs;
        const int n = cb_hop(a.g, c, MU, -1, bs);
        cx<T> U[3][3];
        load_link<P, R, T>(a.U, 1 - a.parity, MU, n, U);
        const T sg = (T)bs;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            if (kb + b >= a.nrhs) break;
            T v[24];
            fload<P, 24, T>(a.in, kb + b, n, v);
            cx<T> ps[4][3], h0[3], h1[3], r0[3], r1[3];
            to_spinor(v, ps);
            proj<MU>(ps, -sf, h0, h1);
            su3_dmv(U, h0, r0);
            su3_dmv(U, h1, r1);
            if constexpr (MU == 3) {
#pragma unroll
                for (int k = 0; k < 3; k++) { r0[k] = sg * r0[k]; r1[k] = sg * r1[k]; }
            }
            recon_acc<MU>(acc[b], r0, r1, -sf);
        }
    }
}

// element j of the chiral 6-vector of block bl: spin 2*bl + j/3, colour j%3
template <typename T>
__device__ __forceinline__ cx<T>& blk(cx<T> v[4][3], int bl, int j) { return v[2 * bl + j / 3][j % 3]; }

// (i, j) of the q-th upper off-diagonal entry of a 6x6 matrix, row-major, i < j
__host__ __device__ constexpr int offd_row(int q) { return q < 5 ? 0 : q < 9 ? 1 : q < 12 ? 2 : q < 14 ? 3 : 4; }
__host__ __device__ constexpr int offd_col(int q) {
    return q < 5 ? 1 + q : q < 9 ? 2 + (q - 5) : q < 12 ? 3 + (q - 9) : q < 14 ? 4 + (q - 12) : 5;
}

// out_b += C_b w_b for both chiral blocks, C packed per block as 6 real
// diagonal entries then the 15 upper off-diagonal entries (row-major, i<j).
// The record is read from base[k * stride + s] (global, or a shared-memory copy).
// FP16: the entries are decoded to their integer codes and the site's scale
// (norm / 32767) multiplies the 24 reals of w once instead of every entry
// (w is scaled in place: callers pass an operand they no longer need).
template <int P, int NB, typename T>
__device__ __forceinline__ void scale_codes16(float sc, cx<T> w[NB][4][3]) {
    if constexpr (P == P16) {
        const T f = (T)(sc * (1.f / 32767.f));
#pragma unroll
        for (int b = 0; b < NB; b++)
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int q = 0; q < 3; q++) w[b][sp][q] = f * w[b][sp][q];
    }
}

template <int P, int NB, typename T, bool SMEM = false>
__device__ __forceinline__ void clover_apply_src(const void* base, int stride, int s, float sc, cx<T> w[NB][4][3],
                                                 cx<T> out[NB][4][3]) {
    typedef Layout<P, 72> Lay;
    scale_codes16<P, NB, T>(sc, w);
#pragma unroll
    for (int k = 0; k < Lay::NC; k++) {
        T v[Lay::RPC];
        load_chunk<P, 72, T, SMEM, true>(base, stride, s, k, sc, v);
#pragma unroll
        for (int u = 0; u < Lay::RPC / 2; u++) {
            const int r = k * Lay::RPC + 2 * u;  // real index of this pair
            const int bl = r / 36;
            const int l = r - 36 * bl;
            if (l < 6) {
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    blk(out[b], bl, l) = blk(out[b], bl, l) + v[2 * u] * blk(w[b], bl, l);
                    blk(out[b], bl, l + 1) = blk(out[b], bl, l + 1) + v[2 * u + 1] * blk(w[b], bl, l + 1);
                }
            } else {
                const int q = (l - 6) / 2;
                const int i = offd_row(q), j = offd_col(q);
                const cx<T> e = mk(v[2 * u], v[2 * u + 1]);
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    cmac(blk(out[b], bl, i), e, blk(w[b], bl, j));
                    cjmac(blk(out[b], bl, j), e, blk(w[b], bl, i));
                }
            }
        }
    }
}

template <int P, int NB, typename T>
__device__ __forceinline__ void clover_apply(const WilsonArgs& a, int s, cx<T> w[NB][4][3], cx<T> out[NB][4][3]) {
    const float sc = (P == P16) ? __ldg(a.clov_norm + s) : 1.f;
    clover_apply_src<P, NB, T, false>(a.clov, a.g.vh, s, sc, w, out);
}

// out_b = A^{-1}_b w_b (dagger: (A^{-1}_b)^+ w_b), A^{-1} stored row-major per block (36 complex)
template <int P, int NB, typename T, bool SMEM = false>
__device__ __forceinline__ void ainv_apply_src(const void* base, int stride, int s, float sc, int dagger,
                                               cx<T> w[NB][4][3], cx<T> out[NB][4][3]) {
    typedef Layout<P, 144> Lay;
    scale_codes16<P, NB, T>(sc, w);  // w scaled in place, entries as integer codes
#pragma unroll
    for (int k = 0; k < Lay::NC; k++) {
        T v[Lay::RPC];
        load_chunk<P, 144, T, SMEM, true>(base, stride, s, k, sc, v);
#pragma unroll
        for (int u = 0; u < Lay::RPC / 2; u++) {
            const int e = (k * Lay::RPC) / 2 + u;
            const int bl = e / 36;
            const int i = (e % 36) / 6;
            const int j = e % 6;
            const cx<T> m = mk(v[2 * u], v[2 * u + 1]);
#pragma unroll
            for (int b = 0; b < NB; b++) {
                if (dagger)
                    cjmac(blk(out[b], bl, j), m, blk(w[b], bl, i));
                else
                    cmac(blk(out[b], bl, i), m, blk(w[b], bl, j));
            }
        }
    }
}

template <int P, int NB, typename T>
__device__ __forceinline__ void ainv_apply(const WilsonArgs& a, int s, cx<T> w[NB][4][3], cx<T> out[NB][4][3]) {
    const float sc = (P == P16) ? __ldg(a.clov_norm + s) : 1.f;
    ainv_apply_src<P, NB, T, false>(a.clov, a.g.vh, s, sc, a.dagger, w, out);
}

// Block reduction of the per-thread |out|^2 (double-float) when RG consecutive
// threads share a site, one right-hand side each (NB = 1), or one thread
// carries NB right-hand sides (RG = 1). The per-block partial of right-hand
// side k goes to norm_out[k * nsb + sb], sb the site block and nsb the number
// of site blocks.
template <int NB, int RG>
__device__ __forceinline__ void reduce_norms_rg(const df nrm[NB], df* norm_out, int grp, int sb, int nsb, int nrhs) {
    static_assert(NB == 1 || RG == 1, "right-hand sides are spread over threads or registers, not both");
    __shared__ float2 red[NB * RG][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int b = 0; b < NB; b++) {
        df v = nrm[b];
#pragma unroll
        for (int o = 16; o >= RG; o >>= 1) v = v + shfl_down_df(v, o);
        if (lane < RG) red[b * RG + lane][wid] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < NB * RG; q++) {
            df v = lane < nw ? df(red[q][lane].x, red[q][lane].y) : df(0.f);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = v + shfl_down_df(v, o);
            const int k = (grp * RG + (q % RG)) * NB + q / RG;
            if (lane == 0 && k < nrhs) norm_out[(size_t)k * nsb + sb] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Compact hop loop for the double-float precision: one copy of the hop body
// runs for all eight hops (no unrolling), with the spin projection driven by a
// small table, because the fully unrolled double-float code does not fit in the
// instruction cache. (1 +- g_mu) in the DeGrand-Rossi basis couples spin 0 with
// spin a and spin 1 with spin b through a unit coefficient (+-1 or +-i), and the
// lower spins are rebuilt from the rotated half spinor the same way.

// v * (sgn * (i if isi else 1))
template <typename T>
__device__ __forceinline__ cx<T> cunit(cx<T> v, bool neg, bool isi) {
    cx<T> w = isi ? mk(-v.i, v.r) : v;
    return neg ? mk(-w.r, -w.i) : w;
}

template <int P, int R, typename T>
__device__ void hop_compact(const WilsonArgs& a, const int c[4], int s, int k0, int h, T sf, cx<T> acc[4][3]) {
    const int mu = h >> 1;
    const bool fwd = (h & 1) == 0;
    float bs;
    const int n = cb_hop(a.g, c, mu, fwd ? 1 : -1, bs);
    cx<T> U[3][3];
    load_link<P, R, T>(a.U, fwd ? a.parity : 1 - a.parity, mu, fwd ? s : n, U);
    T v[24];
    fload<P, 24, T>(a.in, k0, n, v);
    cx<T> ps[4][3];
    to_spinor(v, ps);
    // projector (1 + sp g_mu): sp = sf forward, -sf backward; `neg` flips the sign of sp
    const bool neg_sp = fwd ? (a.dagger != 0) : (a.dagger == 0);
    (void)sf;
    // table per mu: spin a / b coupled to 0 / 1, coefficients c0, c1 (as sign, is-i),
    // and the rebuild of spins 2 and 3 from (r0, r1)
    const int ia = (mu < 2) ? 3 : 2, ib = (mu < 2) ? 2 : 3;
    const bool c0i = (mu == 0 || mu == 2), c1i = c0i;
    const bool c0n = (mu == 1), c1n = (mu == 2);
    cx<T> h0[3], h1[3], r0[3], r1[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const cx<T> pa = ia == 3 ? ps[3][q] : ps[2][q];
        const cx<T> pb = ib == 3 ? ps[3][q] : ps[2][q];
        h0[q] = ps[0][q] + cunit(pa, c0n != neg_sp, c0i);
        h1[q] = ps[1][q] + cunit(pb, c1n != neg_sp, c1i);
    }
    if (fwd) {
        su3_mv(U, h0, r0);
        su3_mv(U, h1, r1);
    } else {
        su3_dmv(U, h0, r0);
        su3_dmv(U, h1, r1);
    }
    const bool flip = bs < 0.f;  // time boundary
    // spin 2 gets e2 * r_{j2}, spin 3 gets e3 * r_{j3}:
    //   mu0: -i r1, -i r0;  mu1: +r1, -r0;  mu2: -i r0, +i r1;  mu3: +r0, +r1  (times sp)
    const bool j2is1 = mu < 2, j3is1 = mu >= 2;
    const bool e2i = (mu == 0 || mu == 2), e3i = e2i;
    const bool e2n = (mu == 0 || mu == 2), e3n = (mu == 0 || mu == 1);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        cx<T> a0 = flip ? mk(-r0[q].r, -r0[q].i) : r0[q];
        cx<T> a1 = flip ? mk(-r1[q].r, -r1[q].i) : r1[q];
        acc[0][q] = acc[0][q] + a0;
        acc[1][q] = acc[1][q] + a1;
        acc[2][q] = acc[2][q] + cunit(j2is1 ? a1 : a0, e2n != neg_sp, e2i);
        acc[3][q] = acc[3][q] + cunit(j3is1 ? a1 : a0, e3n != neg_sp, e3i);
    }
}

// Compact site-local epilogues for double-float (one right-hand side): a loop
// over the twelve output rows with only the six-term row product unrolled.
template <typename T>
__device__ __forceinline__ cx<T> wsel(cx<T> w[4][3], int bl, int j) {
    return bl ? blk(w, 1, j) : blk(w, 0, j);
}

// out = A^{-1} w (dagger: (A^{-1})^+ w); A^{-1}: 36 complex per block, row-major
template <int P, typename T>
__device__ void ainv_apply_rows(const WilsonArgs& a, int s, cx<T> w[4][3], cx<T> out[4][3]) {
    typedef Layout<P, 144> Lay;
    static_assert(Lay::RPC == 2, "one complex entry per chunk");
    const typename Lay::C* base = (const typename Lay::C*)a.clov;
    cx<T> o[12];
#pragma unroll 1
    for (int r = 0; r < 12; r++) {
        const int bl = r / 6, i = r - 6 * bl;
        cx<T> acc = mk((T)0, (T)0);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const int e = a.dagger ? bl * 36 + j * 6 + i : bl * 36 + i * 6 + j;
            T m[2];
            unpack_chunk<P, 144, T>(__ldg(&base[(size_t)e * a.g.vh + s]), 1.f, m);
            const cx<T> me = mk(m[0], m[1]);
            if (a.dagger) cjmac(acc, me, wsel(w, bl, j));
            else cmac(acc, me, wsel(w, bl, j));
        }
        o[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 12; r++) blk(out, r / 6, r % 6) = o[r];
}

// out += C w; C per block: 6 real diagonal entries then 15 upper entries (row-major, i<j)
template <int P, typename T>
__device__ void clover_apply_rows(const WilsonArgs& a, int s, cx<T> w[4][3], cx<T> out[4][3]) {
    typedef Layout<P, 72> Lay;
    static_assert(Lay::RPC == 2, "two reals per chunk");
    const typename Lay::C* base = (const typename Lay::C*)a.clov;
    cx<T> o[12];
#pragma unroll 1
    for (int r = 0; r < 12; r++) {
        const int bl = r / 6, i = r - 6 * bl;
        T d[2];
        unpack_chunk<P, 72, T>(__ldg(&base[(size_t)(18 * bl + i / 2) * a.g.vh + s]), 1.f, d);
        const T di = (i & 1) ? d[1] : d[0];
        cx<T> acc = di * wsel(w, bl, i);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            if (j == i) continue;
            const int lo = j < i ? j : i, hi = j < i ? i : j;
            const int q = lo * 5 - lo * (lo - 1) / 2 + (hi - lo - 1);
            T m[2];
            unpack_chunk<P, 72, T>(__ldg(&base[(size_t)(18 * bl + 3 + q) * a.g.vh + s]), 1.f, m);
            const cx<T> me = mk(m[0], m[1]);
            if (i < j) cmac(acc, me, wsel(w, bl, j));
            else cjmac(acc, me, wsel(w, bl, j));
        }
        o[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 12; r++) blk(out, r / 6, r % 6) = blk(out, r / 6, r % 6) + o[r];
}

// ---------------------------------------------------------------------------
// Single right-hand side: the eight hops are software-pipelined. The raw
// (still encoded) spinor and link chunks of hop h+1 are loaded before hop h is
// decoded and computed, so every thread keeps one hop of gathers in flight
// while it computes; the epilogue operands are copied to shared memory with
// cp.async at kernel start and arrive while the hops are computed.
template <int P, int R> struct HopRaw {
    typename Layout<P, 24>::C sp[Layout<P, 24>::NC];
    typename Layout<P, R>::C u[Layout<P, R>::NC];
    float n;   // FP16 spinor norm
    float bs;  // boundary sign of the hop
};

template <int H, int P, int R>
__device__ __forceinline__ void fetch_hop(const WilsonArgs& a, const int c[4], int s, int k0, HopRaw<P, R>& h) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    typedef typename Layout<P, 24>::C CS;
    typedef typename Layout<P, R>::C CU;
    float bs;
    const int n = cb_hop(a.g, c, MU, FWD ? 1 : -1, bs);
    h.bs = bs;
    const CS* sb = (const CS*)((const char*)a.in.data + (size_t)k0 * a.in.rhs_bytes);
#pragma unroll
    for (int k = 0; k < Layout<P, 24>::NC; k++) h.sp[k] = __ldg(&sb[(size_t)k * a.g.vh + n]);
    if constexpr (P == P16) h.n = __ldg(a.in.norm + (size_t)k0 * a.g.vh + n);
    const int lp = FWD ? a.parity : 1 - a.parity;
    const CU* ub = (const CU*)a.U.data + (size_t)(lp * 4 + MU) * Layout<P, R>::NC * a.g.vh;
    const int ls = FWD ? s : n;
#pragma unroll
    for (int k = 0; k < Layout<P, R>::NC; k++) h.u[k] = __ldg(&ub[(size_t)k * a.g.vh + ls]);
}

template <int H, int P, int R, typename T>
__device__ __forceinline__ void process_hop(const WilsonArgs& a, const HopRaw<P, R>& h, T sf, cx<T> acc[4][3]) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    typedef Layout<P, 24> LS;
    // FP16: spinor and link stay in integer codes (value / scale); the two scales
    // and the boundary sign multiply the 12 reals of the rotated half spinor once
    T v[24];
#pragma unroll
    for (int k = 0; k < LS::NC; k++) {
        if constexpr (P == P16) unpack_codes16<24, T>(h.sp[k], v + k * LS::RPC);
        else unpack_chunk<P, 24, T>(h.sp[k], 1.f, v + k * LS::RPC);
    }
    cx<T> U[3][3];
    decode_link<P, R, T>(h.u, a.U.scale, U);
    const float fu = link_factor<P, R>(a.U.scale);
    cx<T> ps[4][3], h0[3], h1[3], r0[3], r1[3];
    to_spinor(v, ps);
    const T sp = FWD ? sf : -sf;  // projector (1 + sp g_mu)
    proj<MU>(ps, sp, h0, h1);
    if constexpr (FWD) {
        su3_mv(U, h0, r0);
        su3_mv(U, h1, r1);
    } else {
        su3_dmv(U, h0, r0);
        su3_dmv(U, h1, r1);
    }
    if constexpr (P == P16) {
        const T sg = (T)(h.n * (1.f / 32767.f) * fu * (MU == 3 ? h.bs : 1.f));
#pragma unroll
        for (int k = 0; k < 3; k++) { r0[k] = sg * r0[k]; r1[k] = sg * r1[k]; }
    } else if constexpr (MU == 3) {
        const T sg = (T)h.bs;
#pragma unroll
        for (int k = 0; k < 3; k++) { r0[k] = sg * r0[k]; r1[k] = sg * r1[k]; }
    }
    recon_acc<MU>(acc, r0, r1, sp);
}

// hops of right-hand side k0 (the kernel's grid row when NB = 1)
template <int P, int R, typename T>
__device__ __forceinline__ void hops_pipelined(const WilsonArgs& a, const int c[4], int s, int k0, T sf,
                                               cx<T> acc[4][3]) {
    HopRaw<P, R> A, B;
    fetch_hop<0>(a, c, s, k0, A);
    fetch_hop<1>(a, c, s, k0, B); process_hop<0>(a, A, sf, acc);
    fetch_hop<2>(a, c, s, k0, A); process_hop<1>(a, B, sf, acc);
    fetch_hop<3>(a, c, s, k0, B); process_hop<2>(a, A, sf, acc);
    fetch_hop<4>(a, c, s, k0, A); process_hop<3>(a, B, sf, acc);
    fetch_hop<5>(a, c, s, k0, B); process_hop<4>(a, A, sf, acc);
    fetch_hop<6>(a, c, s, k0, A); process_hop<5>(a, B, sf, acc);
    fetch_hop<7>(a, c, s, k0, B); process_hop<6>(a, A, sf, acc);
    process_hop<7>(a, B, sf, acc);
}

// the same with the gathers of two hops ahead in flight (three raw buffers)
template <int P, int R, typename T>
__device__ __forceinline__ void hops_pipelined2(const WilsonArgs& a, const int c[4], int s, int k0, T sf,
                                                cx<T> acc[4][3]) {
    HopRaw<P, R> A, B, C;
    fetch_hop<0>(a, c, s, k0, A);
    fetch_hop<1>(a, c, s, k0, B);
    fetch_hop<2>(a, c, s, k0, C); process_hop<0>(a, A, sf, acc);
    fetch_hop<3>(a, c, s, k0, A); process_hop<1>(a, B, sf, acc);
    fetch_hop<4>(a, c, s, k0, B); process_hop<2>(a, C, sf, acc);
    fetch_hop<5>(a, c, s, k0, C); process_hop<3>(a, A, sf, acc);
    fetch_hop<6>(a, c, s, k0, A); process_hop<4>(a, B, sf, acc);
    fetch_hop<7>(a, c, s, k0, B); process_hop<5>(a, C, sf, acc);
    process_hop<6>(a, A, sf, acc);
    process_hop<7>(a, B, sf, acc);
}

// Prefetched epilogue operands in shared memory: one clover / A^{-1} record per
// site (copied by the first of its RG threads), one y spinor per thread (XPAY),
// and their FP16 norms.
template <int P, int EPI>
__host__ __device__ constexpr int epi_rec_bytes() {
    return (P == P64 || P == PDF) ? 0
         : EPI == EPI_AINV ? (int)(sizeof(typename Layout<P, 144>::C) * Layout<P, 144>::NC)
         : EPI == EPI_XPAY ? (int)(sizeof(typename Layout<P, 72>::C) * Layout<P, 72>::NC)
         : 0;
}
template <int P, int EPI>
__host__ __device__ constexpr int epi_y_bytes() {
    return (P == P64 || P == PDF || EPI != EPI_XPAY) ? 0 : (int)(sizeof(typename Layout<P, 24>::C) * Layout<P, 24>::NC);
}
template <int P, int EPI>
__host__ __device__ constexpr int epi_smem_per_thread() {  // non-zero when the epilogue is prefetched
    return epi_rec_bytes<P, EPI>() + epi_y_bytes<P, EPI>() + (epi_rec_bytes<P, EPI>() ? 8 : 0);
}
template <int P, int EPI>
__host__ __device__ constexpr size_t epi_smem_bytes(int block, int rg) {
    return epi_smem_per_thread<P, EPI>() == 0
               ? 0
               : (size_t)epi_rec_bytes<P, EPI>() * (block / rg) + (size_t)epi_y_bytes<P, EPI>() * block +
                     4 * ((size_t)(block / rg) + block);
}


// Grid: blocks are ordered site block major, right-hand-side group minor, so that
// the groups of one site block run together and share links and clover records
// through L2. Within a block, RG consecutive threads take one site and one
// right-hand side each (their link and clover loads are the same addresses and
// are served once); NB > 1 keeps NB right-hand sides in one thread's registers.
// MINB: minimum resident blocks of 256 threads the compiler must allow (1, or 3
// to cap the registers at 85 per thread for more warps in flight). DEEP: the
// single-RHS FP32/FP16 hops keep two hops of gathers in flight instead of one.
template <int P, int R, int EPI, int NB, int RG = 1, int MINB = 1, bool DEEP = false>
__global__ void __launch_bounds__(256, MINB) wilson_dslash_kernel(WilsonArgs a) {
    typedef typename RealT<P>::T T;
    const int spb = blockDim.x / RG;                       // sites per block
    const int ngroups = (a.nrhs + RG * NB - 1) / (RG * NB);
    const int sb = blockIdx.x / ngroups, grp = blockIdx.x - sb * ngroups;
    const int nsb = gridDim.x / ngroups;
    const int s = sb * spb + threadIdx.x / RG;
    const int kb = (grp * RG + threadIdx.x % RG) * NB;
    df nrm[NB];
#pragma unroll
    for (int b = 0; b < NB; b++) nrm[b] = df(0.f);
    // shared-memory copies of the epilogue operands (FP32/FP16, one RHS per thread)
    constexpr bool PF = (NB == 1) && (epi_smem_per_thread<P, EPI>() > 0);
    extern __shared__ __align__(16) unsigned char lq_smem[];
    typedef typename Layout<P, 144>::C CA;
    typedef typename Layout<P, 72>::C CC;
    typedef typename Layout<P, 24>::C CY;
    const int g = threadIdx.x / RG;   // site slot within the block
    unsigned char* sm_rec = lq_smem;  // clover / inverse record per site slot, chunk-major
    unsigned char* sm_y = sm_rec + (size_t)epi_rec_bytes<P, EPI>() * spb;
    float* sm_norm = (float*)(sm_y + (size_t)epi_y_bytes<P, EPI>() * blockDim.x);  // [spb] record, [blockDim] y
    if (s < a.g.vh && kb < a.nrhs) {
        int c[4];
        cb_coords(a.g, s, a.parity, c);
        if constexpr (PF) {
            if (a.has_clover && threadIdx.x % RG == 0) {
                // one copy per site: chunk k of slot g at k * spb + g
                if constexpr (EPI == EPI_AINV) {
                    CA* d = (CA*)sm_rec;
                    const CA* gsrc = (const CA*)a.clov;
#pragma unroll
                    for (int k = 0; k < Layout<P, 144>::NC; k++) cp_async16(&d[k * spb + g], &gsrc[(size_t)k * a.g.vh + s]);
                } else {
                    CC* d = (CC*)sm_rec;
                    const CC* gsrc = (const CC*)a.clov;
#pragma unroll
                    for (int k = 0; k < Layout<P, 72>::NC; k++) cp_async16(&d[k * spb + g], &gsrc[(size_t)k * a.g.vh + s]);
                }
                if constexpr (P == P16) cp_async4(&sm_norm[g], a.clov_norm + s);
            }
            if constexpr (EPI == EPI_XPAY) {
                prefetch_record<P, 24>(sm_y, (const char*)a.y.data + (size_t)kb * a.y.rhs_bytes, a.g.vh, s);
                if constexpr (P == P16)
                    cp_async4(&sm_norm[spb + threadIdx.x], a.y.norm + (size_t)kb * a.g.vh + s);
            }
            cp_async_commit();
        }
        cx<T> acc[NB][4][3];
#pragma unroll
        for (int b = 0; b < NB; b++)
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int cc = 0; cc < 3; cc++) acc[b][sp][cc] = mk((T)0, (T)0);
        const T sf = a.dagger ? (T)-1 : (T)1;
        if constexpr (NB == 1 && (P == P32 || P == P16) && DEEP) {
            hops_pipelined2<P, R, T>(a, c, s, kb, sf, acc[0]);
        } else if constexpr (NB == 1 && (P == P32 || P == P16)) {
            hops_pipelined<P, R, T>(a, c, s, kb, sf, acc[0]);
        } else if constexpr (P == PDF) {
#pragma unroll 1
            for (int h = 0; h < 8; h++) hop_compact<P, R, T>(a, c, s, kb, h, sf, acc[0]);
        } else {
            hop_dir<0, P, R, NB, T>(a, c, s, kb, sf, acc);
            hop_dir<1, P, R, NB, T>(a, c, s, kb, sf, acc);
            hop_dir<2, P, R, NB, T>(a, c, s, kb, sf, acc);
            hop_dir<3, P, R, NB, T>(a, c, s, kb, sf, acc);
        }
        if constexpr (PF) {
            cp_async_wait_all();
            // the site's record was copied by its first thread: make it visible to the others
            if constexpr (RG > 1) __syncwarp(__activemask());
        }
#pragma unroll
        for (int b = 0; b < NB; b++)
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int cc = 0; cc < 3; cc++) acc[b][sp][cc] = (T)0.5 * acc[b][sp][cc];

        cx<T> res[NB][4][3];
        if constexpr (EPI == EPI_HOP) {
#pragma unroll
            for (int b = 0; b < NB; b++)
#pragma unroll
                for (int sp = 0; sp < 4; sp++)
#pragma unroll
                    for (int cc = 0; cc < 3; cc++) res[b][sp][cc] = acc[b][sp][cc];
        } else if constexpr (EPI == EPI_AINV) {
            if (a.has_clover) {
#pragma unroll
                for (int b = 0; b < NB; b++)
#pragma unroll
                    for (int sp = 0; sp < 4; sp++)
#pragma unroll
                        for (int cc = 0; cc < 3; cc++) res[b][sp][cc] = mk((T)0, (T)0);
                if constexpr (PF)
                    ainv_apply_src<P, NB, T, true>(sm_rec, spb, g, P == P16 ? sm_norm[g] : 1.f, a.dagger, acc, res);
                else if constexpr (P == PDF && NB == 1)
                    ainv_apply_rows<P, T>(a, s, acc[0], res[0]);
                else
                    ainv_apply<P, NB, T>(a, s, acc, res);
            } else {
                // A^{-1} = ((4+m) - i mu_b) / ((4+m)^2 + mu^2) on chiral block b
                const T m4 = (T)a.m4, mu = (T)a.mu, mu1 = (T)a.mu1;
                const T inv = (T)1 / (m4 * m4 + mu * mu);
#pragma unroll
                for (int b = 0; b < NB; b++)
#pragma unroll
                    for (int sp = 0; sp < 4; sp++) {
                        const T mub = sp < 2 ? mu : mu1;
                        const cx<T> f = mk(m4 * inv, -mub * inv);
#pragma unroll
                        for (int cc = 0; cc < 3; cc++) res[b][sp][cc] = f * acc[b][sp][cc];
                    }
            }
        } else {  // EPI_XPAY: out = A y - D psi
            cx<T> yv[NB][4][3];
#pragma unroll
            for (int b = 0; b < NB; b++) {
                T v[24];
                if constexpr (PF) {
                    const float fy = (P == P16) ? sm_norm[spb + threadIdx.x] * (1.f / 32767.f) : 1.f;
#pragma unroll
                    for (int k = 0; k < Layout<P, 24>::NC; k++)
                        unpack_chunk<P, 24, T>(((const CY*)sm_y)[k * blockDim.x + threadIdx.x], fy,
                                               v + k * Layout<P, 24>::RPC);
                } else if (kb + b < a.nrhs) {
                    fload<P, 24, T>(a.y, kb + b, s, v);
                } else {
#pragma unroll
                    for (int q = 0; q < 24; q++) v[q] = (T)0;
                }
                to_spinor(v, yv[b]);
            }
            const T m4 = (T)a.m4, mu = (T)a.mu, mu1 = (T)a.mu1;
#pragma unroll
            for (int b = 0; b < NB; b++)
#pragma unroll
                for (int sp = 0; sp < 4; sp++) {
                    const cx<T> f = mk(m4, sp < 2 ? mu : mu1);
#pragma unroll
                    for (int cc = 0; cc < 3; cc++) res[b][sp][cc] = f * yv[b][sp][cc] - acc[b][sp][cc];
                }
            if (a.has_clover) {
                if constexpr (PF)
                    clover_apply_src<P, NB, T, true>(sm_rec, spb, g, P == P16 ? sm_norm[g] : 1.f, yv, res);
                else if constexpr (P == PDF && NB == 1)
                    clover_apply_rows<P, T>(a, s, yv[0], res[0]);
                else
                    clover_apply<P, NB, T>(a, s, yv, res);
            }
        }
#pragma unroll
        for (int b = 0; b < NB; b++) {
            if (kb + b >= a.nrhs) break;
            T v[24];
            const T g5 = a.gamma5_out ? (T)-1 : (T)1;
#pragma unroll
            for (int sp = 0; sp < 4; sp++)
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    v[(sp * 3 + cc) * 2] = sp < 2 ? res[b][sp][cc].r : g5 * res[b][sp][cc].r;
                    v[(sp * 3 + cc) * 2 + 1] = sp < 2 ? res[b][sp][cc].i : g5 * res[b][sp][cc].i;
                }
            if (a.norm_out) {
                // per-site sum in the kernel's precision, blocks reduce in FP64
                T t = (T)0;
#pragma unroll
                for (int q = 0; q < 24; q++) t = fma(v[q], v[q], t);
                nrm[b] = df_of(t);
            }
            fstore<P, 24, T>(a.out, kb + b, s, v);
        }
    }
    if (a.norm_out) {
        reduce_norms_rg<NB, RG>(nrm, a.norm_out, grp, sb, nsb, a.nrhs);
        fin_tail(a.norm_out, nsb, a.nrhs, a.fin);
    }
}

// site-local out = A^{-1} in (dagger: (A^{-1})^+ in) on fields of parity a.parity
template <int P>
__global__ void __launch_bounds__(256) wilson_ainv_site_kernel(WilsonArgs a) {
    typedef typename RealT<P>::T T;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (s >= a.g.vh || k >= a.nrhs) return;
    T v[24];
    fload<P, 24, T>(a.in, k, s, v);
    cx<T> w[1][4][3], res[1][4][3];
    to_spinor(v, w[0]);
    if (a.has_clover) {
#pragma unroll
        for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int cc = 0; cc < 3; cc++) res[0][sp][cc] = mk((T)0, (T)0);
        if constexpr (P == PDF) ainv_apply_rows<P, T>(a, s, w[0], res[0]);
        else ainv_apply<P, 1, T>(a, s, w, res);
    } else {
        const T m4 = (T)a.m4, mu = (T)a.mu, mu1 = (T)a.mu1;
        const T inv = (T)1 / (m4 * m4 + mu * mu);
#pragma unroll
        for (int sp = 0; sp < 4; sp++) {
            const cx<T> f = mk(m4 * inv, -(sp < 2 ? mu : mu1) * inv);
#pragma unroll
            for (int cc = 0; cc < 3; cc++) res[0][sp][cc] = f * w[0][sp][cc];
        }
    }
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {
            v[(sp * 3 + cc) * 2] = res[0][sp][cc].r;
            v[(sp * 3 + cc) * 2 + 1] = res[0][sp][cc].i;
        }
    fstore<P, 24, T>(a.out, k, s, v);
}

}  // namespace lq
