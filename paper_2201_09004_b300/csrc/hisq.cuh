// hisq.cuh -- staggered hopping term with HISQ fat one-hop and long three-hop links.
//
// For output parity p (Sec. 2.2 Eq. 4 with the fat and Naik links of HISQ):
//   D psi(x) = 1/2 sum_mu eta_mu(x) [V_mu(x) psi(x+mu) - V_mu(x-mu)^+ psi(x-mu)
//              + c_N (W_mu(x) psi(x+3mu) - W_mu(x-3mu)^+ psi(x-3mu))]
// with MILC phases eta_1 = (-1)^t, eta_2 = (-1)^(t+x), eta_3 = (-1)^(t+x+y),
// eta_4 = 1, and the time boundary sign once per crossing. Both x+-mu and
// x+-3mu have the other parity. H is anti-hermitian, so the adjoint is -D.
// Epilogues: EPI_HOP out = D psi; EPI_XPAY out = a*y - D psi (the even-odd
// Schur operator m^2 - H_eo H_oe as two launches, and its shifted versions).
#pragma once
#include <utility>

#include "wilson.cuh"

namespace lq {

struct HisqArgs {
    Geo g;
    GaugeV fat;     // R18
    GaugeV lng;     // R12 or R18
    FieldV in, out, y;
    int parity;
    int dagger;
    double c_naik;
    double a;       // XPAY scale
    const double* ak = nullptr;  // if non-null: the XPAY scale of rhs k at ak[k * SC_N] (device)
    int nrhs;
    df* norm_out;
    FinArgs fin;  // with norm_out: the last block finalises the sums
};

template <int MU, int STEP, int P, int R, int NB, typename T>
__device__ __forceinline__ void stag_hop(const HisqArgs& a, const GaugeV& G, const int c[4], int s, int kb, T coef,
                                         cx<T> acc[NB][3]) {
    // forward: + coef L_mu(x) psi(x + STEP mu)
    {
        float bs;
        const int n = cb_hop(a.g, c, MU, +STEP, bs);
        cx<T> U[3][3];
        load_link<P, R, T>(G, a.parity, MU, s, U);
        const T f = coef * (T)bs;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            if (kb + b >= a.nrhs) break;
            T v[6];
            fload<P, 6, T>(a.in, kb + b, n, v);
            cx<T> ps[3] = {mk(v[0], v[1]), mk(v[2], v[3]), mk(v[4], v[5])}, r[3];
            su3_mv(U, ps, r);
#pragma unroll
            for (int k = 0; k < 3; k++) acc[b][k] = acc[b][k] + f * r[k];
        }
    }
    // backward: - coef L_mu(x - STEP mu)^+ psi(x - STEP mu)
    {
        float bs;
        const int n = cb_hop(a.g, c, MU, -STEP, bs);
        cx<T> U[3][3];
        load_link<P, R, T>(G, 1 - a.parity, MU, n, U);
        const T f = coef * (T)bs;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            if (kb + b >= a.nrhs) break;
            T v[6];
            fload<P, 6, T>(a.in, kb + b, n, v);
            cx<T> ps[3] = {mk(v[0], v[1]), mk(v[2], v[3]), mk(v[4], v[5])}, r[3];
            su3_dmv(U, ps, r);
#pragma unroll
            for (int k = 0; k < 3; k++) acc[b][k] = acc[b][k] - f * r[k];
        }
    }
}

template <int MU, int P, int RL, int NB, typename T>
__device__ __forceinline__ void stag_dir(const HisqArgs& a, const int c[4], int s, int kb, T cn, cx<T> acc[NB][3]) {
    int e;  // eta_mu(x), MILC ordering
    if constexpr (MU == 0) e = c[3];
    else if constexpr (MU == 1) e = c[3] + c[0];
    else if constexpr (MU == 2) e = c[3] + c[0] + c[1];
    else e = 0;
    const T eta = (e & 1) ? (T)-1 : (T)1;
    stag_hop<MU, 1, P, 18, NB, T>(a, a.fat, c, s, kb, eta, acc);
    stag_hop<MU, 3, P, RL, NB, T>(a, a.lng, c, s, kb, eta * cn, acc);
}

// ---------------------------------------------------------------------------
// One right-hand side per thread: the 16 hops (per direction: fat forward,
// fat backward, long forward, long backward) are software-pipelined, the raw
// (still encoded) vector and link chunks of hop j+1 being loaded before hop j
// is decoded and applied.
template <int P, int R> struct StagRaw {
    typename Layout<P, 6>::C sp[Layout<P, 6>::NC];
    typename Layout<P, R>::C u[Layout<P, R>::NC];
    float n;   // FP16 vector norm
    float bs;  // boundary sign of the hop
};

template <int J, int P, int R>
__device__ __forceinline__ void stag_fetch(const HisqArgs& a, const GaugeV& G, const int c[4], int s, int k0,
                                           StagRaw<P, R>& r) {
    constexpr int MU = J >> 2;
    constexpr int STEP = ((J >> 1) & 1) ? 3 : 1;
    constexpr bool FWD = (J & 1) == 0;
    typedef typename Layout<P, 6>::C CS;
    typedef typename Layout<P, R>::C CU;
    float bs;
    const int n = cb_hop(a.g, c, MU, FWD ? STEP : -STEP, bs);
    r.bs = bs;
    const CS* sb = (const CS*)((const char*)a.in.data + (size_t)k0 * a.in.rhs_bytes);
#pragma unroll
    for (int k = 0; k < Layout<P, 6>::NC; k++) r.sp[k] = __ldg(&sb[(size_t)k * a.g.vh + n]);
    if constexpr (P == P16) r.n = __ldg(a.in.norm + (size_t)k0 * a.g.vh + n);
    const int lp = FWD ? a.parity : 1 - a.parity;
    const CU* ub = (const CU*)G.data + (size_t)(lp * 4 + MU) * Layout<P, R>::NC * a.g.vh;
    const int ls = FWD ? s : n;
#pragma unroll
    for (int k = 0; k < Layout<P, R>::NC; k++) r.u[k] = __ldg(&ub[(size_t)k * a.g.vh + ls]);
}

template <int J, int P, int R, typename T>
__device__ __forceinline__ void stag_apply(const GaugeV& G, const StagRaw<P, R>& r, T coef, cx<T> acc[3]) {
    constexpr bool FWD = (J & 1) == 0;
    typedef Layout<P, 6> LS;
    T v[6];
#pragma unroll
    for (int k = 0; k < LS::NC; k++) {
        if constexpr (P == P16) unpack_codes16<6, T>(r.sp[k], v + k * LS::RPC);
        else unpack_chunk<P, 6, T>(r.sp[k], 1.f, v + k * LS::RPC);
    }
    cx<T> U[3][3];
    decode_link<P, R, T>(r.u, G.scale, U);
    const float fu = link_factor<P, R>(G.scale);
    const cx<T> ps[3] = {mk(v[0], v[1]), mk(v[2], v[3]), mk(v[4], v[5])};
    cx<T> o[3];
    if constexpr (FWD) su3_mv(U, ps, o);
    else su3_dmv(U, ps, o);
    // forward hops add, backward hops subtract; FP16 scales and the boundary sign fold in here
    T f = coef * (T)r.bs * (FWD ? (T)1 : (T)-1);
    if constexpr (P == P16) f = f * (T)(r.n * (1.f / 32767.f) * fu);
#pragma unroll
    for (int q = 0; q < 3; q++) acc[q] = acc[q] + f * o[q];
}

template <int P, int RL, typename T, int... J>
__device__ __forceinline__ void stag_hops_pipelined(const HisqArgs& a, const int c[4], int s, int k0, T cn,
                                                    cx<T> acc[3], std::integer_sequence<int, J...>) {
    StagRaw<P, 18> F[2];
    StagRaw<P, RL> L[2];
    // eta_mu(x), MILC ordering
    const T eta[4] = {(c[3] & 1) ? (T)-1 : (T)1, ((c[3] + c[0]) & 1) ? (T)-1 : (T)1,
                      ((c[3] + c[0] + c[1]) & 1) ? (T)-1 : (T)1, (T)1};
    auto fetch = [&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if constexpr (j < 16) {
            if constexpr ((j >> 1) & 1) stag_fetch<j, P, RL>(a, a.lng, c, s, k0, L[j & 1]);
            else stag_fetch<j, P, 18>(a, a.fat, c, s, k0, F[j & 1]);
        }
    };
    auto apply = [&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if constexpr ((j >> 1) & 1) stag_apply<j, P, RL, T>(a.lng, L[j & 1], eta[j >> 2] * cn, acc);
        else stag_apply<j, P, 18, T>(a.fat, F[j & 1], eta[j >> 2], acc);
    };
    fetch(std::integral_constant<int, 0>());
    ((fetch(std::integral_constant<int, J + 1>()), apply(std::integral_constant<int, J>())), ...);
}

// thread / block mapping as in wilson_dslash_kernel (RG threads per site)
template <int P, int RL, int EPI, int NB, int RG = 1>
__global__ void __launch_bounds__(256) hisq_dslash_kernel(HisqArgs a) {
    typedef typename RealT<P>::T T;
    const int spb = blockDim.x / RG;
    const int ngroups = (a.nrhs + RG * NB - 1) / (RG * NB);
    const int sb = blockIdx.x / ngroups, grp = blockIdx.x - sb * ngroups;
    const int nsb = gridDim.x / ngroups;
    const int s = sb * spb + threadIdx.x / RG;
    const int kb = (grp * RG + threadIdx.x % RG) * NB;
    df nrm[NB];
#pragma unroll
    for (int b = 0; b < NB; b++) nrm[b] = df(0.f);
    if (s < a.g.vh && kb < a.nrhs) {
        int c[4];
        cb_coords(a.g, s, a.parity, c);
        cx<T> acc[NB][3];
#pragma unroll
        for (int b = 0; b < NB; b++)
#pragma unroll
            for (int k = 0; k < 3; k++) acc[b][k] = mk((T)0, (T)0);
        const T cn = (T)a.c_naik;
        if constexpr (NB == 1 && (P == P16 || P == P32)) {
            stag_hops_pipelined<P, RL, T>(a, c, s, kb, cn, acc[0], std::make_integer_sequence<int, 16>());
        } else {
            stag_dir<0, P, RL, NB, T>(a, c, s, kb, cn, acc);
            stag_dir<1, P, RL, NB, T>(a, c, s, kb, cn, acc);
            stag_dir<2, P, RL, NB, T>(a, c, s, kb, cn, acc);
            stag_dir<3, P, RL, NB, T>(a, c, s, kb, cn, acc);
        }
        const T half = a.dagger ? (T)-0.5 : (T)0.5;
#pragma unroll
        for (int b = 0; b < NB; b++) {
            if (kb + b >= a.nrhs) break;
            T v[6];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                cx<T> r = half * acc[b][k];
                v[2 * k] = r.r;
                v[2 * k + 1] = r.i;
            }
            if constexpr (EPI == EPI_XPAY) {
                T y[6];
                fload<P, 6, T>(a.y, kb + b, s, y);
                const T sa = a.ak ? (T)__ldg(a.ak + (size_t)(kb + b) * SC_N) : (T)a.a;
#pragma unroll
                for (int k = 0; k < 6; k++) v[k] = sa * y[k] - v[k];
            }
            if (a.norm_out) {
                T t = (T)0;
#pragma unroll
                for (int q = 0; q < 6; q++) t = fma(v[q], v[q], t);
                nrm[b] = df_of(t);
            }
            fstore<P, 6, T>(a.out, kb + b, s, v);
        }
    }
    if (a.norm_out) {
        reduce_norms_rg<NB, RG>(nrm, a.norm_out, grp, sb, nsb, a.nrhs);
        fin_tail(a.norm_out, nsb, a.nrhs, a.fin);
    }
}

}  // namespace lq
