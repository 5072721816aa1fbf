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
    int nrhs;
    df* norm_out;
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
        stag_dir<0, P, RL, NB, T>(a, c, s, kb, cn, acc);
        stag_dir<1, P, RL, NB, T>(a, c, s, kb, cn, acc);
        stag_dir<2, P, RL, NB, T>(a, c, s, kb, cn, acc);
        stag_dir<3, P, RL, NB, T>(a, c, s, kb, cn, acc);
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
                const T sa = (T)a.a;
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
    if (a.norm_out) reduce_norms_rg<NB, RG>(nrm, a.norm_out, grp, sb, nsb, a.nrhs);
}

}  // namespace lq
