// dslash_launch.cuh -- launch templates of the Wilson and HISQ hopping kernels,
// shared by the translation units that instantiate them (dslash.cu: links
// R18 / R12; dslash_r8.cu: R8).
#pragma once
#include "hisq.cuh"
#include "wilson_df.cuh"
#include "runtime.h"

namespace lq {

// right-hand sides per site group, spread over consecutive threads
static inline int pick_rg(int nrhs) {
    if (nrhs >= 4) return 4;
    if (nrhs >= 2) return 2;
    return 1;
}

// site blocks of a launch with `block` threads and rg threads per site
static inline int site_blocks(int vh, int block, int rg) {
    const int spb = block / rg;
    return (vh + spb - 1) / spb;
}

// ------------------------------------------------------------------ Wilson
template <int P, int R, int EPI, int RG, int MINB = 1, bool DEEP = false>
static void wl(const char* name, WilsonArgs a, int block, cudaStream_t st) {
    const int ngroups = (a.nrhs + RG - 1) / RG;
    dim3 grid(site_blocks(a.g.vh, block, RG) * ngroups);
    const size_t smem = epi_smem_bytes<P, EPI>(block, RG);
    launch_smem(name, wilson_dslash_kernel<P, R, EPI, 1, RG, MINB, DEEP>, grid, dim3(block), smem, st, a);
}

// tuning codes of the FP32/FP16 kernels: a block size; kCapped + block size for
// the build whose registers are capped at 85 per thread; kDeep + block size for
// the single-RHS build with two hops of gathers in flight (at most 128 registers)
enum { kCapped = 1000, kDeep = 2000 };

template <int P, int R, int EPI>
static void wl_nb(const char* name, WilsonArgs a, int rg, int cfg, cudaStream_t st) {
    if constexpr (P == P64 || P == PDF) {
        wl<P, R, EPI, 1>(name, a, cfg, st);
    } else {
        const int variant = cfg / 1000, block = cfg % 1000;
        if (rg == 4) {
            if (variant == 1) wl<P, R, EPI, 4, 3>(name, a, block, st);
            else wl<P, R, EPI, 4>(name, a, block, st);
        } else if (rg == 2) {
            wl<P, R, EPI, 2>(name, a, block, st);
        } else {
            if (variant == 1) wl<P, R, EPI, 1, 3>(name, a, block, st);
            else if (variant == 2) wl<P, R, EPI, 1, 2, true>(name, a, block, st);
            else wl<P, R, EPI, 1>(name, a, block, st);
        }
    }
}

template <int P, int R>
static void wl_epi(const char* name, WilsonArgs a, int epi, int nb, int block, cudaStream_t st) {
    if (epi == EPI_HOP) wl_nb<P, R, EPI_HOP>(name, a, nb, block, st);
    else if (epi == EPI_AINV) wl_nb<P, R, EPI_AINV>(name, a, nb, block, st);
    else wl_nb<P, R, EPI_XPAY>(name, a, nb, block, st);
}

// double-float: two threads per site, one right-hand side per grid row
template <int EPI, bool SITE>
static void wl_df(const char* name, WilsonArgs a, int cfg, cudaStream_t st) {
    const int block = cfg % 1000;
    dim3 grid(site_blocks(a.g.vh, block, 2), a.nrhs);
    // cfg / 1000 == 1: the epilogue without row prefetch (fewer registers)
    if (cfg / 1000 == 1)
        launch_smem(name, wilson_dslash_df2_kernel<EPI, SITE, false>, grid, dim3(block), SITE ? 0 : df2_smem_bytes(block),
                    st, a);
    else
        launch_smem(name, wilson_dslash_df2_kernel<EPI, SITE>, grid, dim3(block), SITE ? 0 : df2_smem_bytes(block), st, a);
}

// HISQ
template <int P, int RL, int EPI, int RG>
static void hl(const char* name, HisqArgs a, int block, cudaStream_t st) {
    const int ngroups = (a.nrhs + RG - 1) / RG;
    dim3 grid(site_blocks(a.g.vh, block, RG) * ngroups);
    launch(name, hisq_dslash_kernel<P, RL, EPI, 1, RG>, grid, dim3(block), st, a);
}

template <int P, int RL, int EPI>
static void hl_nb(const char* name, HisqArgs a, int rg, int block, cudaStream_t st) {
    if constexpr (P == P64 || P == PDF) {
        hl<P, RL, EPI, 1>(name, a, block, st);
    } else {
        if (rg == 4) hl<P, RL, EPI, 4>(name, a, block, st);
        else if (rg == 2) hl<P, RL, EPI, 2>(name, a, block, st);
        else hl<P, RL, EPI, 1>(name, a, block, st);
    }
}

template <int P, int RL>
static void hl_epi(const char* name, HisqArgs a, int epi, int nb, int block, cudaStream_t st) {
    if (epi == EPI_XPAY) hl_nb<P, RL, EPI_XPAY>(name, a, nb, block, st);
    else hl_nb<P, RL, EPI_HOP>(name, a, nb, block, st);
}

// R8 instantiations (FP32 / FP16 links), compiled in their own translation unit
void wilson_launch_r8(int prec, const char* name, const WilsonArgs& a, int epi, int nb, int cfg, cudaStream_t st);
void hisq_launch_r8(int prec, const char* name, const HisqArgs& a, int epi, int nb, int block, cudaStream_t st);

}  // namespace lq
