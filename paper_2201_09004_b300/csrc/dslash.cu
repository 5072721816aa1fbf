// dslash.cu -- template dispatch and autotuned launch of the Wilson and HISQ
// hopping kernels. The tuned parameter is the thread-block size; several
// right-hand sides are carried NB = 4 / 2 / 1 per thread.
#include <string>

#include "hisq.cuh"
#include "wilson_df.cuh"
#include "runtime.h"

namespace lq {

// right-hand sides per site group, spread over consecutive threads
static int pick_rg(int nrhs) {
    if (nrhs >= 4) return 4;
    if (nrhs >= 2) return 2;
    return 1;
}

// site blocks of a launch with `block` threads and rg threads per site
static int site_blocks(int vh, int block, int rg) {
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
static void wl_df(const char* name, WilsonArgs a, int block, cudaStream_t st) {
    dim3 grid(site_blocks(a.g.vh, block, 2), a.nrhs);
    launch_smem(name, wilson_dslash_df2_kernel<EPI, SITE>, grid, dim3(block), SITE ? 0 : df2_smem_bytes(block), st, a);
}

static const char* wname(int prec, int epi) {
    static const char* n[4][3] = {
        {"wilson_dslash_f64_hop", "wilson_dslash_f64_ainv", "wilson_dslash_f64_xpay"},
        {"wilson_dslash_f32_hop", "wilson_dslash_f32_ainv", "wilson_dslash_f32_xpay"},
        {"wilson_dslash_f16_hop", "wilson_dslash_f16_ainv", "wilson_dslash_f16_xpay"},
        {"wilson_dslash_f32x2_hop", "wilson_dslash_f32x2_ainv", "wilson_dslash_f32x2_xpay"}};
    return n[prec][epi];
}

int wilson_dslash(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, const Field& in, Field& out,
                  const Field* y, df* norm_out, cudaStream_t st, const FinArgs& fin) {
    if (in.prec != op.prec || out.prec != op.prec || (y && y->prec != op.prec))
        fail(LQ_EINVAL, "wilson_dslash: field precision does not match the operator");
    if (in.kind != LQ_WILSON_FIELD || out.nrhs != in.nrhs) fail(LQ_EINVAL, "wilson_dslash: field shape");
    WilsonArgs a;
    a.g = lat.geo;
    a.U = gauge_view(lat, LQ_THIN, op.prec, op.recon);
    a.in = in.view();
    a.out = out.view();
    a.y = y ? y->view() : out.view();
    a.parity = parity;
    a.dagger = dagger;
    a.has_clover = op.action == LQ_WILSON_TM_CLOVER;
    a.gamma5_out = op.gamma5;
    a.m4 = 4.0 + op.m;
    a.mu = dagger ? -op.mu : op.mu;
    a.nrhs = in.nrhs;
    a.norm_out = norm_out;
    a.fin = FinArgs();  // the tuner's trial launches never finalise
    a.clov = nullptr;
    a.clov_norm = nullptr;
    if (a.has_clover) {
        if (epi == EPI_XPAY) a.clov = clover_block(lat, op.prec, parity, &a.clov_norm);
        else if (epi == EPI_AINV) a.clov = ainv_block(lat, op.m, op.mu, op.prec, parity, &a.clov_norm, st);
    }
    const int nb = (op.prec == LQ_F32 || op.prec == LQ_F16) ? pick_rg(a.nrhs) : 1;
    const char* name = wname(op.prec, epi);
    auto run = [&](int block) {  // block: a tuning code (see wl_nb)
        if (op.prec == LQ_F64) {
            if (op.recon == 18) wl_epi<P64, 18>(name, a, epi, nb, block, st);
            else wl_epi<P64, 12>(name, a, epi, nb, block, st);
        } else if (op.prec == LQ_F32X2) {
            if (epi == EPI_HOP) wl_df<EPI_HOP, false>(name, a, block, st);
            else if (epi == EPI_AINV) wl_df<EPI_AINV, false>(name, a, block, st);
            else wl_df<EPI_XPAY, false>(name, a, block, st);
        } else if (op.prec == LQ_F32) {
            if (op.recon == 18) wl_epi<P32, 18>(name, a, epi, nb, block, st);
            else wl_epi<P32, 12>(name, a, epi, nb, block, st);
        } else {
            if (op.recon == 18) wl_epi<P16, 18>(name, a, epi, nb, block, st);
            else wl_epi<P16, 12>(name, a, epi, nb, block, st);
        }
    };
    std::string key = std::string(name) + "/r" + std::to_string(op.recon) + "/nb" + std::to_string(nb) + "/v" +
                      std::to_string(lat.vh) + "/c" + std::to_string(a.has_clover) + "/n" +
                      std::to_string(norm_out != nullptr);
    std::vector<int> cand = {64, 128, 256};
    if ((op.prec == LQ_F32 || op.prec == LQ_F16) && nb != 2)
        for (int b : {64, 128, 256}) cand.push_back(kCapped + b);
    if ((op.prec == LQ_F32 || op.prec == LQ_F16) && nb == 1)
        for (int b : {64, 128}) cand.push_back(kDeep + b);
    int cfg = tuned_block(key, st, run, cand);
    a.fin = norm_out ? fin : FinArgs();
    run(cfg);
    const int block = cfg % 1000;
    return site_blocks(lat.vh, block, op.prec == LQ_F32X2 ? 2 : nb);
}

void wilson_ainv_site(Lattice& lat, const OpDesc& op, int parity, int dagger, const Field& in, Field& out,
                      cudaStream_t st) {
    if (in.prec != out.prec || in.nrhs != out.nrhs) fail(LQ_EINVAL, "wilson_ainv_site: field mismatch");
    WilsonArgs a;
    a.g = lat.geo;
    a.U = GaugeV{nullptr, lat.vh, 1.f};
    a.in = in.view();
    a.out = out.view();
    a.y = out.view();
    a.parity = parity;
    a.dagger = dagger;
    a.has_clover = op.action == LQ_WILSON_TM_CLOVER;
    a.m4 = 4.0 + op.m;
    a.mu = dagger ? -op.mu : op.mu;
    a.nrhs = in.nrhs;
    a.norm_out = nullptr;
    a.clov = nullptr;
    a.clov_norm = nullptr;
    if (a.has_clover) a.clov = ainv_block(lat, op.m, op.mu, in.prec, parity, &a.clov_norm, st);
    dim3 grid((lat.vh + 127) / 128, in.nrhs);
    if (in.prec == LQ_F64) launch("wilson_ainv_site", wilson_ainv_site_kernel<P64>, grid, dim3(128), st, a);
    else if (in.prec == LQ_F32X2)
        launch("wilson_ainv_site", wilson_dslash_df2_kernel<EPI_AINV, true>, dim3((lat.vh + 63) / 64, in.nrhs),
               dim3(128), st, a);
    else if (in.prec == LQ_F32) launch("wilson_ainv_site", wilson_ainv_site_kernel<P32>, grid, dim3(128), st, a);
    else launch("wilson_ainv_site", wilson_ainv_site_kernel<P16>, grid, dim3(128), st, a);
}

// ------------------------------------------------------------------- HISQ
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

static const char* hname(int prec, int epi) {
    static const char* n[4][2] = {{"hisq_dslash_f64_hop", "hisq_dslash_f64_xpay"},
                                  {"hisq_dslash_f32_hop", "hisq_dslash_f32_xpay"},
                                  {"hisq_dslash_f16_hop", "hisq_dslash_f16_xpay"},
                                  {"hisq_dslash_f32x2_hop", "hisq_dslash_f32x2_xpay"}};
    return n[prec][epi == EPI_XPAY ? 1 : 0];
}

int hisq_dslash(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, double aa, const Field& in,
                Field& out, const Field* y, df* norm_out, cudaStream_t st, const FinArgs& fin, const double* ak) {
    if (in.prec != op.prec || out.prec != op.prec || (y && y->prec != op.prec))
        fail(LQ_EINVAL, "hisq_dslash: field precision does not match the operator");
    if (in.kind != LQ_STAGGERED_FIELD || out.nrhs != in.nrhs) fail(LQ_EINVAL, "hisq_dslash: field shape");
    HisqArgs a;
    a.g = lat.geo;
    a.fat = gauge_view(lat, LQ_FAT, op.prec, 18);
    a.lng = gauge_view(lat, LQ_LONG, op.prec, op.recon);
    a.in = in.view();
    a.out = out.view();
    a.y = y ? y->view() : out.view();
    a.parity = parity;
    a.dagger = dagger;
    a.c_naik = op.c_naik;
    a.a = aa;
    a.ak = ak;
    a.nrhs = in.nrhs;
    a.norm_out = norm_out;
    a.fin = FinArgs();  // the tuner's trial launches never finalise
    const int nb = (op.prec == LQ_F32 || op.prec == LQ_F16) ? pick_rg(a.nrhs) : 1;
    const char* name = hname(op.prec, epi);
    auto run = [&](int block) {
        if (op.prec == LQ_F64) {
            if (op.recon == 18) hl_epi<P64, 18>(name, a, epi, nb, block, st);
            else hl_epi<P64, 12>(name, a, epi, nb, block, st);
        } else if (op.prec == LQ_F32X2) {
            hl_epi<PDF, 18>(name, a, epi, nb, block, st);
        } else if (op.prec == LQ_F32) {
            if (op.recon == 18) hl_epi<P32, 18>(name, a, epi, nb, block, st);
            else hl_epi<P32, 12>(name, a, epi, nb, block, st);
        } else {
            if (op.recon == 18) hl_epi<P16, 18>(name, a, epi, nb, block, st);
            else hl_epi<P16, 12>(name, a, epi, nb, block, st);
        }
    };
    std::string key = std::string(name) + "/r" + std::to_string(op.recon) + "/nb" + std::to_string(nb) + "/v" +
                      std::to_string(lat.vh) + "/n" + std::to_string(norm_out != nullptr);
    int block = tuned_block(key, st, run);
    a.fin = norm_out ? fin : FinArgs();
    run(block);
    return site_blocks(lat.vh, block, nb);
}

}  // namespace lq
