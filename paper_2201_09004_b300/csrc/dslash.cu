// dslash.cu -- template dispatch and autotuned launch of the Wilson and HISQ
// hopping kernels. The tuned parameter is the thread-block size; several
// right-hand sides are carried NB = 4 / 2 / 1 per thread.
#include <string>

#include "dslash_launch.cuh"
#include "hisq_x2.cuh"
#include "wilson_x2.cuh"

namespace lq {

// FP16 / R12 single-right-hand-side kernels on packed FP32 pairs (wilson_x2.cuh).
// Tuning codes (variant * 1000 + block size):
//   3: registers for 4 resident blocks of 128 threads (128 per thread), two hops in flight;
//   4: 6 blocks (85 registers), two hops in flight;
//   5: 5 blocks (102 registers), one hop in flight;  6: 6 blocks, one hop in flight;
//   7: blocks of 256 threads, 2 resident (128 registers), two hops in flight (half the
//      blocks, and so half the partial sums of a fused reduction).
enum { kX2 = 3000, kX2c = 4000, kX2d = 5000, kX2e = 6000, kX2w = 7000 };

// (programmatic dependent launch: the kernel begins with pdl_start)
template <int EPI, bool DAG, int MINB, int DEPTH, int BT = 128>
static void wl_x2(const char* name, const WilsonArgs& a, int block, cudaStream_t st) {
    dim3 grid((a.g.vh + block - 1) / block);
    launch_pdl(name, wilson_f16x2_kernel<EPI, DAG, MINB, DEPTH, BT>, grid, dim3(block), x2_smem_bytes<EPI>(block),
               st, a);
}

// several right-hand sides, RG = 4 threads per site (variants 3 and 5 of the single-RHS codes)
template <int EPI, bool DAG, int MINB, int DEPTH>
static void wl_x2m(const char* name, const WilsonArgs& a, int block, cudaStream_t st) {
    constexpr int RG = 4;
    const int ngroups = (a.nrhs + RG - 1) / RG;
    dim3 grid(site_blocks(a.g.vh, block, RG) * ngroups);
    launch_smem(name, wilson_f16x2_mrhs_kernel<EPI, DAG, MINB, DEPTH, RG>, grid, dim3(block),
                x2_smem_bytes<EPI>(block, RG), st, a);
}

template <int EPI, bool DAG>
static void wl_x2_var(const char* name, const WilsonArgs& a, int cfg, cudaStream_t st) {
    if (a.nrhs > 1) {
        if (cfg / 1000 == 5) wl_x2m<EPI, DAG, 5, 1>(name, a, cfg % 1000, st);
        else wl_x2m<EPI, DAG, 4, 2>(name, a, cfg % 1000, st);
        return;
    }
    const int block = cfg % 1000;
    switch (cfg / 1000) {
        case 4: wl_x2<EPI, DAG, 6, 2>(name, a, block, st); break;
        case 5: wl_x2<EPI, DAG, 5, 1>(name, a, block, st); break;
        case 6: wl_x2<EPI, DAG, 6, 1>(name, a, block, st); break;
        case 7: wl_x2<EPI, DAG, 2, 2, 256>(name, a, block, st); break;
        default: wl_x2<EPI, DAG, 4, 2>(name, a, block, st); break;
    }
}

template <int EPI>
static void wl_x2_cfg(const char* name, const WilsonArgs& a, int cfg, cudaStream_t st) {
    if (a.dagger) wl_x2_var<EPI, true>(name, a, cfg, st);
    else wl_x2_var<EPI, false>(name, a, cfg, st);
}

static const char* wname(int prec, int epi) {
    static const char* n[4][3] = {
        {"wilson_dslash_f64_hop", "wilson_dslash_f64_ainv", "wilson_dslash_f64_xpay"},
        {"wilson_dslash_f32_hop", "wilson_dslash_f32_ainv", "wilson_dslash_f32_xpay"},
        {"wilson_dslash_f16_hop", "wilson_dslash_f16_ainv", "wilson_dslash_f16_xpay"},
        {"wilson_dslash_f32x2_hop", "wilson_dslash_f32x2_ainv", "wilson_dslash_f32x2_xpay"}};
    return n[prec][epi];
}

WilsonArgs wilson_args(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, const Field& in, Field& out,
                       const Field* y, cudaStream_t st) {
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
    a.mu1 = dagger ? -mu_block1(op) : mu_block1(op);
    a.m4f = (float)a.m4;
    a.muf = (float)a.mu;
    a.mu1f = (float)a.mu1;
    a.nrhs = in.nrhs;
    a.norm_out = nullptr;
    a.fin = FinArgs();
    a.clov = nullptr;
    a.clov_norm = nullptr;
    if (a.has_clover) {
        if (epi == EPI_XPAY) a.clov = clover_block(lat, op.prec, parity, &a.clov_norm);
        else if (epi == EPI_AINV) a.clov = ainv_block(lat, op.m, op.mu, mu_block1(op), op.prec, parity, &a.clov_norm, st);
    }
    return a;
}

int wilson_dslash(Lattice& lat, const OpDesc& op, int parity, int dagger, int epi, const Field& in, Field& out,
                  const Field* y, df* norm_out, cudaStream_t st, const FinArgs& fin, const Field* rb, Field* lo) {
    WilsonArgs a = wilson_args(lat, op, parity, dagger, epi, in, out, y, st);
    a.norm_out = norm_out;
    if (rb || lo) {  // the residual epilogue of the double-float A y - D kernel
        if (!rb || op.prec != LQ_F32X2 || epi != EPI_XPAY || a.gamma5_out || rb->prec != LQ_F32X2 ||
            rb->kind != LQ_WILSON_FIELD || rb->nrhs != out.nrhs || (lo && (lo->prec != LQ_F16 ||
            lo->kind != LQ_WILSON_FIELD || lo->nrhs != out.nrhs)))
            fail(LQ_EINVAL, "wilson_dslash: residual epilogue needs double-float A y - D, fields of its shape");
        a.rb = rb->view();
        if (lo) a.lo = lo->view();
    }
    a.fin = FinArgs();  // the tuner's trial launches never finalise
    const int nb = (op.prec == LQ_F32 || op.prec == LQ_F16) ? pick_rg(a.nrhs) : 1;
    const char* name = wname(op.prec, epi);
    // the packed-pair FP16 kernels: R12 links, one right-hand side, the clover epilogues
    // (or none), no g5 on the output, and lattices whose site index fits the fast division
    const bool x2 = op.prec == LQ_F16 && op.recon == 12 && (a.nrhs == 1 || nb == 4) && !a.gamma5_out &&
                    lat.geo.fast && (epi == EPI_HOP || a.has_clover);
    auto run = [&](int block) {  // block: a tuning code (see wl_nb)
        if (x2 && block >= kX2) {
            if (epi == EPI_HOP) wl_x2_cfg<EPI_HOP>(name, a, block, st);
            else if (epi == EPI_AINV) wl_x2_cfg<EPI_AINV>(name, a, block, st);
            else wl_x2_cfg<EPI_XPAY>(name, a, block, st);
        } else if (op.prec == LQ_F64) {
            if (op.recon == 18) wl_epi<P64, 18>(name, a, epi, nb, block, st);
            else wl_epi<P64, 12>(name, a, epi, nb, block, st);
        } else if (op.prec == LQ_F32X2) {
            if (epi == EPI_HOP) wl_df<EPI_HOP, false>(name, a, block, st);
            else if (epi == EPI_AINV) wl_df<EPI_AINV, false>(name, a, block, st);
            else wl_df<EPI_XPAY, false>(name, a, block, st);
        } else if (op.recon == 8) {
            wilson_launch_r8(op.prec, name, a, epi, nb, block, st);
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
                      std::to_string(norm_out != nullptr) + (rb ? (lo ? "/res16" : "/res") : "");
    std::vector<int> cand = {64, 128, 256};
    if ((op.prec == LQ_F32 || op.prec == LQ_F16) && nb != 2)
        for (int b : {64, 128, 256}) cand.push_back(kCapped + b);
    if (op.prec == LQ_F32X2 && epi != EPI_HOP)  // the double-float epilogue without row prefetch
        for (int b : {64, 128, 256}) cand.push_back(1000 + b);
    if ((op.prec == LQ_F32 || op.prec == LQ_F16) && nb == 1)
        for (int b : {64, 128}) cand.push_back(kDeep + b);
    if (x2 && a.nrhs == 1) {
        for (int v : {kX2, kX2c, kX2d, kX2e})
            for (int b : {64, 128}) cand.push_back(v + b);
        cand.push_back(kX2w + 256);
    }
    if (x2 && a.nrhs > 1)
        for (int v : {kX2, kX2d})
            for (int b : {64, 128}) cand.push_back(v + b);
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
    a.mu1 = dagger ? -mu_block1(op) : mu_block1(op);
    a.nrhs = in.nrhs;
    a.norm_out = nullptr;
    a.clov = nullptr;
    a.clov_norm = nullptr;
    if (a.has_clover) a.clov = ainv_block(lat, op.m, op.mu, mu_block1(op), in.prec, parity, &a.clov_norm, st);
    dim3 grid((lat.vh + 127) / 128, in.nrhs);
    if (in.prec == LQ_F64) launch("wilson_ainv_site", wilson_ainv_site_kernel<P64>, grid, dim3(128), st, a);
    else if (in.prec == LQ_F32X2)
        launch("wilson_ainv_site", wilson_dslash_df2_kernel<EPI_AINV, true>, dim3((lat.vh + 63) / 64, in.nrhs),
               dim3(128), st, a);
    else if (in.prec == LQ_F32) launch("wilson_ainv_site", wilson_ainv_site_kernel<P32>, grid, dim3(128), st, a);
    else launch("wilson_ainv_site", wilson_ainv_site_kernel<P16>, grid, dim3(128), st, a);
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
    // the packed-pair FP16 kernel (hisq_x2.cuh): R12 long links, one right-hand side;
    // tuning codes 3000 + block (128 registers), 4000 + block (85) and 5000 + block (64)
    const bool x2 = op.prec == LQ_F16 && op.recon == 12 && a.nrhs == 1 && lat.geo.fast;
    // 2 to 4 right-hand sides: the packed-pair kernel once per right-hand side (tuning codes
    // 9000 + block) beside the scalar kernel with its lanes per site; its partial sums land
    // in the layout of a multi-right-hand-side launch (rhs k at norm_out + k * blocks); not
    // with a finalising last block
    const bool x2m = op.prec == LQ_F16 && op.recon == 12 && a.nrhs >= 2 && a.nrhs <= 4 && lat.geo.fast &&
                     fin.sc == nullptr;
    auto run = [&](int block) {
        if (x2m && block >= 9000) {
            const int bs = block % 1000;
            dim3 grid((a.g.vh + bs - 1) / bs);
            for (int k = 0; k < a.nrhs; k++) {
                HisqArgs ak_ = a;
                ak_.nrhs = 1;
                ak_.in.data = (char*)a.in.data + (size_t)k * a.in.rhs_bytes;
                ak_.in.norm = a.in.norm + (size_t)k * a.g.vh;
                ak_.out.data = (char*)a.out.data + (size_t)k * a.out.rhs_bytes;
                ak_.out.norm = a.out.norm + (size_t)k * a.g.vh;
                ak_.y.data = (char*)a.y.data + (size_t)k * a.y.rhs_bytes;
                ak_.y.norm = a.y.norm + (size_t)k * a.g.vh;
                if (a.ak) ak_.ak = a.ak + (size_t)k * SC_N;
                if (a.norm_out) ak_.norm_out = a.norm_out + (size_t)k * grid.x;
                if (epi == EPI_XPAY) launch(name, hisq_f16x2_kernel<EPI_XPAY, 4>, grid, dim3(bs), st, ak_);
                else launch(name, hisq_f16x2_kernel<EPI_HOP, 4>, grid, dim3(bs), st, ak_);
            }
        } else if (x2 && block >= 3000) {
            const int bs = block % 1000, v = block / 1000;
            dim3 grid((a.g.vh + bs - 1) / bs);
            if (epi == EPI_XPAY) {
                if (v == 5) launch(name, hisq_f16x2_kernel<EPI_XPAY, 8>, grid, dim3(bs), st, a);
                else if (v == 4) launch(name, hisq_f16x2_kernel<EPI_XPAY, 6>, grid, dim3(bs), st, a);
                else launch(name, hisq_f16x2_kernel<EPI_XPAY, 4>, grid, dim3(bs), st, a);
            } else {
                if (v == 5) launch(name, hisq_f16x2_kernel<EPI_HOP, 8>, grid, dim3(bs), st, a);
                else if (v == 4) launch(name, hisq_f16x2_kernel<EPI_HOP, 6>, grid, dim3(bs), st, a);
                else launch(name, hisq_f16x2_kernel<EPI_HOP, 4>, grid, dim3(bs), st, a);
            }
        } else if (op.prec == LQ_F64) {
            if (op.recon == 18) hl_epi<P64, 18>(name, a, epi, nb, block, st);
            else hl_epi<P64, 12>(name, a, epi, nb, block, st);
        } else if (op.prec == LQ_F32X2) {
            hl_epi<PDF, 18>(name, a, epi, nb, block, st);
        } else if (op.recon == 8) {
            hisq_launch_r8(op.prec, name, a, epi, nb, block, st);
        } else if (op.prec == LQ_F32) {
            if (op.recon == 18) hl_epi<P32, 18>(name, a, epi, nb, block, st);
            else hl_epi<P32, 12>(name, a, epi, nb, block, st);
        } else {
            if (op.recon == 18) hl_epi<P16, 18>(name, a, epi, nb, block, st);
            else hl_epi<P16, 12>(name, a, epi, nb, block, st);
        }
    };
    std::string key = std::string(name) + "/r" + std::to_string(op.recon) + "/nb" + std::to_string(nb) + "/v" +
                      std::to_string(lat.vh) + "/n" + std::to_string(norm_out != nullptr) + "/f" +
                      std::to_string(fin.sc != nullptr);
    std::vector<int> cand = {64, 128, 256};
    if (x2)
        for (int c : {3064, 3128, 4064, 4128, 5064, 5128}) cand.push_back(c);
    if (x2m)
        for (int c : {9064, 9128}) cand.push_back(c);
    int block = tuned_block(key, st, run, cand);
    a.fin = norm_out ? fin : FinArgs();
    run(block);
    if (x2m && block >= 9000) return site_blocks(lat.vh, block % 1000, 1);
    return site_blocks(lat.vh, block % 1000, nb);
}

}  // namespace lq
