// dslash_r8.cu -- the Wilson and HISQ hopping kernels with R8 links (thin
// Wilson links, HISQ long links) in FP32 and FP16.
#include "dslash_launch.cuh"

namespace lq {

void wilson_launch_r8(int prec, const char* name, const WilsonArgs& a, int epi, int nb, int cfg, cudaStream_t st) {
    if (prec == LQ_F32) wl_epi<P32, 8>(name, a, epi, nb, cfg, st);
    else if (prec == LQ_F16) wl_epi<P16, 8>(name, a, epi, nb, cfg, st);
    else fail(LQ_EINVAL, "recon 8 is for LQ_F32 and LQ_F16 links");
}

void hisq_launch_r8(int prec, const char* name, const HisqArgs& a, int epi, int nb, int block, cudaStream_t st) {
    if (prec == LQ_F32) hl_epi<P32, 8>(name, a, epi, nb, block, st);
    else if (prec == LQ_F16) hl_epi<P16, 8>(name, a, epi, nb, block, st);
    else fail(LQ_EINVAL, "recon 8 is for LQ_F32 and LQ_F16 links");
}

}  // namespace lq
