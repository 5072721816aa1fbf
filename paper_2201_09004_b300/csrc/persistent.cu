// persistent.cu -- the inner iterations of the mixed-precision CG on the normal
// equations of the even-odd Schur operator as one persistent kernel.
//
// One cooperative launch (every block resident at once) runs `iters` CG
// iterations of the sloppy solve: the two Schur-operator applications, each an
// A^{-1} D launch (odd sites) and an A y - D launch (even sites) of the FP16
// packed-pair kernel (wilson_x2.cuh), the vector updates, and the three
// reductions that give alpha and beta, separated by grid-wide barriers instead
// of kernel boundaries. The blocks stride over the sites of each phase; the
// scalars stay in registers and shared memory, and the kernel writes them to the
// solver's scalar block at the end for the host's (lagged) convergence and
// reliable-update checks, exactly as the per-kernel path and its CUDA graphs do.
// Per iteration (Sec. 2.1's even-odd operator, CG on Mhat^+ Mhat):
//   t = A_oo^{-1} H_oe p;   q = A_ee p - H_eo t;            alpha = |r|^2 / |q|^2
//   x += alpha p;  s -= alpha q;                              |s|^2
//   t = (A_oo^{-1})^+ H_oe^+ s;  r = A_ee^+ s - H_eo^+ t;      beta = |r'|^2 / |r|^2
//   p = r + beta p
// Six barriers per iteration. Spinor loads go through L2 (ld.global.cg), since
// the kernel writes the fields it reads. Each barrier wait is bounded: after
// about half a second the kernel records the failure in the scalar block
// (SC_BREAK = 2) and returns; the host turns that into an error.
#include "runtime.h"
#include "wilson_x2.cuh"

namespace lq {

namespace {

constexpr int kThreads = 128;
constexpr unsigned long long kWaitNs = 500ull * 1000 * 1000;  // bound of one barrier wait

struct PcgArgs {
    WilsonArgs op[4];       // A^{-1} D p -> t, A p - D t -> q, and the adjoints on s -> t, r
    FieldV x, p, s, q, r;   // x: FP32 sloppy solution; p, s, q, r: FP16, even sites
    double* sc;             // the right-hand side's scalar block (SC_*)
    df* part;               // 2 x gridDim.x partial sums (two buffers, used in turn)
    unsigned* bar;          // barrier: [0] arrivals, [1] generation
    int iters;              // at most this many iterations
    double stop2;           // stop after the iteration whose |s|^2 falls below this (the host's
                            // reliable-update or convergence threshold, squared)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier (all blocks resident). Returns false, in every thread of the
// block, if the wait ran out; the others then time out too.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();  // this block's writes before its arrival
        ok = 1;
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g0) {
                if (global_ns() - t0 > kWaitNs) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();  // the other blocks' writes before ours that follow
    }
    __syncthreads();
    return ok != 0;
}

// grid-wide sum of every thread's v, the same value in every thread of every block:
// each block's total goes to buf[blockIdx.x], and after the barrier every block adds
// the totals in the same fixed order
__device__ bool grid_sum(df v, df* buf, unsigned* bar, double& out) {
    __shared__ double tot;
    const df b = block_sum_df(v);
    if (threadIdx.x == 0) buf[blockIdx.x] = b;
    if (!grid_barrier(bar, gridDim.x)) return false;
    df sum(0.f);
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const float2 w = __ldcg((const float2*)(buf + i));
        sum = sum + df(w.x, w.y);
    }
    sum = block_sum_df(sum);
    if (threadIdx.x == 0) tot = df_to_double(sum);
    __syncthreads();
    out = tot;
    return true;
}

__device__ __forceinline__ void ld24_cg(const FieldV& f, int s, float* v) {
    const int4* b = (const int4*)f.data;
    const float sc = __ldcg(f.norm + s) * (1.f / 32767.f);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int4 c = __ldcg(&b[(size_t)k * f.vh + s]);
        unpack_chunk<P16, 24, float>(c, 1.f, v + 8 * k);
    }
#pragma unroll
    for (int q = 0; q < 24; q++) v[q] *= sc;
}

__device__ __forceinline__ void ld24_cg_f32(const FieldV& f, int s, float* v) {
    const float4* b = (const float4*)f.data;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const float4 c = __ldcg(&b[(size_t)k * f.vh + s]);
        v[4 * k] = c.x; v[4 * k + 1] = c.y; v[4 * k + 2] = c.z; v[4 * k + 3] = c.w;
    }
}

__global__ void __launch_bounds__(kThreads, 4) pcg_kernel(PcgArgs a) {
    extern __shared__ __align__(16) unsigned char lq_smem[];
    double* S = a.sc;
    // converged, or already below the threshold (the host acts on it one launch late)
    if (S[SC_FROZEN] != 0.0 || S[SC_SS] < a.stop2) return;
    const int vh = a.op[0].g.vh;
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x + threadIdx.x;
    df* buf[2] = {a.part, a.part + gridDim.x};
    int nb = 0;
    double rr = S[SC_RR], qq = 0, ss = 0, rrn = 0, alpha = 0, beta = 0;
    bool ok = true;
    int done = 0;
    for (int it = 0; it < a.iters && ok; it++) {
        df dummy(0.f), acc(0.f);
        for (int s = first; s < vh; s += stride) x2_site<EPI_AINV, false, true>(a.op[0], s, threadIdx.x, blockDim.x, threadIdx.x, blockDim.x, 0, 0u, lq_smem, false, true, dummy);
        if (!(ok = grid_barrier(a.bar, gridDim.x))) break;
        for (int s = first; s < vh; s += stride) x2_site<EPI_XPAY, false, true>(a.op[1], s, threadIdx.x, blockDim.x, threadIdx.x, blockDim.x, 0, 0u, lq_smem, true, true, acc);
        if (!(ok = grid_sum(acc, buf[nb], a.bar, qq))) break;
        nb ^= 1;
        alpha = qq > 0.0 ? rr / qq : 0.0;
        // x += alpha p, s -= alpha q, |s|^2
        const float al = (float)alpha;
        acc = df(0.f);
        for (int s = first; s < vh; s += stride) {
            float vp[24], vs[24], vq[24], vx[24];
            ld24_cg(a.p, s, vp);
            ld24_cg(a.s, s, vs);
            ld24_cg(a.q, s, vq);
            ld24_cg_f32(a.x, s, vx);
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < 24; q++) {
                vx[q] = fmaf(al, vp[q], vx[q]);
                vs[q] = fmaf(-al, vq[q], vs[q]);
                t = fmaf(vs[q], vs[q], t);
            }
            acc = acc + df_of(t);
            fstore<P32, 24, float>(a.x, 0, s, vx);
            fstore<P16, 24, float>(a.s, 0, s, vs);
        }
        if (!(ok = grid_sum(acc, buf[nb], a.bar, ss))) break;
        nb ^= 1;
        acc = df(0.f);
        for (int s = first; s < vh; s += stride) x2_site<EPI_AINV, true, true>(a.op[2], s, threadIdx.x, blockDim.x, threadIdx.x, blockDim.x, 0, 0u, lq_smem, false, true, dummy);
        if (!(ok = grid_barrier(a.bar, gridDim.x))) break;
        for (int s = first; s < vh; s += stride) x2_site<EPI_XPAY, true, true>(a.op[3], s, threadIdx.x, blockDim.x, threadIdx.x, blockDim.x, 0, 0u, lq_smem, true, true, acc);
        if (!(ok = grid_sum(acc, buf[nb], a.bar, rrn))) break;
        nb ^= 1;
        beta = rr > 0.0 ? rrn / rr : 0.0;
        rr = rrn;
        // p = r + beta p
        const float be = (float)beta;
        for (int s = first; s < vh; s += stride) {
            float vp[24], vr[24];
            ld24_cg(a.p, s, vp);
            ld24_cg(a.r, s, vr);
#pragma unroll
            for (int q = 0; q < 24; q++) vp[q] = fmaf(be, vp[q], vr[q]);
            fstore<P16, 24, float>(a.p, 0, s, vp);
        }
        if (!(ok = grid_barrier(a.bar, gridDim.x))) break;
        done++;
        if (ss < a.stop2) break;  // the same in every block
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!ok) {
            S[SC_BREAK] = 2.0;  // a barrier wait ran out: the iterate is not valid
            return;
        }
        S[SC_QQ] = qq;
        S[SC_ALPHA] = alpha;
        S[SC_SS] = ss;
        S[SC_RRN] = rrn;
        S[SC_BETA] = beta;
        S[SC_RR] = rr;
        S[SC_ITERS] += (double)done;
    }
}

// A kernel that only meets at grid barriers, for the test of the bounded wait: with
// expect > gridDim.x blocks the first barrier never completes and the wait runs out.
__global__ void barrier_probe_kernel(unsigned* bar, unsigned expect, int rounds, int* failed) {
    for (int i = 0; i < rounds; i++) {
        if (!grid_barrier(bar, expect)) {
            if (threadIdx.x == 0) atomicExch(failed, 1);
            return;
        }
    }
}

}  // namespace

size_t pcg_smem_bytes() { return x2_smem_bytes<EPI_AINV>(kThreads); }

bool persistent_cg_supported(const Lattice& lat, const OpDesc& op, int nrhs) {
    return op.action == LQ_WILSON_TM_CLOVER && op.prec == LQ_F16 && op.recon == 12 && nrhs == 1 && !op.gamma5 &&
           lat.geo.fast != 0;
}

int persistent_cg_blocks(const Lattice& lat) {
    int per_sm = 0;
    const size_t smem = pcg_smem_bytes();
    opt_in_smem((const void*)pcg_kernel, smem);
    LQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel, kThreads, smem));
    if (per_sm < 1) fail(LQ_ECUDA, "the persistent CG kernel cannot be resident");
    const int need = (lat.vh + kThreads - 1) / kThreads;
    return std::min(need, per_sm * num_sms());
}

void persistent_cg_run(Lattice& lat, const OpDesc& op, Field& x, Field& p, Field& s, Field& q, Field& r, Field& t,
                       double* sc, df* part, unsigned* bar, int iters, double stop2, cudaStream_t st) {
    PcgArgs a;
    a.op[0] = wilson_args(lat, op, 1, 0, EPI_AINV, p, t, nullptr, st);
    a.op[1] = wilson_args(lat, op, 0, 0, EPI_XPAY, t, q, &p, st);
    a.op[2] = wilson_args(lat, op, 1, 1, EPI_AINV, s, t, nullptr, st);
    a.op[3] = wilson_args(lat, op, 0, 1, EPI_XPAY, t, r, &s, st);
    a.x = x.view();
    a.p = p.view();
    a.s = s.view();
    a.q = q.view();
    a.r = r.view();
    a.sc = sc;
    a.part = part;
    a.bar = bar;
    a.iters = iters;
    a.stop2 = stop2;
    const int blocks = persistent_cg_blocks(lat);
    void* args[] = {&a};
    int slot = prof_begin("persistent_cg", st);
    LQ_CUDA(cudaLaunchCooperativeKernel((const void*)pcg_kernel, dim3(blocks), dim3(kThreads), args, pcg_smem_bytes(),
                                        st));
    prof_end(slot, st);
    count_launch();
}

}  // namespace lq

using namespace lq;

extern "C" int lq_barrier_selftest(int blocks, int expect, int rounds, int* failed) {
    try {
        if (!failed || blocks < 1 || blocks > 64 || expect < blocks || expect > 64 || rounds < 1 || rounds > 1000)
            fail(LQ_EINVAL, "blocks in [1, 64], expect in [blocks, 64], rounds in [1, 1000]");
        void* dev = nullptr;
        LQ_CUDA(cudaMalloc(&dev, 16));
        struct Free {
            void* p;
            ~Free() { cudaFree(p); }
        } guard{dev};
        LQ_CUDA(cudaMemset(dev, 0, 16));
        unsigned* bar = (unsigned*)dev;
        int* flag = (int*)((char*)dev + 8);
        // a cooperative launch: all blocks are resident at once, as the barrier requires
        unsigned ex = (unsigned)expect;
        void* args[] = {&bar, &ex, &rounds, &flag};
        LQ_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_probe_kernel, dim3(blocks), dim3(32), args, 0, nullptr));
        LQ_CUDA(cudaDeviceSynchronize());
        LQ_CUDA(cudaMemcpy(failed, flag, sizeof(int), cudaMemcpyDeviceToHost));
        return *failed ? LQ_ETIMEOUT : LQ_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.code;
    } catch (...) {
        set_last_error("unexpected internal error");
        return LQ_EINVAL;
    }
}
