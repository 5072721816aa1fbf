// wilson_df.cuh -- the Wilson hopping kernel in double-float precision, two
// threads per site.
//
// The FP64-accuracy steps of the mixed solvers (reliable updates, source
// preparation, reconstruction of the odd sites, the final true residual) run
// in double-float arithmetic on the FP32 pipes. With one thread per site the
// kernel holds about 180 registers (a full 4x3 accumulator, a link and a
// spinor, each real as a hi/lo pair) and only eight warps fit on an SM to hide
// the neighbour gathers. Here the two threads of a site split the work by
// half-spinor component (Sec. 2.1: (1 +- g_mu) has rank two): thread h loads
// spin h of each neighbour and the spin that (1 +- g_mu) couples to it, forms
// half-spinor component h, multiplies it by the link and accumulates into
// upper spin h and one lower spin. After the eight hops the pair exchanges
// partial sums with two-lane shuffles so that thread h holds chiral block h
// (spins 2h and 2h+1), and applies the site-local epilogue to that 6-vector:
// block h of A^{-1}, or A y - D psi with block h of the clover term. Each
// output row is written as soon as it is formed.
#pragma once
#include "wilson.cuh"

namespace lq {

typedef cx<df> cd;

__device__ __forceinline__ cd ld_cd(const float4* base, size_t idx) {
    const float4 c = __ldg(base + idx);
    return mk(df(c.x, c.y), df(c.z, c.w));
}
__device__ __forceinline__ void st_cd(float4* base, size_t idx, cd v) {
    base[idx] = make_float4(v.r.hi, v.r.lo, v.i.hi, v.i.lo);
}
// value of the other thread of the pair (lanes 2g, 2g+1)
__device__ __forceinline__ cd pair_swap(cd v) {
    cd o;
    o.r.hi = __shfl_xor_sync(0xffffffffu, v.r.hi, 1);
    o.r.lo = __shfl_xor_sync(0xffffffffu, v.r.lo, 1);
    o.i.hi = __shfl_xor_sync(0xffffffffu, v.i.hi, 1);
    o.i.lo = __shfl_xor_sync(0xffffffffu, v.i.lo, 1);
    return o;
}
__device__ __forceinline__ df cnorm2(cd v) { return v.r * v.r + v.i * v.i; }

// Dot-product accumulator: the running sum keeps its high part exact with a
// two-sum per term and collects every rounding and product error in a plain
// FP32 low part, normalised once at the end (12 FP32 instructions per real
// multiply-add instead of 17 for a normalised double-float multiply and add).
struct dfacc {
    float hi, lo;
};
__device__ __forceinline__ void acc_prod(dfacc& a, df x, df y) {  // a += x y
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    const float s = __fadd_rn(a.hi, p);
    const float bb = __fsub_rn(s, a.hi);
    const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t, e));
}
__device__ __forceinline__ void acc_add(dfacc& a, df x) {  // a += x
    const float s = __fadd_rn(a.hi, x.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x.hi, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t, x.lo));
}
__device__ __forceinline__ df acc_done(dfacc a) { return df_fast_two_sum(a.hi, a.lo); }

struct cacc {
    dfacc r, i;
};
__device__ __forceinline__ cacc cacc_zero() { return cacc{{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ void cacc_mac(cacc& a, cd x, cd y) {  // a += x y
    acc_prod(a.r, x.r, y.r);
    acc_prod(a.r, -x.i, y.i);
    acc_prod(a.i, x.r, y.i);
    acc_prod(a.i, x.i, y.r);
}
__device__ __forceinline__ void cacc_cjmac(cacc& a, cd x, cd y) {  // a += conj(x) y
    acc_prod(a.r, x.r, y.r);
    acc_prod(a.r, x.i, y.i);
    acc_prod(a.i, x.r, y.i);
    acc_prod(a.i, -x.i, y.r);
}
__device__ __forceinline__ void cacc_add(cacc& a, cd x) {
    acc_add(a.r, x.r);
    acc_add(a.i, x.i);
}
__device__ __forceinline__ cd cacc_done(cacc a) { return mk(acc_done(a.r), acc_done(a.i)); }

// dynamic shared memory of the hop staging (two slots of 21 chunks per site)
__host__ __device__ constexpr size_t df2_smem_bytes(int block) { return (size_t)2 * 21 * 16 * (block / 2); }

// SITE = true: no hops, w = block h of `in` at the site (out = A^{-1} in).
template <int EPI, bool SITE>
__global__ void __launch_bounds__(256, 2) wilson_dslash_df2_kernel(WilsonArgs a) {
    const int h = threadIdx.x & 1;
    const int k = blockIdx.y;
    const int spb = blockDim.x >> 1;
    const int s_raw = blockIdx.x * spb + (threadIdx.x >> 1);
    const bool live = s_raw < a.g.vh;
    const int s = live ? s_raw : a.g.vh - 1;  // a pair past the end computes a valid site, stores nothing
    const size_t vh = (size_t)a.g.vh;
    const bool dag = a.dagger != 0;
    const float4* in = (const float4*)((const char*)a.in.data + (size_t)k * a.in.rhs_bytes);

    cd w[6];   // chiral block h: spins 2h, 2h+1 (index 3 * spin' + colour)
    cd yv[6];  // EPI_XPAY: block h of y, loaded while the pair exchanges its sums
    if constexpr (SITE) {
#pragma unroll
        for (int j = 0; j < 6; j++) w[j] = ld_cd(in, (size_t)(6 * h + j) * vh + s);
    } else {
        int c[4];
        cb_coords(a.g, s, a.parity, c);
        // The link (9 chunks) and neighbour spinor (12 chunks) of hop i+1 are copied
        // into shared memory with cp.async while hop i computes: stage[slot][chunk][site],
        // the two threads of a site copying alternate chunks.
        extern __shared__ __align__(16) unsigned char lq_smem[];
        float4* stage = (float4*)lq_smem;
        const int g = threadIdx.x >> 1;
        auto issue = [&](int hop, int slot) -> float {
            const int mu = hop >> 1;
            const bool fwd = (hop & 1) == 0;
            float bs;
            const int n = cb_hop(a.g, c, mu, fwd ? 1 : -1, bs);
            const float4* ub = (const float4*)a.U.data + (size_t)((fwd ? a.parity : 1 - a.parity) * 4 + mu) * 9 * vh;
            const size_t ls = (size_t)(fwd ? s : n);
#pragma unroll
            for (int k = h; k < 21; k += 2) {
                const float4* src = k < 9 ? ub + (size_t)k * vh + ls : in + (size_t)(k - 9) * vh + n;
                cp_async16(&stage[(slot * 21 + k) * spb + g], src);
            }
            cp_async_commit();
            return bs;
        };
        // upper spin h, lower spins 2 and 3: lazily normalised sums over the eight hops
        cacc upa[3], l2a[3], l3a[3];
#pragma unroll
        for (int q = 0; q < 3; q++) upa[q] = l2a[q] = l3a[q] = cacc_zero();
        float bs_next = issue(0, 0);
#pragma unroll 1
        for (int hop = 0; hop < 8; hop++) {
            const int mu = hop >> 1;
            const bool fwd = (hop & 1) == 0;
            const float bs = bs_next;
            if (hop < 7) {
                __syncwarp();  // both threads of the pair are done with the slot about to be refilled
                bs_next = issue(hop + 1, (hop + 1) & 1);
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            } else {
                cp_async_wait_all();
            }
            __syncwarp();  // the partner's copies of this hop are visible
            const float4* sl = stage + (size_t)((hop & 1) * 21) * spb + g;
            cx<df> U[3][3];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const float4 v = sl[k * spb];
                U[k / 3][k % 3] = mk(df(v.x, v.y), df(v.z, v.w));
            }
            // projector (1 + sp g_mu): sp = +-1 forward / backward, flipped for the adjoint
            const bool neg_sp = fwd ? dag : !dag;
            // component h couples spin h with spin pb through +-1 or +-i (DeGrand-Rossi)
            const int pb = mu < 2 ? 3 - h : 2 + h;
            const bool ci = (mu == 0 || mu == 2);
            const bool cn = (mu == 1 && h == 0) || (mu == 2 && h == 1);
            cd hv[3];
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const float4 va = sl[(9 + h * 3 + q) * spb];
                const float4 vp = sl[(9 + pb * 3 + q) * spb];
                // the sum stays unnormalised (exact high part, rounding in the low part)
                cacc t = cacc_zero();
                cacc_add(t, mk(df(va.x, va.y), df(va.z, va.w)));
                cacc_add(t, cunit(mk(df(vp.x, vp.y), df(vp.z, vp.w)), cn != neg_sp, ci));
                hv[q] = mk(df(t.r.hi, t.r.lo), df(t.i.hi, t.i.lo));
            }
            cd r[3];  // U hv or U^+ hv, unnormalised
#pragma unroll
            for (int i = 0; i < 3; i++) {
                cacc t = cacc_zero();
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    if (fwd) cacc_mac(t, U[i][j], hv[j]);
                    else cacc_cjmac(t, U[j][i], hv[j]);
                }
                r[i] = mk(df(t.r.hi, t.r.lo), df(t.i.hi, t.i.lo));
            }
            // rebuild: upper spin h gets r; lower spin (3 if to3 else 2) gets +-r or +-i r
            const bool flip = bs < 0.f;  // time boundary
            const bool to3 = mu < 2 ? (h == 0) : (h == 1);
            const bool ei = (mu == 0 || mu == 2);
            const bool en = mu == 0 || (mu == 1 && h == 0) || (mu == 2 && h == 0);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const cd rq = flip ? mk(-r[q].r, -r[q].i) : r[q];
                cacc_add(upa[q], rq);
                const cd e = cunit(rq, en != neg_sp, ei);
                if (to3) cacc_add(l3a[q], e);
                else cacc_add(l2a[q], e);
            }
        }
        cd up[3], lo2[3], lo3[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            up[q] = cacc_done(upa[q]);
            lo2[q] = cacc_done(l2a[q]);
            lo3[q] = cacc_done(l3a[q]);
        }
        if constexpr (EPI == EPI_XPAY) {
            const float4* yb = (const float4*)((const char*)a.y.data + (size_t)k * a.y.rhs_bytes);
#pragma unroll
            for (int j = 0; j < 6; j++) yv[j] = ld_cd(yb, (size_t)(6 * h + j) * vh + s);
        }
        // thread 0 takes the partner's upper spin (spin 1); thread 1 the partner's lower spins
        const df half(0.5f);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const cd ra = pair_swap(h ? up[q] : lo2[q]);
            const cd rb = pair_swap(lo3[q]);
            const cd w0 = h ? lo2[q] + ra : up[q];
            const cd w1 = h ? lo3[q] + rb : ra;
            w[q] = mk(half * w0.r, half * w0.i);
            w[3 + q] = mk(half * w1.r, half * w1.i);
        }
    }

    float4* out = (float4*)((char*)a.out.data + (size_t)k * a.out.rhs_bytes);
    df nrm(0.f);
    const bool neg_out = a.gamma5_out && h == 1;  // g5 negates chiral block 1 (spins 2, 3)
    if constexpr (EPI == EPI_HOP) {
#pragma unroll
        for (int i = 0; i < 6; i++) {
            if (live) st_cd(out, (size_t)(6 * h + i) * vh + s, neg_out ? mk(-w[i].r, -w[i].i) : w[i]);
            nrm = nrm + cnorm2(w[i]);
        }
    } else if constexpr (EPI == EPI_AINV) {
        if (a.has_clover) {
            // rows of block h of A^{-1} (36 complex, row-major); the adjoint reads the transpose,
            // conjugated. The entries of row i+1 are in flight while row i is computed.
            const float4* A = (const float4*)a.clov;
            auto entry = [&](int i, int j) { return (size_t)(dag ? h * 36 + j * 6 + i : h * 36 + i * 6 + j) * vh + s; };
            float4 cur[6], nxt[6];
#pragma unroll
            for (int j = 0; j < 6; j++) cur[j] = __ldg(A + entry(0, j));
#pragma unroll 1
            for (int i = 0; i < 6; i++) {
                if (i < 5) {
#pragma unroll
                    for (int j = 0; j < 6; j++) nxt[j] = __ldg(A + entry(i + 1, j));
                }
                cacc t = cacc_zero();
#pragma unroll
                for (int j = 0; j < 6; j++) {
                    const cd m = mk(df(cur[j].x, cur[j].y), df(cur[j].z, cur[j].w));
                    if (dag) cacc_cjmac(t, m, w[j]);
                    else cacc_mac(t, m, w[j]);
                }
#pragma unroll
                for (int j = 0; j < 6; j++) cur[j] = nxt[j];
                const cd acc = cacc_done(t);
                if (live) st_cd(out, (size_t)(6 * h + i) * vh + s, neg_out ? mk(-acc.r, -acc.i) : acc);
                nrm = nrm + cnorm2(acc);
            }
        } else {
            // A^{-1} = ((4+m) - i mu_h) / ((4+m)^2 + mu^2) on chiral block h (mu_0 = mu, mu_1 = mu1)
            const double inv = 1.0 / (a.m4 * a.m4 + a.mu * a.mu);
            const cd f = mk(df(a.m4 * inv), df(-(h ? a.mu1 : a.mu) * inv));
#pragma unroll
            for (int i = 0; i < 6; i++) {
                const cd o = f * w[i];
                if (live) st_cd(out, (size_t)(6 * h + i) * vh + s, neg_out ? mk(-o.r, -o.i) : o);
                nrm = nrm + cnorm2(o);
            }
        }
    } else {  // EPI_XPAY: out = ((4+m) + i mu_h + C) y - w on block h
        const cd f = mk(df(a.m4), df(h ? a.mu1 : a.mu));
        // C block h: 6 real diagonal entries (3 chunks) then the 15 upper entries
        // (row-major, i < j); chunk (i, j) of row i is the diagonal pair for j == i.
        // The chunks of row i+1 are in flight while row i is computed.
        const float4* C = (const float4*)a.clov;
        const bool clov = a.has_clover != 0;
        auto chunk = [&](int i, int j) {
            const int lo = j < i ? j : i, hi = j < i ? i : j;
            const int q = lo * 5 - lo * (lo - 1) / 2 + (hi - lo - 1);
            return (size_t)(18 * h + (j == i ? i / 2 : 3 + q)) * vh + s;
        };
        float4 cur[6], nxt[6];
        if (clov) {
#pragma unroll
            for (int j = 0; j < 6; j++) cur[j] = __ldg(C + chunk(0, j));
        }
#pragma unroll 1
        for (int i = 0; i < 6; i++) {
            if (clov && i < 5) {
#pragma unroll
                for (int j = 0; j < 6; j++) nxt[j] = __ldg(C + chunk(i + 1, j));
            }
            cacc t = cacc_zero();
#pragma unroll
            for (int j = 0; j < 6; j++) {
                if (j == i) {
                    const df di = !clov ? df(0.f) : (i & 1) ? df(cur[j].z, cur[j].w) : df(cur[j].x, cur[j].y);
                    cacc_mac(t, mk(f.r + di, f.i), yv[j]);
                    cacc_add(t, mk(-w[j].r, -w[j].i));
                } else if (clov) {
                    const cd m = mk(df(cur[j].x, cur[j].y), df(cur[j].z, cur[j].w));
                    if (i < j) cacc_mac(t, m, yv[j]);
                    else cacc_cjmac(t, m, yv[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < 6; j++) cur[j] = nxt[j];
            const cd acc = cacc_done(t);
            if (live) st_cd(out, (size_t)(6 * h + i) * vh + s, neg_out ? mk(-acc.r, -acc.i) : acc);
            nrm = nrm + cnorm2(acc);
        }
    }
    if (a.norm_out) {
        const df v[1] = {live ? nrm : df(0.f)};
        reduce_norms_rg<1, 1>(v, a.norm_out, k, blockIdx.x, gridDim.x, a.nrhs);
        fin_tail(a.norm_out, gridDim.x, a.nrhs, a.fin);
    }
}

}  // namespace lq
