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
// output row is written as soon as it is formed. The real and imaginary parts of
// every complex double-float value are register pairs, and each operation on them
// is one packed FP32 instruction for both.
#pragma once
#include "wilson.cuh"

namespace lq {

typedef cx<df> cd;

// A complex double-float number as two register pairs: h = (re.hi, im.hi), l = (re.lo,
// im.lo), the layout of a double-float chunk (see core.cuh). The arithmetic below runs
// on both lanes at once with the packed FP32 instructions of B300 (one instruction for
// two operations); a - b is fma(b, -1, a), exact in its product and rounded once.
struct cdp {
    float2 h, l;
};
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, p2(-1.f, -1.f), a); }
__device__ __forceinline__ cdp ld_cdp(const float4* base, size_t idx) {
    const float4 c = __ldg(base + idx);
    return cdp{p2(c.x, c.y), p2(c.z, c.w)};
}
__device__ __forceinline__ cdp cdp_of(float4 c) { return cdp{p2(c.x, c.y), p2(c.z, c.w)}; }
__device__ __forceinline__ void st_cdp(float4* base, size_t idx, cdp v) {
    base[idx] = make_float4(v.h.x, v.h.y, v.l.x, v.l.y);
}
__device__ __forceinline__ cdp cdp_neg(cdp v) {
    return cdp{__fmul2_rn(v.h, p2(-1.f, -1.f)), __fmul2_rn(v.l, p2(-1.f, -1.f))};
}
// v * (+-1 or +-i)
__device__ __forceinline__ cdp cdp_unit(cdp v, bool neg, bool isi) {
    const float2 sg = isi ? p2(neg ? 1.f : -1.f, neg ? -1.f : 1.f) : p2(neg ? -1.f : 1.f, neg ? -1.f : 1.f);
    const float2 h = isi ? p2(v.h.y, v.h.x) : v.h;  // i (a + ib) = -b + ia
    const float2 l = isi ? p2(v.l.y, v.l.x) : v.l;
    return cdp{__fmul2_rn(h, sg), __fmul2_rn(l, sg)};
}
// value of the other thread of the pair (lanes 2g, 2g+1)
__device__ __forceinline__ cdp pair_swap(cdp v) {
    cdp o;
    o.h.x = __shfl_xor_sync(0xffffffffu, v.h.x, 1);
    o.h.y = __shfl_xor_sync(0xffffffffu, v.h.y, 1);
    o.l.x = __shfl_xor_sync(0xffffffffu, v.l.x, 1);
    o.l.y = __shfl_xor_sync(0xffffffffu, v.l.y, 1);
    return o;
}

// Lazily normalised sum of both lanes: the high pair is kept exact by a two-sum per
// term, every rounding and product error goes to the plain low pair, normalised once
// at the end (per real multiply-add 6 packed instructions instead of 12 scalar ones).
struct caccp {
    float2 h, l;
};
__device__ __forceinline__ caccp caccp_zero() { return caccp{p2(0.f, 0.f), p2(0.f, 0.f)}; }
// a += x (both lanes)
__device__ __forceinline__ void accp_add(caccp& a, float2 xh, float2 xl) {
    const float2 s = __fadd2_rn(a.h, xh);
    const float2 bb = sub2(s, a.h);
    const float2 t = __fadd2_rn(sub2(a.h, sub2(s, bb)), sub2(xh, bb));
    a.h = s;
    a.l = __fadd2_rn(a.l, __fadd2_rn(t, xl));
}
// a += x y (both lanes)
__device__ __forceinline__ void accp_prod(caccp& a, float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 p = __fmul2_rn(xh, yh);
    float2 e = __ffma2_rn(xh, yh, __fmul2_rn(p, p2(-1.f, -1.f)));
    e = __ffma2_rn(xh, yl, e);
    e = __ffma2_rn(xl, yh, e);
    accp_add(a, p, e);
}
__device__ __forceinline__ void caccp_add(caccp& a, cdp x) { accp_add(a, x.h, x.l); }
// a += x y (complex): (re, im) += (x.re, x.re) (y.re, y.im) + (-x.im, x.im) (y.im, y.re)
__device__ __forceinline__ void caccp_mac(caccp& a, cdp x, cdp y) {
    accp_prod(a, p2(x.h.x, x.h.x), p2(x.l.x, x.l.x), y.h, y.l);
    accp_prod(a, p2(-x.h.y, x.h.y), p2(-x.l.y, x.l.y), p2(y.h.y, y.h.x), p2(y.l.y, y.l.x));
}
// a += conj(x) y: (re, im) += (x.re, x.re) (y.re, y.im) + (x.im, -x.im) (y.im, y.re)
__device__ __forceinline__ void caccp_cjmac(caccp& a, cdp x, cdp y) {
    accp_prod(a, p2(x.h.x, x.h.x), p2(x.l.x, x.l.x), y.h, y.l);
    accp_prod(a, p2(x.h.y, -x.h.y), p2(x.l.y, -x.l.y), p2(y.h.y, y.h.x), p2(y.l.y, y.l.x));
}
// the unnormalised sum as a value (the low pair may be large; later sums absorb it)
__device__ __forceinline__ cdp caccp_raw(caccp a) { return cdp{a.h, a.l}; }
// normalised: (h, l) = fast two-sum of the high and low pairs
__device__ __forceinline__ cdp caccp_done(caccp a) {
    const float2 s = __fadd2_rn(a.h, a.l);
    const float2 e = sub2(a.l, sub2(s, a.h));
    return cdp{s, e};
}
__device__ __forceinline__ cdp cdp_scale_half(cdp v) {
    return cdp{__fmul2_rn(v.h, p2(0.5f, 0.5f)), __fmul2_rn(v.l, p2(0.5f, 0.5f))};
}
__device__ __forceinline__ cdp cdp_add(cdp a, cdp b) {  // normalised sum
    caccp t{a.h, a.l};
    accp_add(t, b.h, b.l);
    return caccp_done(t);
}
__device__ __forceinline__ df cdp_norm2(cdp v) {
    const df re(v.h.x, v.l.x), im(v.h.y, v.l.y);
    return re * re + im * im;
}

// dynamic shared memory: the hop staging (two slots of 21 chunks per site) and the 12
// chunks per site of the residual's rb (used by A y - D with rb, copied at the start);
// 110.6 KB for 256 threads, two blocks per SM as the launch bounds ask
__host__ __device__ constexpr size_t df2_smem_bytes(int block) { return (size_t)(2 * 21 + 12) * 16 * (block / 2); }

// SITE = true: no hops, w = block h of `in` at the site (out = A^{-1} in). ROWPF: the
// epilogue loads the entries of row i+1 while row i is computed (more registers in flight).
// The grid is (site blocks, right-hand sides); its blocks are taken in the order of their
// linear index with the right-hand side varying fastest, so that the blocks of one site
// block and all right-hand sides run together and meet the links (and the clover or
// A^{-1} record) in L2.
template <int EPI, bool SITE, bool ROWPF = true>
__global__ void __launch_bounds__(256, 2) wilson_dslash_df2_kernel(WilsonArgs a) {
    const int h = threadIdx.x & 1;
    const int lin = blockIdx.y * gridDim.x + blockIdx.x;
    const int k = lin % gridDim.y;   // right-hand side
    const int sb = lin / gridDim.y;  // site block
    const int spb = blockDim.x >> 1;
    const int s_raw = sb * spb + (threadIdx.x >> 1);
    const bool live = s_raw < a.g.vh;
    const int s = live ? s_raw : a.g.vh - 1;  // a pair past the end computes a valid site, stores nothing
    const size_t vh = (size_t)a.g.vh;
    const bool dag = a.dagger != 0;
    const float4* in = (const float4*)((const char*)a.in.data + (size_t)k * a.in.rhs_bytes);

    cdp w[6];   // chiral block h: spins 2h, 2h+1 (index 3 * spin' + colour)
    cdp yv[6];  // EPI_XPAY: block h of y, loaded while the pair exchanges its sums
    const float4* rbs = nullptr;  // EPI_XPAY with rb: block h of rb in shared memory
    if constexpr (SITE) {
#pragma unroll
        for (int j = 0; j < 6; j++) w[j] = ld_cdp(in, (size_t)(6 * h + j) * vh + s);
    } else {
        int c[4];
        cb_coords(a.g, s, a.parity, c);
        // The link (9 chunks) and neighbour spinor (12 chunks) of hop i+1 are copied
        // into shared memory with cp.async while hop i computes: stage[slot][chunk][site],
        // the two threads of a site copying alternate chunks.
        extern __shared__ __align__(16) unsigned char lq_smem[];
        float4* stage = (float4*)lq_smem;
        const int g = threadIdx.x >> 1;
        if (EPI == EPI_XPAY && a.rb.data) {
            // rb of the residual: copied first, so that the hops' waits also cover it
            float4* rbw = stage + (size_t)2 * 21 * spb;
            const float4* src = (const float4*)((const char*)a.rb.data + (size_t)k * a.rb.rhs_bytes);
#pragma unroll
            for (int j = 0; j < 6; j++) cp_async16(&rbw[(6 * h + j) * spb + g], src + (size_t)(6 * h + j) * vh + s);
            cp_async_commit();
            rbs = rbw + g;
        }
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
        caccp upa[3], l2a[3], l3a[3];
#pragma unroll
        for (int q = 0; q < 3; q++) upa[q] = l2a[q] = l3a[q] = caccp_zero();
        float bs_next = issue(0, 0);
#pragma unroll
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
            cdp U[3][3];
#pragma unroll
            for (int k = 0; k < 9; k++) U[k / 3][k % 3] = cdp_of(sl[k * spb]);
            // projector (1 + sp g_mu): sp = +-1 forward / backward, flipped for the adjoint
            const bool neg_sp = fwd ? dag : !dag;
            // component h couples spin h with spin pb through +-1 or +-i (DeGrand-Rossi)
            const int pb = mu < 2 ? 3 - h : 2 + h;
            const bool ci = (mu == 0 || mu == 2);
            const bool cn = (mu == 1 && h == 0) || (mu == 2 && h == 1);
            cdp hv[3];
#pragma unroll
            for (int q = 0; q < 3; q++) {
                // the sum stays unnormalised (exact high part, rounding in the low part)
                caccp t{cdp_of(sl[(9 + h * 3 + q) * spb]).h, cdp_of(sl[(9 + h * 3 + q) * spb]).l};
                caccp_add(t, cdp_unit(cdp_of(sl[(9 + pb * 3 + q) * spb]), cn != neg_sp, ci));
                hv[q] = caccp_raw(t);
            }
            cdp r[3];  // U hv or U^+ hv, unnormalised
#pragma unroll
            for (int i = 0; i < 3; i++) {
                caccp t = caccp_zero();
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    if (fwd) caccp_mac(t, U[i][j], hv[j]);
                    else caccp_cjmac(t, U[j][i], hv[j]);
                }
                r[i] = caccp_raw(t);
            }
            // rebuild: upper spin h gets r; lower spin (3 if to3 else 2) gets +-r or +-i r
            const bool flip = bs < 0.f;  // time boundary
            const bool to3 = mu < 2 ? (h == 0) : (h == 1);
            const bool ei = (mu == 0 || mu == 2);
            const bool en = mu == 0 || (mu == 1 && h == 0) || (mu == 2 && h == 0);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const cdp rq = flip ? cdp_neg(r[q]) : r[q];
                caccp_add(upa[q], rq);
                const cdp e = cdp_unit(rq, en != neg_sp, ei);
                if (to3) caccp_add(l3a[q], e);
                else caccp_add(l2a[q], e);
            }
        }
        cdp up[3], lo2[3], lo3[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            up[q] = caccp_done(upa[q]);
            lo2[q] = caccp_done(l2a[q]);
            lo3[q] = caccp_done(l3a[q]);
        }
        if constexpr (EPI == EPI_XPAY) {
            const float4* yb = (const float4*)((const char*)a.y.data + (size_t)k * a.y.rhs_bytes);
#pragma unroll
            for (int j = 0; j < 6; j++) yv[j] = ld_cdp(yb, (size_t)(6 * h + j) * vh + s);
        }
        // thread 0 takes the partner's upper spin (spin 1); thread 1 the partner's lower spins
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const cdp ra = pair_swap(h ? up[q] : lo2[q]);
            const cdp rb = pair_swap(lo3[q]);
            const cdp w0 = h ? cdp_add(lo2[q], ra) : up[q];
            const cdp w1 = h ? cdp_add(lo3[q], rb) : ra;
            w[q] = cdp_scale_half(w0);
            w[3 + q] = cdp_scale_half(w1);
        }
    }

    float4* out = (float4*)((char*)a.out.data + (size_t)k * a.out.rhs_bytes);
    df nrm(0.f);
    const bool neg_out = a.gamma5_out && h == 1;  // g5 negates chiral block 1 (spins 2, 3)
    if constexpr (EPI == EPI_HOP) {
#pragma unroll
        for (int i = 0; i < 6; i++) {
            if (live) st_cdp(out, (size_t)(6 * h + i) * vh + s, neg_out ? cdp_neg(w[i]) : w[i]);
            nrm = nrm + cdp_norm2(w[i]);
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
                if (ROWPF && i < 5) {
#pragma unroll
                    for (int j = 0; j < 6; j++) nxt[j] = __ldg(A + entry(i + 1, j));
                } else if (!ROWPF && i > 0) {
#pragma unroll
                    for (int j = 0; j < 6; j++) cur[j] = __ldg(A + entry(i, j));
                }
                caccp t = caccp_zero();
#pragma unroll
                for (int j = 0; j < 6; j++) {
                    const cdp m = cdp_of(cur[j]);
                    if (dag) caccp_cjmac(t, m, w[j]);
                    else caccp_mac(t, m, w[j]);
                }
                if (ROWPF) {
#pragma unroll
                    for (int j = 0; j < 6; j++) cur[j] = nxt[j];
                }
                const cdp acc = caccp_done(t);
                if (live) st_cdp(out, (size_t)(6 * h + i) * vh + s, neg_out ? cdp_neg(acc) : acc);
                nrm = nrm + cdp_norm2(acc);
            }
        } else {
            // A^{-1} = ((4+m) - i mu_h) / ((4+m)^2 + mu^2) on chiral block h (mu_0 = mu, mu_1 = mu1)
            const double inv = 1.0 / (a.m4 * a.m4 + a.mu * a.mu);
            const df fr(a.m4 * inv), fi(-(h ? a.mu1 : a.mu) * inv);
            const cdp f{p2(fr.hi, fi.hi), p2(fr.lo, fi.lo)};
#pragma unroll
            for (int i = 0; i < 6; i++) {
                caccp t = caccp_zero();
                caccp_mac(t, f, w[i]);
                const cdp o = caccp_done(t);
                if (live) st_cdp(out, (size_t)(6 * h + i) * vh + s, neg_out ? cdp_neg(o) : o);
                nrm = nrm + cdp_norm2(o);
            }
        }
    } else {  // EPI_XPAY: out = ((4+m) + i mu_h + C) y - w on block h
        const df fr(a.m4), fi(h ? a.mu1 : a.mu);
        // C block h: 6 real diagonal entries (3 chunks) then the 15 upper entries
        // (row-major, i < j); chunk (i, j) of row i is the diagonal pair for j == i.
        // The chunks of row i+1 are in flight while row i is computed.
        const float4* C = (const float4*)a.clov;
        const bool clov = a.has_clover != 0;
        const int spb2 = spb;
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
            if (ROWPF && clov && i < 5) {
#pragma unroll
                for (int j = 0; j < 6; j++) nxt[j] = __ldg(C + chunk(i + 1, j));
            } else if (!ROWPF && clov && i > 0) {
#pragma unroll
                for (int j = 0; j < 6; j++) cur[j] = __ldg(C + chunk(i, j));
            }
            caccp t = caccp_zero();
#pragma unroll
            for (int j = 0; j < 6; j++) {
                if (j == i) {
                    // diagonal: the two reals of chunk (i, i) are entries 2(i/2), 2(i/2)+1
                    const df di = !clov ? df(0.f) : (i & 1) ? df(cur[j].y, cur[j].w) : df(cur[j].x, cur[j].z);
                    const df dr = fr + di;
                    caccp_mac(t, cdp{p2(dr.hi, fi.hi), p2(dr.lo, fi.lo)}, yv[j]);
                    caccp_add(t, cdp_neg(w[j]));
                } else if (clov) {
                    const cdp m = cdp_of(cur[j]);
                    if (i < j) caccp_mac(t, m, yv[j]);
                    else caccp_cjmac(t, m, yv[j]);
                }
            }
            if (ROWPF) {
#pragma unroll
                for (int j = 0; j < 6; j++) cur[j] = nxt[j];
            }
            cdp acc = caccp_done(t);
            if (neg_out) acc = cdp_neg(acc);
            if (rbs) acc = cdp_add(cdp_of(rbs[(6 * h + i) * spb2]), cdp_neg(acc));  // rb - (A y - w)
            if (live) st_cdp(out, (size_t)(6 * h + i) * vh + s, acc);
            nrm = nrm + cdp_norm2(acc);
        }
        if (a.lo.data) {
            // FP16 copy of the site: this thread's 12 reals read back from out (rounded to
            // FP32 as the FP16 store rounds them), the site's max |v| over both threads
            float v[12];
#pragma unroll
            for (int j = 0; j < 6; j++) {
                const float4 c = live ? __ldcg(out + (size_t)(6 * h + j) * vh + s) : make_float4(0.f, 0.f, 0.f, 0.f);
                v[2 * j] = __fadd_rn(c.x, c.z);
                v[2 * j + 1] = __fadd_rn(c.y, c.w);
            }
            float m = 0.f;
#pragma unroll
            for (int j = 0; j < 12; j++) m = fmaxf(m, fabsf(v[j]));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
            const float f = m > 0.f ? __fdividef(32767.f, m) : 0.f;
            // reals 0-11 of the site (h = 0) are chunk 0 and the first half of chunk 1,
            // reals 12-23 (h = 1) the second half of chunk 1 and chunk 2
            int4* lb = (int4*)((char*)a.lo.data + (size_t)k * a.lo.rhs_bytes);
            const int4 full = h ? make_int4(pack16f(v[4], v[5], f), pack16f(v[6], v[7], f), pack16f(v[8], v[9], f),
                                            pack16f(v[10], v[11], f))
                                : make_int4(pack16f(v[0], v[1], f), pack16f(v[2], v[3], f), pack16f(v[4], v[5], f),
                                            pack16f(v[6], v[7], f));
            const int2 half = h ? make_int2(pack16f(v[0], v[1], f), pack16f(v[2], v[3], f))
                                : make_int2(pack16f(v[8], v[9], f), pack16f(v[10], v[11], f));
            if (live) {
                lb[(size_t)(h ? 2 : 0) * vh + s] = full;
                ((int2*)(lb + vh + s))[h] = half;
                if (h == 0) a.lo.norm[(size_t)k * vh + s] = m;
            }
        }
    }
    if (a.norm_out) {
        const df v[1] = {live ? nrm : df(0.f)};
        reduce_norms_rg<1, 1>(v, a.norm_out, k, sb, gridDim.x, a.nrhs);
        fin_tail(a.norm_out, gridDim.x, a.nrhs, a.fin);
    }
}

}  // namespace lq
