// eigen.cu -- low modes of H_w = g5 D_w(-rho) (Sec. 2.3), the eigenvectors the
// overlap operator's sign function is deflated with.
//
// The method follows the paper's: a Chebyshev polynomial of the operator
// enhances the low modes without changing the eigenvectors, and a restarted
// Arnoldi iteration on that polynomial finds them. Here the filter is
//   A = T_d(w(H_w^2)),  w(y) = (2y - a - b) / (b - a),  [a, b] = [lambda_cut^2, lambda_max^2],
// bounded by 1 on [a, b] and growing fast below a (d even, so A > 1 there): the
// modes with |lambda| < lambda_cut become the largest eigenvalues of A. A is
// hermitian, so the Arnoldi Hessenberg matrix is tridiagonal up to rounding;
// it is kept in full (classical Gram-Schmidt applied twice against every basis
// vector) and diagonalised on the host (Jacobi, herm_eig.h). At a restart the
// `keep` Ritz vectors of the largest Ritz values and the last Arnoldi vector
// form the new basis (thick restart): their projected matrix is diagonal plus
// the coupling row to the last vector, and the iteration continues from there.
// The nev wanted Ritz vectors are checked by a Rayleigh-Ritz step with H_w
// itself, which also separates eigenvalues +-lambda that A cannot tell apart;
// the solve ends when every |H_w z - lambda z| <= tol.
//
// Vectors are full-lattice double-float fields (two "right-hand sides": even and
// odd sites), so the eigenpairs reach FP64 accuracy on the FP32 pipes.
#include <math.h>

#include <algorithm>
#include <vector>

#include "herm_eig.h"
#include "runtime.h"

namespace lq {

// deterministic start vector: reals from a 64-bit mix of (rhs, site, component)
__global__ void eig_start_kernel(FieldV f) {
    const int k = blockIdx.y;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < f.vh; s += gridDim.x * blockDim.x) {
        double v[24];
        for (int q = 0; q < 24; q++) {
            unsigned long long z = ((unsigned long long)k << 40) ^ ((unsigned long long)s << 8) ^ (unsigned long long)q;
            z += 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            v[q] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        }
        fstore<PDF, 24, double>(f, k, s, v);
    }
}

namespace {

struct EigWork {
    Lattice& lat;
    cudaStream_t st;
    std::vector<void*> held;
    Field field() {
        Field f = ws_field(lat, LQ_WILSON_FIELD, LQ_F32X2, 2, st);
        held.push_back(f.data);
        return f;
    }
    void* raw(size_t bytes, bool pinned) {
        held.push_back(ws_get(lat, bytes, pinned, st));
        return held.back();
    }
    ~EigWork() {
        for (void* p : held) ws_put(lat, p, st);
    }
};

// dot products and Gram-Schmidt steps on full-lattice fields (both parities)
struct FullBlas {
    Lattice& lat;
    cudaStream_t st;
    FieldV* list_dev;   // device list of field views (cap entries)
    df* part;           // partials: 2 parities x cap x 2 x RED_BLOCKS
    df* hpart;          // pinned host copy
    double* coef_dev;   // 2 parities x cap complex coefficients
    int cap;
    // pageable sources: each copy is staged before cudaMemcpyAsync returns
    void upload(const std::vector<FieldV>& v) {
        if ((int)v.size() > cap) fail(LQ_EINVAL, "eigensolver: too many basis vectors");
        LQ_CUDA(cudaMemcpyAsync(list_dev, v.data(), sizeof(FieldV) * v.size(), cudaMemcpyHostToDevice, st));
    }
    // <v_i, w> for every v_i of vs (sums over both parities)
    std::vector<zcx> dots(const std::vector<Field>& vs, const Field& w) {
        std::vector<FieldV> l;
        for (const Field& f : vs) l.push_back(f.view());
        upload(l);
        const int nv = (int)vs.size();
        blas_cdot_multi(list_dev, nv, w, part, st);
        const size_t cnt = (size_t)2 * nv * 2 * RED_BLOCKS;
        LQ_CUDA(cudaMemcpyAsync(hpart, part, sizeof(df) * cnt, cudaMemcpyDeviceToHost, st));
        LQ_CUDA(cudaStreamSynchronize(st));
        std::vector<zcx> out(nv);
        for (int i = 0; i < nv; i++) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 2; k++)
                for (int b = 0; b < RED_BLOCKS; b++) {
                    const df& pr = hpart[(((size_t)k * nv + i) * 2 + 0) * RED_BLOCKS + b];
                    const df& pi = hpart[(((size_t)k * nv + i) * 2 + 1) * RED_BLOCKS + b];
                    re += (double)pr.hi + (double)pr.lo;
                    im += (double)pi.hi + (double)pi.lo;
                }
            out[i] = zcx(re, im);
        }
        return out;
    }
    double norm(const Field& w) { return std::sqrt(std::max(0.0, dots({w}, w)[0].real())); }
    // w -= sum_i c_i v_i
    void subtract(const std::vector<Field>& vs, const std::vector<zcx>& c, Field& w) {
        std::vector<FieldV> l;
        for (const Field& f : vs) l.push_back(f.view());
        l.push_back(w.view());
        upload(l);
        const int nv = (int)vs.size();
        std::vector<double> ch((size_t)2 * cap * 2, 0.0);
        for (int k = 0; k < 2; k++)
            for (int i = 0; i < nv; i++) {
                ch[((size_t)k * cap + i) * 2] = c[i].real();
                ch[((size_t)k * cap + i) * 2 + 1] = c[i].imag();
            }
        LQ_CUDA(cudaMemcpyAsync(coef_dev, ch.data(), sizeof(double) * ch.size(), cudaMemcpyHostToDevice, st));
        blas_gcr_orth(list_dev, nullptr, nv, coef_dev, cap, w, st);
    }
};

FullBlas make_full_blas(EigWork& work, int cap) {
    return FullBlas{work.lat,
                    work.st,
                    (FieldV*)work.raw(sizeof(FieldV) * cap, false),
                    (df*)work.raw(sizeof(df) * 2 * cap * 2 * RED_BLOCKS, false),
                    (df*)work.raw(sizeof(df) * 2 * cap * 2 * RED_BLOCKS, true),
                    (double*)work.raw(sizeof(double) * 2 * cap * 2, false),
                    cap};
}

}  // namespace

void hw_eigensolve(Lattice& lat, double rho, const lq_eig_params& p, std::vector<double>& evals,
                   std::vector<Field>& evecs, lq_eig_info& info, cudaStream_t st) {
    const int nev = p.nev;
    if (nev < 1 || nev > 48) fail(LQ_EINVAL, "nev must be in [1, 48]");
    const int m = p.nkv > 0 ? p.nkv : std::min(2 * nev + 8, 64);
    if (m < nev + 2 || m > 64) fail(LQ_EINVAL, "nkv must be in [nev + 2, 64]");
    int d = p.degree > 0 ? p.degree : 24;
    if (d & 1) d++;  // even: T_d > 1 below the filter interval
    if (!(p.lambda_max > p.lambda_cut && p.lambda_cut > 0.0)) fail(LQ_EINVAL, "need 0 < lambda_cut < lambda_max");
    if (!(p.tol > 0.0)) fail(LQ_EINVAL, "tol must be positive");
    const int max_restarts = p.max_restarts > 0 ? p.max_restarts : 100;
    const int keep = std::min(nev + (m - nev) / 2, m - 1);
    const double a = p.lambda_cut * p.lambda_cut, b = p.lambda_max * p.lambda_max;

    EigWork work{lat, st, {}};
    std::vector<Field> V(m + 1), W(keep), HZ(nev);
    for (auto& f : V) f = work.field();
    for (auto& f : W) f = work.field();
    for (auto& f : HZ) f = work.field();
    Field t0 = work.field(), t1 = work.field(), u = work.field(), w = work.field();
    FullBlas fb = make_full_blas(work, m + 2);
    int64_t applications = 0;

    // out = T_d(w(H^2)) in: T_0 = in, T_1 = w(H^2) in, T_{n+1} = 2 w(H^2) T_n - T_{n-1}
    const double zh = 2.0 / (b - a), zc = -(a + b) / (b - a);
    auto filter = [&](const Field& in, Field& out) {
        Field prev = t0, cur = t1;
        blas_copy(prev, in, st);
        hw_apply_full(lat, rho, in, u, st);
        hw_apply_full(lat, rho, u, out, st);
        blas_lincomb4(cur, zh, out, zc, in, 0.0, in, st, false);
        for (int n = 1; n < d; n++) {
            hw_apply_full(lat, rho, cur, u, st);
            hw_apply_full(lat, rho, u, out, st);
            // next = 2 (zh H^2 cur + zc cur) - prev, written over prev
            blas_lincomb4(prev, 2.0 * zh, out, 2.0 * zc, cur, 0.0, cur, st, true);
            std::swap(prev, cur);
        }
        blas_copy(out, cur, st);
        applications += 2 * d;
    };

    // start: a fixed pseudo-random vector, normalised
    launch("eig_start", eig_start_kernel, dim3((lat.vh + 127) / 128, 2), dim3(128), st, V[0].view());
    {
        const double n0 = fb.norm(V[0]);
        blas_lincomb4(V[0], 1.0 / n0, V[0], 0.0, V[0], 0.0, V[0], st, false);
    }
    std::vector<zcx> H((size_t)m * m, zcx(0.0, 0.0));
    int j0 = 0;
    double beta_last = 0.0;
    info.converged = 0;
    info.restarts = 0;
    info.max_residual = 0.0;
    evals.assign(nev, 0.0);
    for (int restart = 0;; restart++) {
        // Arnoldi steps j0 .. m-1 on A with classical Gram-Schmidt applied twice
        for (int j = j0; j < m; j++) {
            filter(V[j], w);
            std::vector<Field> basis(V.begin(), V.begin() + j + 1);
            std::vector<zcx> h = fb.dots(basis, w);
            fb.subtract(basis, h, w);
            std::vector<zcx> h2 = fb.dots(basis, w);
            fb.subtract(basis, h2, w);
            for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = h[i] + h2[i];
            const double beta = fb.norm(w);
            if (!(beta > 0.0) || !std::isfinite(beta)) fail(LQ_EBREAKDOWN, "eigensolver: the Krylov space closed");
            if (j + 1 < m) H[(size_t)(j + 1) * m + j] = beta;
            beta_last = beta;
            blas_lincomb4(V[j + 1], 1.0 / beta, w, 0.0, w, 0.0, w, st, false);
        }
        // Ritz pairs of A; the largest Ritz values belong to the lowest |lambda| of H_w
        std::vector<double> theta;
        std::vector<zcx> Y;
        herm_eig(m, H, theta, Y);
        std::vector<int> order(m);
        for (int i = 0; i < m; i++) order[i] = m - 1 - i;  // descending
        // new basis: Ritz vectors z_l = sum_i Y[i][l] v_i for the `keep` largest
        for (int l = 0; l < keep; l++) {
            std::vector<zcx> c(m);
            for (int i = 0; i < m; i++) c[i] = -Y[(size_t)i * m + order[l]];
            blas_zero(W[l], st);
            fb.subtract(std::vector<Field>(V.begin(), V.begin() + m), c, W[l]);
        }
        for (int l = 0; l < keep; l++) std::swap(V[l], W[l]);
        std::swap(V[keep], V[m]);
        // projected matrix of the new basis: diag(theta) and the coupling to v_keep
        std::fill(H.begin(), H.end(), zcx(0.0, 0.0));
        for (int l = 0; l < keep; l++) {
            H[(size_t)l * m + l] = theta[order[l]];
            const zcx cpl = beta_last * Y[(size_t)(m - 1) * m + order[l]];
            H[(size_t)keep * m + l] = cpl;
            H[(size_t)l * m + keep] = std::conj(cpl);
        }
        j0 = keep;

        // Rayleigh-Ritz with H_w on the nev wanted Ritz vectors, and their residuals
        std::vector<Field> Z(V.begin(), V.begin() + nev);
        for (int i = 0; i < nev; i++) hw_apply_full(lat, rho, Z[i], HZ[i], st);
        applications += nev;
        std::vector<zcx> G((size_t)nev * nev);
        for (int bcol = 0; bcol < nev; bcol++) {
            std::vector<zcx> g = fb.dots(Z, HZ[bcol]);  // <z_a, H z_b>
            for (int arow = 0; arow < nev; arow++) G[(size_t)arow * nev + bcol] = g[arow];
        }
        std::vector<double> mu;
        std::vector<zcx> S;
        herm_eig(nev, G, mu, S);
        // eigenvectors e_i = sum_a S[a][i] z_a into W[0..nev), residuals from H e_i - mu_i e_i
        double worst = 0.0;
        for (int i = 0; i < nev; i++) {
            std::vector<zcx> c(nev);
            for (int arow = 0; arow < nev; arow++) c[arow] = -S[(size_t)arow * nev + i];
            blas_zero(W[i], st);
            fb.subtract(Z, c, W[i]);  // e_i
            blas_zero(u, st);
            fb.subtract(HZ, c, u);  // H e_i
            blas_lincomb4(t0, 1.0, u, -mu[i], W[i], 0.0, u, st, false);
            worst = std::max(worst, fb.norm(t0));
        }
        info.restarts = restart;
        info.max_residual = worst;
        if (worst <= p.tol || restart + 1 >= max_restarts) {
            info.converged = worst <= p.tol ? 1 : 0;
            std::vector<int> idx(nev);  // ascending |lambda|
            for (int i = 0; i < nev; i++) idx[i] = i;
            std::sort(idx.begin(), idx.end(), [&](int x, int y) { return std::fabs(mu[x]) < std::fabs(mu[y]); });
            evecs.clear();
            for (int i = 0; i < nev; i++) {
                evals[i] = mu[idx[i]];
                // copied out of the work set into fields the caller returns to the cache
                Field f = ws_field(lat, LQ_WILSON_FIELD, LQ_F32X2, 2, st);
                blas_copy(f, W[idx[i]], st);
                evecs.push_back(f);
            }
            break;
        }
    }
    info.operator_applications = (int)std::min<int64_t>(applications, 2147483647);
}

// out = eps(H_w) in with the eigenvectors z_i (eigenvalues lambda_i) projected out
// of the polynomial's argument and their exact sign added back:
//   eps(H) v = sum_i sign(lambda_i) z_i <z_i, v> + x P(x^2) (v - sum_i z_i <z_i, v>)
void sign_apply_deflated(Lattice& lat, double rho, double lmax, double eps, const std::vector<double>& c,
                         const std::vector<double>& evals, const std::vector<Field>& evecs, const Field& v, Field& out,
                         cudaStream_t st) {
    const int nev = (int)evecs.size();
    EigWork work{lat, st, {}};
    Field vp = work.field();
    FullBlas fb = make_full_blas(work, nev + 2);
    std::vector<zcx> proj = nev ? fb.dots(evecs, v) : std::vector<zcx>();
    blas_copy(vp, v, st);
    if (nev) fb.subtract(evecs, proj, vp);  // v - sum z_i <z_i, v>
    sign_apply(lat, rho, lmax, eps, c, vp, out, st);
    if (nev) {
        std::vector<zcx> back(nev);
        for (int i = 0; i < nev; i++) back[i] = -(evals[i] >= 0.0 ? 1.0 : -1.0) * proj[i];
        fb.subtract(evecs, back, out);  // + sum sign(lambda_i) z_i <z_i, v>
    }
}

}  // namespace lq
