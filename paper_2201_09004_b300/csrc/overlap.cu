// overlap.cu -- building blocks of the overlap operator (Sec. 2.3):
//   D_ov = (1/rho) (1 + g5 eps(H_w)),  H_w = g5 D_w(-rho),  rho ~ 1.5,
// with eps the sign function. H_w is applied by the Wilson kernels with the g5
// multiplication fused into their epilogue (the fused g5 D_w kernel of Sec. 3).
// eps(H_w) is approximated, on the part of the spectrum with
// lambda_min <= |lambda| <= lambda_max, by x P(x^2) with x = H_w / lambda_max and
// P a Chebyshev polynomial of 1 / sqrt(y) on [eps^2, 1], eps = lambda_min /
// lambda_max; P is evaluated on vectors with the Clenshaw recurrence (Sec. 2.3:
// it keeps the round-off of the high-order terms under control). The paper fits
// the polynomial by exact interpolation at trial points refined at the extrema
// of the error (a Remez-like exchange); here the coefficients interpolate at the
// Chebyshev nodes, whose error is within a small factor of the minimax one, and
// the order is the smallest that meets the requested deviation on a dense grid.
#include <math.h>

#include <vector>

#include "runtime.h"

namespace lq {

// coefficients of p(y) = sum_k c_k T_k(z), z = (2y - a - b)/(b - a), interpolating
// 1/sqrt(y) at the n Chebyshev nodes of [a, b] (c_0 carries its factor 1/2)
static void cheb_inv_sqrt(double a, double b, int n, std::vector<double>& c) {
    std::vector<double> g(n);
    for (int j = 0; j < n; j++) {
        const double z = cos(M_PI * (j + 0.5) / n);
        g[j] = 1.0 / sqrt(0.5 * ((b - a) * z + a + b));
    }
    c.assign(n, 0.0);
    for (int k = 0; k < n; k++) {
        double s = 0.0;
        for (int j = 0; j < n; j++) s += g[j] * cos(M_PI * k * (j + 0.5) / n);
        c[k] = 2.0 * s / n;
    }
    c[0] *= 0.5;
}

// p at z by the Clenshaw recurrence
static double cheb_eval(const std::vector<double>& c, double z) {
    double b1 = 0.0, b2 = 0.0;
    for (int k = (int)c.size() - 1; k >= 1; k--) {
        const double b0 = c[k] + 2.0 * z * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return c[0] + z * b1 - b2;
}

// max over x in [eps, 1] of |1 - x p(x^2)| (sampled densely, log-spaced and linear)
static double sign_deviation(const std::vector<double>& c, double eps) {
    const double a = eps * eps, b = 1.0;
    double worst = 0.0;
    const int ns = 3000;
    for (int i = 0; i <= ns; i++) {
        const double xl = eps * pow(1.0 / eps, (double)i / ns);
        const double xs = eps + (1.0 - eps) * i / ns;
        for (double x : {xl, xs}) {
            const double y = x * x;
            const double z = (2.0 * y - a - b) / (b - a);
            worst = std::max(worst, fabs(1.0 - x * cheb_eval(c, z)));
        }
    }
    return worst;
}

// the smallest order (found by doubling, then bisection) whose deviation is <= delta
void sign_coefficients(double eps, double delta, int max_order, std::vector<double>& c, double& dev) {
    if (!(eps > 0.0 && eps < 1.0)) fail(LQ_EINVAL, "lambda_min / lambda_max must lie in (0, 1)");
    if (!(delta > 0.0)) fail(LQ_EINVAL, "the deviation bound must be positive");
    const double a = eps * eps, b = 1.0;
    int hi = 8;
    std::vector<double> t;
    for (;;) {
        cheb_inv_sqrt(a, b, hi, t);
        dev = sign_deviation(t, eps);
        if (dev <= delta) break;
        if (hi >= max_order) fail(LQ_EINVAL, "the sign function needs more than max_order Chebyshev terms");
        hi = std::min(2 * hi, max_order);
    }
    int lo = hi / 2;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        cheb_inv_sqrt(a, b, mid, t);
        const double d = sign_deviation(t, eps);
        if (d <= delta) hi = mid;
        else lo = mid;
    }
    cheb_inv_sqrt(a, b, hi, c);
    dev = sign_deviation(c, eps);
}

// out = g5 D_w(-rho) in on the full lattice; full vectors are fields of two
// "right-hand sides": rhs 0 the even sites, rhs 1 the odd sites
static void hw_apply(Lattice& lat, const OpDesc& d, const Field& in, Field& out, cudaStream_t st) {
    for (int p = 0; p < 2; p++) {
        const Field x_other = in.sub(1 - p, 1), x_same = in.sub(p, 1);
        Field o = out.sub(p, 1);
        wilson_dslash(lat, d, p, 0, EPI_XPAY, x_other, o, &x_same, nullptr, st);
    }
}

static OpDesc hw_desc(double rho, int prec) {
    OpDesc d;
    d.action = LQ_WILSON_TM;
    d.m = -rho;
    d.mu = 0.0;
    d.c_naik = 0.0;
    d.prec = prec;
    d.recon = 18;
    d.gamma5 = 1;
    return d;
}

void hw_apply_full(Lattice& lat, double rho, const Field& in, Field& out, cudaStream_t st) {
    hw_apply(lat, hw_desc(rho, in.prec), in, out, st);
}

// out = eps(H_w) in  ~  (H_w / lmax) P((H_w / lmax)^2) in, Clenshaw over the coefficients c
void sign_apply(Lattice& lat, double rho, double lmax, double eps, const std::vector<double>& c, const Field& v,
                Field& out, cudaStream_t st) {
    const OpDesc d = hw_desc(rho, v.prec);
    const int prec = v.prec;
    // work vectors from the lattice's workspace cache, returned on scope exit
    struct Work {
        Lattice& lat;
        cudaStream_t st;
        std::vector<void*> held;
        Field get(int prec) {
            Field f = ws_field(lat, LQ_WILSON_FIELD, prec, 2, st);
            held.push_back(f.data);
            return f;
        }
        ~Work() {
            for (void* p : held) ws_put(lat, p, st);
        }
    } work{lat, st, {}};
    Field b1 = work.get(prec), b2 = work.get(prec), t = work.get(prec), u = work.get(prec);
    const double a = eps * eps, b = 1.0;
    // Z w = (2 H^2 w / lmax^2 - (a + b) w) / (b - a)
    const double zh = 2.0 / (lmax * lmax * (b - a)), zc = -(a + b) / (b - a);
    blas_zero(b1, st);
    blas_zero(b2, st);
    const int n = (int)c.size();
    for (int k = n - 1; k >= 1; k--) {
        // b_k = c_k v + 2 Z b_{k+1} - b_{k+2}, written into b2's storage (b_{k+2} is not needed after)
        hw_apply(lat, d, b1, u, st);
        hw_apply(lat, d, u, t, st);
        blas_lincomb4(b2, c[k], v, 2.0 * zh, t, 2.0 * zc, b1, st);
        std::swap(b1, b2);  // now b1 = b_k, b2 = b_{k+1}
    }
    // P v = c_0 v + Z b_1 - b_2
    hw_apply(lat, d, b1, u, st);
    hw_apply(lat, d, u, t, st);
    blas_lincomb4(b2, c[0], v, zh, t, zc, b1, st);
    // eps(H) v = H (P v) / lmax
    hw_apply(lat, d, b2, u, st);
    blas_lincomb4(out, 0.0, v, 1.0 / lmax, u, 0.0, u, st, false);
}

}  // namespace lq
