// herm_eig.h -- eigen-decomposition of a small dense hermitian matrix on the
// host by the cyclic Jacobi method (the projected matrices of the eigensolver,
// at most a few dozen rows). Host-only C++; no CUDA.
//
// Each rotation acts on one pair (p, q): with a_pq = r e^{i phi}, the diagonal
// phase W = diag(1, e^{-i phi}) makes the 2x2 block [[a_pp, r], [r, a_qq]] real
// symmetric, and the plane rotation J = [[c, s], [-s, c]] with
// t = tan(theta) = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// zeta = (a_qq - a_pp) / (2 r), c = 1 / sqrt(1 + t^2), s = t c diagonalises it,
// so U = W J zeroes a_pq in U^+ A U. Sweeps over all pairs repeat until the
// off-diagonal mass is negligible against the matrix norm.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace lq {

typedef std::complex<double> zcx;

// A (m x m, row-major, hermitian; only its hermitian part is used) = V diag(w) V^+;
// column j of V (row-major V[i * m + j]) is the eigenvector of w[j]; w ascending.
inline void herm_eig(int m, std::vector<zcx> A, std::vector<double>& w, std::vector<zcx>& V) {
    for (int i = 0; i < m; i++)  // symmetrise: (A + A^+) / 2
        for (int j = i; j < m; j++) {
            const zcx h = 0.5 * (A[i * m + j] + std::conj(A[j * m + i]));
            A[i * m + j] = h;
            A[j * m + i] = std::conj(h);
        }
    for (int i = 0; i < m; i++) A[i * m + i] = zcx(A[i * m + i].real(), 0.0);
    V.assign((size_t)m * m, zcx(0.0, 0.0));
    for (int i = 0; i < m; i++) V[i * m + i] = 1.0;
    double norm2 = 0.0;
    for (const zcx& a : A) norm2 += std::norm(a);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) off += std::norm(A[p * m + q]);
        if (off <= 1e-32 * norm2 || off == 0.0) break;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                const zcx apq = A[p * m + q];
                const double r = std::abs(apq);
                if (r == 0.0) continue;
                const zcx e = apq / r;  // e^{i phi}
                const double app = A[p * m + p].real(), aqq = A[q * m + q].real();
                const double zeta = (aqq - app) / (2.0 * r);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                // U = W J on (p, q): U_pp = c, U_pq = s, U_qp = -s e^{-i phi}, U_qq = c e^{-i phi}
                const zcx upp = c, upq = s, uqp = -s * std::conj(e), uqq = c * std::conj(e);
                for (int k = 0; k < m; k++) {  // columns: A <- A U
                    const zcx akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = akp * upp + akq * uqp;
                    A[k * m + q] = akp * upq + akq * uqq;
                }
                for (int k = 0; k < m; k++) {  // rows: A <- U^+ A
                    const zcx apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = std::conj(upp) * apk + std::conj(uqp) * aqk;
                    A[q * m + k] = std::conj(upq) * apk + std::conj(uqq) * aqk;
                }
                A[p * m + q] = A[q * m + p] = 0.0;
                A[p * m + p] = zcx(A[p * m + p].real(), 0.0);
                A[q * m + q] = zcx(A[q * m + q].real(), 0.0);
                for (int k = 0; k < m; k++) {  // V <- V U
                    const zcx vkp = V[k * m + p], vkq = V[k * m + q];
                    V[k * m + p] = vkp * upp + vkq * uqp;
                    V[k * m + q] = vkp * upq + vkq * uqq;
                }
            }
    }
    std::vector<int> order(m);
    for (int i = 0; i < m; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return A[a * m + a].real() < A[b * m + b].real(); });
    w.resize(m);
    std::vector<zcx> Vs((size_t)m * m);
    for (int j = 0; j < m; j++) {
        w[j] = A[order[j] * m + order[j]].real();
        for (int i = 0; i < m; i++) Vs[i * m + j] = V[i * m + order[j]];
    }
    V.swap(Vs);
}

}  // namespace lq
