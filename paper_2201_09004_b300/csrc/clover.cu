// clover.cu -- clover term (Sec. 2.1 Eq. 3) built on the device from the thin
// links, and the site-local twisted-clover inverse. The paper computes both on
// the GPU ("dynamical clover") because the inverse of the twisted clover term
// has a complex diagonal and is not hermitian (Sec. 2.1).
//
// C(x) = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x), sigma = (i/2)[g_mu, g_nu],
// Fhat = (Q - Q^+)/8 made traceless, Q the four plaquette leaves at x (all with
// orientation mu then nu). In the DeGrand-Rossi basis sigma commutes with
// g5 = diag(1,1,-1,-1), so C is two hermitian 6x6 blocks (spins {0,1}, {2,3}).
// Packed per block: 6 real diagonal entries, then the 15 upper off-diagonal
// entries (row-major, i<j) as complex numbers: 36 reals, 72 per site.
// A = (4+m) + C + i mu g5 is, per block b with g5 = chi_b = +1/-1,
// A_b = (4+m) + C_b + i mu_b with mu_b = chi_b mu (mu_b = mu for the scalar
// twist (4+m) + i mu + C); its inverse is stored as 36 complex numbers
// (row-major) per block, 144 reals per site, and computed by Gauss-Jordan
// elimination with partial pivoting in FP64.
#include <string.h>

#include "runtime.h"

namespace lq {

__constant__ double c_sigma[6][2][2][2][2];  // plane, chiral block, row, col, re/im

// DeGrand-Rossi gamma matrices (this library's own table), [mu][row][col][re/im]
static void host_gamma(double g[4][4][4][2]) {
    memset(g, 0, sizeof(double) * 4 * 4 * 4 * 2);
    // g1 = [[0, i s1], [-i s1, 0]]
    g[0][0][3][1] = 1; g[0][1][2][1] = 1; g[0][2][1][1] = -1; g[0][3][0][1] = -1;
    // g2 = [[0, -i s2], [i s2, 0]]
    g[1][0][3][0] = -1; g[1][1][2][0] = 1; g[1][2][1][0] = 1; g[1][3][0][0] = -1;
    // g3 = [[0, i s3], [-i s3, 0]]
    g[2][0][2][1] = 1; g[2][1][3][1] = -1; g[2][2][0][1] = -1; g[2][3][1][1] = 1;
    // g4 = [[0, 1], [1, 0]]
    g[3][0][2][0] = 1; g[3][1][3][0] = 1; g[3][2][0][0] = 1; g[3][3][1][0] = 1;
}

static void upload_sigma() {
    static int done_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (done_dev == dev) return;
    double g[4][4][4][2];
    host_gamma(g);
    double sig[6][2][2][2][2];
    int pl = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, pl++) {
            // sigma = (i/2)(g_mu g_nu - g_nu g_mu)
            double full[4][4][2];
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    double re = 0, im = 0;
                    for (int k = 0; k < 4; k++) {
                        double ar = g[mu][a][k][0], ai = g[mu][a][k][1], br = g[nu][k][b][0], bi = g[nu][k][b][1];
                        re += ar * br - ai * bi;
                        im += ar * bi + ai * br;
                        ar = g[nu][a][k][0]; ai = g[nu][a][k][1]; br = g[mu][k][b][0]; bi = g[mu][k][b][1];
                        re -= ar * br - ai * bi;
                        im -= ar * bi + ai * br;
                    }
                    full[a][b][0] = -0.5 * im;  // (i/2) (re + i im)
                    full[a][b][1] = 0.5 * re;
                }
            for (int blk = 0; blk < 2; blk++)
                for (int r = 0; r < 2; r++)
                    for (int c = 0; c < 2; c++) {
                        sig[pl][blk][r][c][0] = full[2 * blk + r][2 * blk + c][0];
                        sig[pl][blk][r][c][1] = full[2 * blk + r][2 * blk + c][1];
                    }
        }
    LQ_CUDA(cudaMemcpyToSymbol(c_sigma, sig, sizeof(sig)));
    done_dev = dev;
}

typedef cx<double> zd;

__device__ __forceinline__ void ld_link(const double* canon, int V, int mu, int lex, zd U[3][3]) {
    const double* u = canon + ((size_t)mu * V + lex) * 18;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) U[a][b] = mk(u[(a * 3 + b) * 2], u[(a * 3 + b) * 2 + 1]);
}

// C = op(A) op(B), op = adjoint when DA / DB
template <bool DA, bool DB>
__device__ __forceinline__ void mm(const zd A[3][3], const zd B[3][3], zd C[3][3]) {
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) {
            zd acc = mk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                zd a = DA ? cj(A[k][r]) : A[r][k];
                zd b = DB ? cj(B[s][k]) : B[k][s];
                cmac(acc, a, b);
            }
            C[r][s] = acc;
        }
}

__device__ __forceinline__ int lexc(const Geo& g, const int c[4]) {
    return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

__device__ __forceinline__ int shifted(const Geo& g, const int c[4], int mu, int dm, int nu, int dn) {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] = (n[mu] + dm + g.L[mu]) % g.L[mu];
    n[nu] = (n[nu] + dn + g.L[nu]) % g.L[nu];
    return lexc(g, n);
}

__device__ __forceinline__ void addm(zd Q[3][3], const zd T[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) Q[a][b] = Q[a][b] + T[a][b];
}

// sum of the four leaves of plane (mu, nu) at x
__device__ void leaves(const double* canon, int V, const Geo& g, const int c[4], int mu, int nu, zd Q[3][3]) {
    zd A[3][3], B[3][3], T1[3][3], T2[3][3];
    const int x = lexc(g, c);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) Q[a][b] = mk(0.0, 0.0);
    // U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    ld_link(canon, V, mu, x, A);
    ld_link(canon, V, nu, shifted(g, c, mu, 1, nu, 0), B);
    mm<false, false>(A, B, T1);
    ld_link(canon, V, mu, shifted(g, c, mu, 0, nu, 1), A);
    mm<false, true>(T1, A, T2);
    ld_link(canon, V, nu, x, B);
    mm<false, true>(T2, B, T1);
    addm(Q, T1);
    // U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    ld_link(canon, V, nu, x, A);
    ld_link(canon, V, mu, shifted(g, c, mu, -1, nu, 1), B);
    mm<false, true>(A, B, T1);
    ld_link(canon, V, nu, shifted(g, c, mu, -1, nu, 0), A);
    mm<false, true>(T1, A, T2);
    ld_link(canon, V, mu, shifted(g, c, mu, -1, nu, 0), B);
    mm<false, false>(T2, B, T1);
    addm(Q, T1);
    // U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    ld_link(canon, V, mu, shifted(g, c, mu, -1, nu, 0), A);
    ld_link(canon, V, nu, shifted(g, c, mu, -1, nu, -1), B);
    mm<true, true>(A, B, T1);
    ld_link(canon, V, mu, shifted(g, c, mu, -1, nu, -1), A);
    mm<false, false>(T1, A, T2);
    ld_link(canon, V, nu, shifted(g, c, mu, 0, nu, -1), B);
    mm<false, false>(T2, B, T1);
    addm(Q, T1);
    // U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    ld_link(canon, V, nu, shifted(g, c, mu, 0, nu, -1), A);
    ld_link(canon, V, mu, shifted(g, c, mu, 0, nu, -1), B);
    mm<true, false>(A, B, T1);
    ld_link(canon, V, nu, shifted(g, c, mu, 1, nu, -1), A);
    mm<false, false>(T1, A, T2);
    ld_link(canon, V, mu, x, B);
    mm<false, true>(T2, B, T1);
    addm(Q, T1);
}

// one thread per site of parity blockIdx.y; writes packed C (FP64)
__global__ void clover_build_kernel(const double* canon, int V, Geo g, double c_sw, void* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (s >= g.vh) return;
    int c[4];
    cb_coords(g, s, p, c);
    zd C[2][6][6];
    for (int b = 0; b < 2; b++)
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) C[b][i][j] = mk(0.0, 0.0);
    int pl = 0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++, pl++) {
            zd Q[3][3], F[3][3];
            leaves(canon, V, g, c, mu, nu, Q);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) F[a][b] = 0.125 * (Q[a][b] - cj(Q[b][a]));
            zd tr = (1.0 / 3.0) * (F[0][0] + F[1][1] + F[2][2]);
            for (int a = 0; a < 3; a++) F[a][a] = F[a][a] - tr;
            for (int b = 0; b < 2; b++)
                for (int s1 = 0; s1 < 2; s1++)
                    for (int s2 = 0; s2 < 2; s2++) {
                        // coefficient c_sw * (i/2) * sigma[pl][b][s1][s2]
                        zd sg = mk(c_sigma[pl][b][s1][s2][0], c_sigma[pl][b][s1][s2][1]);
                        zd f = (0.5 * c_sw) * ti(sg);
                        for (int a = 0; a < 3; a++)
                            for (int a2 = 0; a2 < 3; a2++) cmac(C[b][s1 * 3 + a][s2 * 3 + a2], f, F[a][a2]);
                    }
        }
    double v[72];
    for (int b = 0; b < 2; b++) {
        double* w = v + 36 * b;
        for (int i = 0; i < 6; i++) w[i] = C[b][i][i].r;
        int q = 0;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++, q++) {
                w[6 + 2 * q] = C[b][i][j].r;
                w[6 + 2 * q + 1] = C[b][i][j].i;
            }
    }
    char* base = (char*)out + (size_t)p * 36 * g.vh * sizeof(double2);
    store_reals<P64, 72, double>(base, g.vh, s, nullptr, 1.f, v);
}

// canonical 12x12 clover (hermitian, commuting with g5) -> packed FP64
__global__ void clover_pack_kernel(const double* canon, Geo g, void* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (s >= g.vh) return;
    int c[4];
    cb_coords(g, s, p, c);
    const double* m = canon + (size_t)lexc(g, c) * 288;  // 12x12 complex
    double v[72];
    for (int b = 0; b < 2; b++) {
        double* w = v + 36 * b;
        for (int i = 0; i < 6; i++) w[i] = m[((6 * b + i) * 12 + 6 * b + i) * 2];
        int q = 0;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++, q++) {
                w[6 + 2 * q] = m[((6 * b + i) * 12 + 6 * b + j) * 2];
                w[6 + 2 * q + 1] = m[((6 * b + i) * 12 + 6 * b + j) * 2 + 1];
            }
    }
    char* base = (char*)out + (size_t)p * 36 * g.vh * sizeof(double2);
    store_reals<P64, 72, double>(base, g.vh, s, nullptr, 1.f, v);
}

// A^{-1} per site from packed C (FP64), Gauss-Jordan with partial pivoting
__global__ void ainv_kernel(const void* cl, Geo g, double m4, double mu0, double mu1, void* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (s >= g.vh) return;
    double v[72];
    load_reals<P64, 72, double>((const char*)cl + (size_t)p * 36 * g.vh * sizeof(double2), g.vh, s, 1.f, v);
    double o[144];
    for (int b = 0; b < 2; b++) {
        const double mub = b == 0 ? mu0 : mu1;
        zd A[6][12];
        const double* w = v + 36 * b;
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 12; j++) A[i][j] = mk(0.0, 0.0);
        for (int i = 0; i < 6; i++) {
            A[i][i] = mk(w[i] + m4, mub);
            A[i][6 + i] = mk(1.0, 0.0);
        }
        int q = 0;
        for (int i = 0; i < 6; i++)
            for (int j = i + 1; j < 6; j++, q++) {
                zd e = mk(w[6 + 2 * q], w[6 + 2 * q + 1]);
                A[i][j] = e;
                A[j][i] = cj(e);
            }
        for (int col = 0; col < 6; col++) {
            int piv = col;
            double best = A[col][col].r * A[col][col].r + A[col][col].i * A[col][col].i;
            for (int r = col + 1; r < 6; r++) {
                double t = A[r][col].r * A[r][col].r + A[r][col].i * A[r][col].i;
                if (t > best) { best = t; piv = r; }
            }
            if (piv != col)
                for (int j = 0; j < 12; j++) { zd t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
            zd d = A[col][col];
            double dn = 1.0 / (d.r * d.r + d.i * d.i);
            zd inv = mk(d.r * dn, -d.i * dn);
            for (int j = 0; j < 12; j++) A[col][j] = inv * A[col][j];
            for (int r = 0; r < 6; r++) {
                if (r == col) continue;
                zd f = A[r][col];
                for (int j = 0; j < 12; j++) A[r][j] = A[r][j] - f * A[col][j];
            }
        }
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) {
                o[72 * b + (i * 6 + j) * 2] = A[i][6 + j].r;
                o[72 * b + (i * 6 + j) * 2 + 1] = A[i][6 + j].i;
            }
    }
    store_reals<P64, 144, double>((char*)out + (size_t)p * 72 * g.vh * sizeof(double2), g.vh, s, nullptr, 1.f, o);
}

// FP64 packed site records (NR reals, both parities) -> precision P
template <int P, int NR>
__global__ void convert_sites_kernel(const void* src, Geo g, void* dst, float* norm) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (s >= g.vh) return;
    double v[NR];
    load_reals<P64, NR, double>((const char*)src + (size_t)p * (NR / 2) * g.vh * sizeof(double2), g.vh, s, 1.f, v);
    typedef Layout<P, NR> Lay;
    char* base = (char*)dst + (size_t)p * Lay::NC * g.vh * sizeof(typename Lay::C);
    store_reals<P, NR, double>(base, g.vh, s, P == P16 ? norm + (size_t)p * g.vh : nullptr, 1.f, v);
}

static size_t rec_bytes(int prec, int nr, int vh) {
    return (size_t)2 * nr * prec_bytes(prec) * vh;
}

template <int NR>
static void make_precisions(Lattice& lat, void* d64, void* out[3], float** norm, cudaStream_t st) {
    dim3 grid((lat.vh + 127) / 128, 2);
    out[LQ_F64] = d64;
    out[LQ_F32] = dev_alloc(&lat, rec_bytes(LQ_F32, NR, lat.vh));
    out[LQ_F16] = dev_alloc(&lat, rec_bytes(LQ_F16, NR, lat.vh));
    out[LQ_F32X2] = dev_alloc(&lat, rec_bytes(LQ_F32X2, NR, lat.vh));
    *norm = (float*)dev_alloc(&lat, sizeof(float) * 2 * lat.vh);
    launch("convert_sites", convert_sites_kernel<P32, NR>, grid, dim3(128), st, (const void*)d64, lat.geo,
           out[LQ_F32], (float*)nullptr);
    launch("convert_sites", convert_sites_kernel<P16, NR>, grid, dim3(128), st, (const void*)d64, lat.geo,
           out[LQ_F16], *norm);
    launch("convert_sites", convert_sites_kernel<PDF, NR>, grid, dim3(128), st, (const void*)d64, lat.geo,
           out[LQ_F32X2], (float*)nullptr);
}

static void free_ainv_entry(Lattice& lat, Lattice::Ainv& a);

void free_clover(Lattice& lat) {
    for (int p = 0; p < 4; p++) {
        dev_free(&lat, lat.clovC[p], rec_bytes(p, 72, lat.vh));
        lat.clovC[p] = nullptr;
    }
    dev_free(&lat, lat.clovC_norm, sizeof(float) * 2 * lat.vh);
    lat.clovC_norm = nullptr;
    for (auto& kv : lat.ainv) free_ainv_entry(lat, kv.second);
    lat.ainv.clear();
    lat.has_clover = false;
}

void build_clover(Lattice& lat, double c_sw, cudaStream_t st) {
    if (!lat.canon[LQ_THIN]) fail(LQ_EINVAL, "lq_load_clover: thin gauge field not loaded");
    upload_sigma();
    free_clover(lat);
    void* d64 = dev_alloc(&lat, rec_bytes(LQ_F64, 72, lat.vh));
    dim3 grid((lat.vh + 63) / 64, 2);
    launch("clover_build", clover_build_kernel, grid, dim3(64), st, (const double*)lat.canon[LQ_THIN], lat.V,
           lat.geo, c_sw, d64);
    make_precisions<72>(lat, d64, lat.clovC, &lat.clovC_norm, st);
    LQ_CUDA(cudaStreamSynchronize(st));
    lat.has_clover = true;
    lat.c_sw = c_sw;
}

void load_clover_canonical(Lattice& lat, const double* canon_dev, cudaStream_t st) {
    free_clover(lat);
    void* d64 = dev_alloc(&lat, rec_bytes(LQ_F64, 72, lat.vh));
    dim3 grid((lat.vh + 127) / 128, 2);
    launch("clover_pack", clover_pack_kernel, grid, dim3(128), st, canon_dev, lat.geo, d64);
    make_precisions<72>(lat, d64, lat.clovC, &lat.clovC_norm, st);
    LQ_CUDA(cudaStreamSynchronize(st));
    lat.has_clover = true;
}

// builds A^{-1} in precision prec only (through a temporary FP64 copy)
void build_ainv(Lattice& lat, double m, double mu0, double mu1, int prec, Lattice::Ainv& out, cudaStream_t st) {
    void* d64 = dev_alloc(&lat, rec_bytes(LQ_F64, 144, lat.vh));
    dim3 grid((lat.vh + 63) / 64, 2);
    launch("clover_inverse", ainv_kernel, grid, dim3(64), st, (const void*)lat.clovC[LQ_F64], lat.geo, 4.0 + m, mu0,
           mu1, d64);
    if (prec == LQ_F64) {
        out.data[LQ_F64] = d64;
        return;
    }
    dim3 g2((lat.vh + 127) / 128, 2);
    out.data[prec] = dev_alloc(&lat, rec_bytes(prec, 144, lat.vh));
    if (prec == LQ_F32)
        launch("convert_sites", convert_sites_kernel<P32, 144>, g2, dim3(128), st, (const void*)d64, lat.geo,
               out.data[prec], (float*)nullptr);
    else if (prec == LQ_F32X2)
        launch("convert_sites", convert_sites_kernel<PDF, 144>, g2, dim3(128), st, (const void*)d64, lat.geo,
               out.data[prec], (float*)nullptr);
    else {
        if (!out.norm) out.norm = (float*)dev_alloc(&lat, sizeof(float) * 2 * lat.vh);
        launch("convert_sites", convert_sites_kernel<P16, 144>, g2, dim3(128), st, (const void*)d64, lat.geo,
               out.data[prec], out.norm);
    }
    LQ_CUDA(cudaStreamSynchronize(st));
    dev_free(&lat, d64, rec_bytes(LQ_F64, 144, lat.vh));
}

static void free_ainv_entry(Lattice& lat, Lattice::Ainv& a) {
    for (int p = 0; p < 4; p++) dev_free(&lat, a.data[p], rec_bytes(p, 144, lat.vh));
    dev_free(&lat, a.norm, sizeof(float) * 2 * lat.vh);
}

// drop least-recently-used unpinned entries beyond the cache size, never `keep` (lat.mu held)
static void trim_ainv(Lattice& lat, const std::tuple<double, double, double>* keep) {
    while (lat.ainv.size() > kAinvCache) {
        auto victim = lat.ainv.end();
        for (auto it = lat.ainv.begin(); it != lat.ainv.end(); ++it)
            if (it->second.pins == 0 && !(keep && it->first == *keep) &&
                (victim == lat.ainv.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == lat.ainv.end()) return;
        free_ainv_entry(lat, victim->second);
        lat.ainv.erase(victim);
    }
}

void pin_ainv(Lattice& lat, double m, double mu0, double mu1, bool pin) {
    std::lock_guard<std::mutex> lk(lat.mu);
    auto& e = lat.ainv[std::make_tuple(m, mu0, mu1)];
    e.last_use = ++lat.ainv_clock;
    e.pins += pin ? 1 : -1;
    if (!pin) trim_ainv(lat, nullptr);
}

const void* clover_block(Lattice& lat, int prec, int parity, const float** norm) {
    if (!lat.has_clover) fail(LQ_EINVAL, "clover term not loaded");
    size_t per = rec_bytes(prec, 72, lat.vh) / 2;
    *norm = prec == LQ_F16 ? lat.clovC_norm + (size_t)parity * lat.vh : nullptr;
    return (const char*)lat.clovC[prec] + per * parity;
}

const void* ainv_block(Lattice& lat, double m, double mu0, double mu1, int prec, int parity, const float** norm,
                       cudaStream_t st) {
    std::lock_guard<std::mutex> lk(lat.mu);
    if (!lat.has_clover) fail(LQ_EINVAL, "clover term not loaded");
    const auto key = std::make_tuple(m, mu0, mu1);
    auto& e = lat.ainv[key];
    e.last_use = ++lat.ainv_clock;
    if (!e.data[prec]) {
        if (stream_capturing(st)) fail(LQ_EINVAL, "clover inverse for a new (m, mu) requested during capture");
        build_ainv(lat, m, mu0, mu1, prec, e, st);
    }
    const void* ptr = (const char*)e.data[prec] + rec_bytes(prec, 144, lat.vh) / 2 * parity;
    *norm = prec == LQ_F16 ? e.norm + (size_t)parity * lat.vh : nullptr;
    if (lat.ainv.size() > kAinvCache) trim_ainv(lat, &key);
    return ptr;
}

}  // namespace lq
