/*
 * oracle.c -- plain FP64 CPU oracle for the lattice Dirac operators and Krylov
 * solvers of arXiv:2201.09004 ("Performance of the GPU inverters with
 * Chroma+QUDA for various fermion actions").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code with the CUDA library: the two meet only through
 * the seeded input arrays of paper_2201_09004_b300/synth.py.
 *
 * Everything here is the plain definition: full lattice (no even-odd split),
 * no link compression, FP64, one site at a time, loops in the order the
 * formulas are written. OpenMP only distributes independent sites.
 *
 * Canonical layouts (complex doubles, interleaved re/im, C order):
 *   gauge   [mu][t][z][y][x][3][3]    U_mu(x): transporter x -> x+mu
 *   spinor  [t][z][y][x][4][3]        [spin][colour]
 *   colour  [t][z][y][x][3]
 *   clover  [t][z][y][x][12][12]      row/col index = 3*spin + colour
 * Site index i = x + Lx*(y + Ly*(z + Lz*t)), dims L = {Lx, Ly, Lz, Lt}.
 *
 * Conventions (readings of the paper where it is silent or garbled):
 *   Wilson, Sec. 2.1 Eq. 2. The paper's D_w = (1/2) sum_{mu,eta} (1 + eta g_mu)
 *   U(x, x+eta mu) delta_{y,x+eta mu} - (4+m) delta_{xy}. The operator built
 *   here is M = -D_w with the same projectors:
 *     M psi(x) = (4+m) psi(x) + i mu g5 psi(x) + C(x) psi(x)
 *                - 1/2 sum_mu [(1+g_mu) U_mu(x) psi(x+mu) + (1-g_mu) U_mu(x-mu)^+ psi(x-mu)].
 *   The complex mass m_cri + omega of Sec. 2.1 Eq. 1 enters as a real part m
 *   and a twisted part i mu g5 (twist_mode 0); twist_mode 1 is the literal
 *   scalar complex mass (4 + m + i mu).
 *   Clover, Sec. 2.1 Eq. 3 (printed without normalisation), read as the
 *   standard Sheikholeslami-Wohlert term
 *     C(x) = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x),
 *     sigma_{mu nu} = (i/2)[g_mu, g_nu],
 *     Fhat = (Q - Q^+)/8 made traceless, Q the sum of the four plaquette
 *     leaves of the (mu,nu) plane that start and end at x.
 *   Gamma matrices: DeGrand-Rossi basis, g5 = g1 g2 g3 g4 = diag(1,1,-1,-1).
 *   Staggered/HISQ, Sec. 2.2 Eq. 4 with the fat one-hop and long three-hop
 *   links of the HISQ action:
 *     D psi(x) = m psi(x) + s_h H psi(x),
 *     H psi(x) = 1/2 sum_mu eta_mu(x) [V_mu(x) psi(x+mu) - V_mu(x-mu)^+ psi(x-mu)
 *                 + c_N (W_mu(x) psi(x+3mu) - W_mu(x-3mu)^+ psi(x-3mu))].
 *   Phases from the spin diagonalisation of Sec. 2.2: MILC ordering
 *   psi^st = g4^t g1^x g2^y g3^z psi gives eta_1=(-1)^t, eta_2=(-1)^(t+x),
 *   eta_3=(-1)^(t+x+y), eta_4=1; CPS ordering g1^x g2^y g3^z g4^t gives
 *   eta_1=1, eta_2=(-1)^x, eta_3=(-1)^(x+y), eta_4=(-1)^(x+y+z).
 *   Boundary: periodic in space; in time the sign bc_t (-1 = antiperiodic)
 *   multiplies every hop once per crossing of the t = Lt-1 -> 0 boundary.
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int L[4];
    int bc_t;
    int64_t V;
} geom;

typedef struct {
    int L[4];
    int bc_t;
    const cplx* U;       /* thin links */
    const cplx* clover;  /* NULL: no clover term */
    double m, mu;
    int twist_mode;      /* 0: i mu g5, 1: scalar i mu */
} or_wilson;

typedef struct {
    int L[4];
    int bc_t;
    const cplx* V;       /* fat links */
    const cplx* W;       /* long links (NULL: no Naik term) */
    double c_naik;
    double m;
    int conv;            /* 0: MILC phases, 1: CPS phases */
    int hop_sign;        /* +1: m + H (MILC/QUDA), -1: m - H (CPS/Chroma) */
} or_hisq;

/* ---------------------------------------------------------------- geometry */

static geom make_geom(const int L[4], int bc_t) {
    geom g;
    for (int d = 0; d < 4; d++) g.L[d] = L[d];
    g.bc_t = bc_t;
    g.V = (int64_t)L[0] * L[1] * L[2] * L[3];
    return g;
}

static void site_coords(const geom* g, int64_t i, int c[4]) {
    for (int d = 0; d < 4; d++) {
        c[d] = (int)(i % g->L[d]);
        i /= g->L[d];
    }
}

static int64_t site_index(const geom* g, const int c[4]) {
    return c[0] + (int64_t)g->L[0] * (c[1] + (int64_t)g->L[1] * (c[2] + (int64_t)g->L[2] * c[3]));
}

/* floor division for possibly negative a */
static int floordiv(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/* Site x + k*mu, and the boundary sign picked up on the way: bc_t raised to
 * the number of times the straight path crosses the time boundary. */
static int64_t hop(const geom* g, int64_t i, int mu, int k, double* sign) {
    int c[4];
    site_coords(g, i, c);
    int moved = c[mu] + k;
    int wraps = floordiv(moved, g->L[mu]);
    c[mu] = moved - wraps * g->L[mu];
    double s = 1.0;
    if (mu == 3 && g->bc_t == -1 && (wraps & 1)) s = -1.0;
    *sign = s;
    return site_index(g, c);
}

/* ----------------------------------------------------------- small algebra */

static const cplx* link(const cplx* U, int64_t V, int mu, int64_t i) { return U + (mu * V + i) * 9; }

static void su3_mul(const cplx* a, const cplx* b, cplx* c) {      /* c = a b */
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += a[r * 3 + k] * b[k * 3 + s];
            c[r * 3 + s] = acc;
        }
}

static void su3_dag(const cplx* a, cplx* c) {
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) c[r * 3 + s] = conj(a[s * 3 + r]);
}

static void mat_vec(const cplx* a, const cplx* v, cplx* out) {    /* out = a v */
    for (int r = 0; r < 3; r++) {
        cplx acc = 0;
        for (int k = 0; k < 3; k++) acc += a[r * 3 + k] * v[k];
        out[r] = acc;
    }
}

static void mat_dag_vec(const cplx* a, const cplx* v, cplx* out) {  /* out = a^+ v */
    for (int r = 0; r < 3; r++) {
        cplx acc = 0;
        for (int k = 0; k < 3; k++) acc += conj(a[k * 3 + r]) * v[k];
        out[r] = acc;
    }
}

/* DeGrand-Rossi gamma matrices, index [mu][row][col], mu = 0..3 for x,y,z,t:
 *   g1 = [[0, i s1], [-i s1, 0]], g2 = [[0, -i s2], [i s2, 0]],
 *   g3 = [[0, i s3], [-i s3, 0]], g4 = [[0, 1], [1, 0]]. */
static cplx GAMMA[4][4][4];
static cplx GAMMA5[4][4];
static int gamma_ready = 0;

static void init_gamma(void) {
    if (gamma_ready) return;
    memset(GAMMA, 0, sizeof(GAMMA));
    /* g1 */
    GAMMA[0][0][3] = I;  GAMMA[0][1][2] = I;  GAMMA[0][2][1] = -I; GAMMA[0][3][0] = -I;
    /* g2 */
    GAMMA[1][0][3] = -1; GAMMA[1][1][2] = 1;  GAMMA[1][2][1] = 1;  GAMMA[1][3][0] = -1;
    /* g3 */
    GAMMA[2][0][2] = I;  GAMMA[2][1][3] = -I; GAMMA[2][2][0] = -I; GAMMA[2][3][1] = I;
    /* g4 */
    GAMMA[3][0][2] = 1;  GAMMA[3][1][3] = 1;  GAMMA[3][2][0] = 1;  GAMMA[3][3][1] = 1;
    /* g5 = g1 g2 g3 g4 */
    cplx t1[4][4], t2[4][4];
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += GAMMA[0][a][k] * GAMMA[1][k][b];
            t1[a][b] = s;
        }
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += t1[a][k] * GAMMA[2][k][b];
            t2[a][b] = s;
        }
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += t2[a][k] * GAMMA[3][k][b];
            GAMMA5[a][b] = s;
        }
    gamma_ready = 1;
}

/* export the basis so the tests can check the Clifford algebra */
void or_gamma(int mu, double* out /* [4][4][2] */) {
    init_gamma();
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            cplx v = (mu == 4) ? GAMMA5[a][b] : GAMMA[mu][a][b];
            out[(a * 4 + b) * 2] = creal(v);
            out[(a * 4 + b) * 2 + 1] = cimag(v);
        }
}

/* ------------------------------------------------------- Wilson hopping term */

/* (H psi)(x) for one site. Sec. 2.1 Eq. 2, sign flipped (M = -D_w):
 *   H psi(x) = 1/2 sum_mu [(1+g_mu) U_mu(x) psi(x+mu) + (1-g_mu) U_mu(x-mu)^+ psi(x-mu)].
 * The adjoint H^+ has matrix elements H^+(x,y) = H(y,x)^+. With
 * H(x-mu, x) = 1/2 (1+g_mu) U_mu(x-mu) and H(x+mu, x) = 1/2 (1-g_mu) U_mu(x)^+,
 * and hermitian g_mu, this is
 *   H^+ psi(x) = 1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu)]. */
static void wilson_hop_site(const geom* g, const cplx* U, int dagger, const cplx* in, int64_t i,
                            cplx out[12]) {
    for (int k = 0; k < 12; k++) out[k] = 0;
    double pf = dagger ? -1.0 : 1.0;  /* sign of g_mu in the forward projector */
    for (int mu = 0; mu < 4; mu++) {
        for (int dir = 0; dir < 2; dir++) {
            double sgn;
            int64_t j = hop(g, i, mu, dir == 0 ? +1 : -1, &sgn);
            const cplx* psi = in + j * 12;
            cplx upsi[4][3];
            for (int s = 0; s < 4; s++) {
                if (dir == 0)
                    mat_vec(link(U, g->V, mu, i), psi + 3 * s, upsi[s]);
                else
                    mat_dag_vec(link(U, g->V, mu, j), psi + 3 * s, upsi[s]);
            }
            double gs = (dir == 0) ? pf : -pf;  /* projector (1 + gs g_mu) */
            for (int a = 0; a < 4; a++)
                for (int c = 0; c < 3; c++) {
                    cplx acc = upsi[a][c];
                    for (int b = 0; b < 4; b++) acc += gs * GAMMA[mu][a][b] * upsi[b][c];
                    out[a * 3 + c] += 0.5 * sgn * acc;
                }
        }
    }
}

/* (M psi)(x) (or M^+ when dagger) for one site:
 *   M = (4+m) + i mu g5 + C - H,  M^+ = (4+m) - i mu g5 + C - H^+  (C hermitian). */
static void wilson_M_site(const or_wilson* p, const geom* g, int dagger, const cplx* in, int64_t i,
                          cplx out[12]) {
    cplx h[12];
    wilson_hop_site(g, p->U, dagger, in, i, h);
    const cplx* psi = in + i * 12;
    double tw = dagger ? -p->mu : p->mu;
    for (int a = 0; a < 4; a++)
        for (int c = 0; c < 3; c++) {
            cplx v = (4.0 + p->m) * psi[a * 3 + c];
            if (p->twist_mode == 0) {
                for (int b = 0; b < 4; b++) v += I * tw * GAMMA5[a][b] * psi[b * 3 + c];
            } else {
                v += I * tw * psi[a * 3 + c];
            }
            out[a * 3 + c] = v - h[a * 3 + c];
        }
    if (p->clover) {
        const cplx* C = p->clover + i * 144;
        for (int r = 0; r < 12; r++) {
            cplx acc = 0;
            for (int k = 0; k < 12; k++) acc += C[r * 12 + k] * psi[k];
            out[r] += acc;
        }
    }
}

void or_wilson_hop(const int L[4], int bc_t, const double* U, int dagger, const double* in, double* out) {
    init_gamma();
    geom g = make_geom(L, bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g.V; i++)
        wilson_hop_site(&g, (const cplx*)U, dagger, (const cplx*)in, i, (cplx*)out + i * 12);
}

void or_wilson_apply(const or_wilson* p, int dagger, const double* in, double* out) {
    init_gamma();
    geom g = make_geom(p->L, p->bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g.V; i++)
        wilson_M_site(p, &g, dagger, (const cplx*)in, i, (cplx*)out + i * 12);
}

/* M psi at a list of sites only: out[k] = (M psi)(sites[k]) */
void or_wilson_apply_sites(const or_wilson* p, int dagger, const double* in, const int64_t* sites,
                           int64_t nsites, double* out) {
    init_gamma();
    geom g = make_geom(p->L, p->bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nsites; k++)
        wilson_M_site(p, &g, dagger, (const cplx*)in, sites[k], (cplx*)out + k * 12);
}

void or_wilson_hop_sites(const int L[4], int bc_t, const double* U, int dagger, const double* in,
                         const int64_t* sites, int64_t nsites, double* out) {
    init_gamma();
    geom g = make_geom(L, bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nsites; k++)
        wilson_hop_site(&g, (const cplx*)U, dagger, (const cplx*)in, sites[k], (cplx*)out + k * 12);
}

/* ------------------------------------------------------------------ clover */

/* Sum of the four plaquette leaves of the (mu,nu) plane that start and end at
 * x, all with the same orientation (mu then nu):
 *   U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *   U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
 *   U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
 *   U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
 * Links carry no boundary sign: each closed loop crosses any boundary an even
 * number of times. */
static void clover_leaves(const geom* g, const cplx* U, int64_t x, int mu, int nu, cplx Q[9]) {
    double s;
    int64_t xpm = hop(g, x, mu, +1, &s), xpn = hop(g, x, nu, +1, &s);
    int64_t xmm = hop(g, x, mu, -1, &s), xmn = hop(g, x, nu, -1, &s);
    int64_t xpn_mm = hop(g, xpn, mu, -1, &s);
    int64_t xmm_mn = hop(g, xmm, nu, -1, &s);
    int64_t xmn_pm = hop(g, xmn, mu, +1, &s);
    int64_t V = g->V;
    cplx a[9], b[9], t[9], t2[9], leaf[9];
    for (int k = 0; k < 9; k++) Q[k] = 0;

    /* leaf 1 */
    su3_mul(link(U, V, mu, x), link(U, V, nu, xpm), t);
    su3_dag(link(U, V, mu, xpn), a);
    su3_mul(t, a, t2);
    su3_dag(link(U, V, nu, x), b);
    su3_mul(t2, b, leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];

    /* leaf 2 */
    su3_dag(link(U, V, mu, xpn_mm), a);
    su3_mul(link(U, V, nu, x), a, t);
    su3_dag(link(U, V, nu, xmm), b);
    su3_mul(t, b, t2);
    su3_mul(t2, link(U, V, mu, xmm), leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];

    /* leaf 3 */
    su3_dag(link(U, V, mu, xmm), a);
    su3_dag(link(U, V, nu, xmm_mn), b);
    su3_mul(a, b, t);
    su3_mul(t, link(U, V, mu, xmm_mn), t2);
    su3_mul(t2, link(U, V, nu, xmn), leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];

    /* leaf 4 */
    su3_dag(link(U, V, nu, xmn), a);
    su3_mul(a, link(U, V, mu, xmn), t);
    su3_mul(t, link(U, V, nu, xmn_pm), t2);
    su3_dag(link(U, V, mu, x), b);
    su3_mul(t2, b, leaf);
    for (int k = 0; k < 9; k++) Q[k] += leaf[k];
}

/* C(x) = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x), a 12x12 matrix
 * per site with index 3*spin + colour (Sec. 2.1 Eq. 3, standard normalisation). */
void or_clover_build(const int L[4], const double* Ud, double c_sw, double* out) {
    init_gamma();
    geom g = make_geom(L, 1);
    const cplx* U = (const cplx*)Ud;
    /* sigma_{mu nu} = (i/2) (g_mu g_nu - g_nu g_mu) */
    static cplx sigma[4][4][4][4];
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++)
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) {
                    cplx s = 0;
                    for (int k = 0; k < 4; k++)
                        s += GAMMA[mu][a][k] * GAMMA[nu][k][b] - GAMMA[nu][a][k] * GAMMA[mu][k][b];
                    sigma[mu][nu][a][b] = 0.5 * I * s;
                }
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < g.V; x++) {
        cplx* C = (cplx*)out + x * 144;
        for (int k = 0; k < 144; k++) C[k] = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                cplx Q[9], F[9];
                clover_leaves(&g, U, x, mu, nu, Q);
                for (int r = 0; r < 3; r++)
                    for (int s = 0; s < 3; s++) F[r * 3 + s] = (Q[r * 3 + s] - conj(Q[s * 3 + r])) / 8.0;
                cplx tr = (F[0] + F[4] + F[8]) / 3.0;
                F[0] -= tr; F[4] -= tr; F[8] -= tr;
                for (int a = 0; a < 4; a++)
                    for (int b = 0; b < 4; b++)
                        for (int r = 0; r < 3; r++)
                            for (int s = 0; s < 3; s++)
                                C[(a * 3 + r) * 12 + (b * 3 + s)] +=
                                    c_sw * 0.5 * I * sigma[mu][nu][a][b] * F[r * 3 + s];
            }
    }
}

/* average plaquette <Re tr P>/3 over sites and the six planes */
double or_plaquette(const int L[4], const double* Ud) {
    geom g = make_geom(L, 1);
    const cplx* U = (const cplx*)Ud;
    double sum = 0.0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
    for (int64_t x = 0; x < g.V; x++) {
        double s;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                int64_t xpm = hop(&g, x, mu, +1, &s), xpn = hop(&g, x, nu, +1, &s);
                cplx t[9], a[9], t2[9], b[9], P[9];
                su3_mul(link(U, g.V, mu, x), link(U, g.V, nu, xpm), t);
                su3_dag(link(U, g.V, mu, xpn), a);
                su3_mul(t, a, t2);
                su3_dag(link(U, g.V, nu, x), b);
                su3_mul(t2, b, P);
                sum += creal(P[0] + P[4] + P[8]) / 3.0;
            }
    }
    return sum / (6.0 * (double)g.V);
}

/* ------------------------------------------------------------ staggered/HISQ */

static double eta(int conv, int mu, const int c[4]) {
    int e;
    if (conv == 0) {         /* MILC: psi^st = g4^t g1^x g2^y g3^z psi */
        switch (mu) {
            case 0: e = c[3]; break;
            case 1: e = c[3] + c[0]; break;
            case 2: e = c[3] + c[0] + c[1]; break;
            default: e = 0; break;
        }
    } else {                 /* CPS: psi^st = g1^x g2^y g3^z g4^t psi */
        switch (mu) {
            case 0: e = 0; break;
            case 1: e = c[0]; break;
            case 2: e = c[0] + c[1]; break;
            default: e = c[0] + c[1] + c[2]; break;
        }
    }
    return (e & 1) ? -1.0 : 1.0;
}

void or_staggered_eta(int conv, int mu, const int c[4], double* out) { *out = eta(conv, mu, c); }

/* One hop term of H with its matrix element written from x's side.
 * Forward:  H(x, x+k mu) = +1/2 coef eta_mu(x) L_mu(x)
 * Backward: H(x, x-k mu) = -1/2 coef eta_mu(x) L_mu(x-k mu)^+
 * (L = V for k = 1 with coef 1, L = W for k = 3 with coef c_N.) */
static void hisq_H_site(const or_hisq* p, const geom* g, int dagger, const cplx* in, int64_t i, cplx out[3]) {
    int c[4];
    site_coords(g, i, c);
    for (int k = 0; k < 3; k++) out[k] = 0;
    for (int mu = 0; mu < 4; mu++) {
        for (int which = 0; which < 2; which++) {
            const cplx* L = which == 0 ? p->V : p->W;
            if (!L) continue;
            int step = which == 0 ? 1 : 3;
            double coef = which == 0 ? 1.0 : p->c_naik;
            double sf, sb;
            int64_t jf = hop(g, i, mu, +step, &sf);
            int64_t jb = hop(g, i, mu, -step, &sb);
            cplx t[3];
            if (!dagger) {
                double e = eta(p->conv, mu, c);
                mat_vec(link(L, g->V, mu, i), in + jf * 3, t);
                for (int k = 0; k < 3; k++) out[k] += 0.5 * coef * e * sf * t[k];
                mat_dag_vec(link(L, g->V, mu, jb), in + jb * 3, t);
                for (int k = 0; k < 3; k++) out[k] -= 0.5 * coef * e * sb * t[k];
            } else {
                /* H^+(x,y) = H(y,x)^+:
                 *   y = x - k mu: H(y, y + k mu)^+ = 1/2 coef eta_mu(y) L_mu(y)^+
                 *   y = x + k mu: H(y, y - k mu)^+ = -1/2 coef eta_mu(y) L_mu(x)   */
                int cf[4], cb[4];
                site_coords(g, jf, cf);
                site_coords(g, jb, cb);
                mat_dag_vec(link(L, g->V, mu, jb), in + jb * 3, t);
                for (int k = 0; k < 3; k++) out[k] += 0.5 * coef * eta(p->conv, mu, cb) * sb * t[k];
                mat_vec(link(L, g->V, mu, i), in + jf * 3, t);
                for (int k = 0; k < 3; k++) out[k] -= 0.5 * coef * eta(p->conv, mu, cf) * sf * t[k];
            }
        }
    }
}

static void hisq_D_site(const or_hisq* p, const geom* g, int dagger, const cplx* in, int64_t i, cplx out[3]) {
    cplx h[3];
    hisq_H_site(p, g, dagger, in, i, h);
    for (int k = 0; k < 3; k++) out[k] = p->m * in[i * 3 + k] + p->hop_sign * h[k];
}

void or_hisq_hop(const or_hisq* p, int dagger, const double* in, double* out) {
    geom g = make_geom(p->L, p->bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g.V; i++) hisq_H_site(p, &g, dagger, (const cplx*)in, i, (cplx*)out + i * 3);
}

void or_hisq_apply(const or_hisq* p, int dagger, const double* in, double* out) {
    geom g = make_geom(p->L, p->bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g.V; i++) hisq_D_site(p, &g, dagger, (const cplx*)in, i, (cplx*)out + i * 3);
}

void or_hisq_hop_sites(const or_hisq* p, int dagger, const double* in, const int64_t* sites, int64_t n,
                       double* out) {
    geom g = make_geom(p->L, p->bc_t);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k++) hisq_H_site(p, &g, dagger, (const cplx*)in, sites[k], (cplx*)out + k * 3);
}

/* ------------------------------------------------------------ vector algebra */

static cplx vdot(int64_t n, const cplx* a, const cplx* b) {  /* sum conj(a) b */
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int64_t k = 0; k < n; k++) {
        cplx t = conj(a[k]) * b[k];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

static double vnorm2(int64_t n, const cplx* a) {
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t k = 0; k < n; k++) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
    return s;
}

/* y += a x */
static void vaxpy(int64_t n, cplx a, const cplx* x, cplx* y) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k++) y[k] += a * x[k];
}

/* ------------------------------------------------------------------ solvers */

typedef void (*op_fn)(const void* ctx, int dagger, const cplx* in, cplx* out);

static void wilson_op(const void* ctx, int dagger, const cplx* in, cplx* out) {
    or_wilson_apply((const or_wilson*)ctx, dagger, (const double*)in, (double*)out);
}

static void hisq_op(const void* ctx, int dagger, const cplx* in, cplx* out) {
    or_hisq_apply((const or_hisq*)ctx, dagger, (const double*)in, (double*)out);
}

/* CG on the normal equations M^+ M x = M^+ b (CGNR):
 *   x = 0, s = b, r = M^+ s, p = r;
 *   loop: q = M p; alpha = |r|^2/|q|^2; x += alpha p; s -= alpha q;
 *         r' = M^+ s; beta = |r'|^2/|r|^2; p = r' + beta p;
 *   stop when |s|/|b| <= tol (s is the residual b - M x of the system itself). */
static int cgnr(op_fn A, const void* ctx, int64_t n, const cplx* b, cplx* x, double tol, int maxiter,
                int* iters, double* relres) {
    cplx* s = malloc(n * sizeof(cplx));
    cplx* r = malloc(n * sizeof(cplx));
    cplx* p = malloc(n * sizeof(cplx));
    cplx* q = malloc(n * sizeof(cplx));
    memset(x, 0, n * sizeof(cplx));
    memcpy(s, b, n * sizeof(cplx));
    double bb = vnorm2(n, b);
    A(ctx, 1, s, r);
    memcpy(p, r, n * sizeof(cplx));
    double rr = vnorm2(n, r);
    double ss = bb;
    int k = 0;
    while (k < maxiter && sqrt(ss / bb) > tol) {
        A(ctx, 0, p, q);
        double alpha = rr / vnorm2(n, q);
        vaxpy(n, alpha, p, x);
        vaxpy(n, -alpha, q, s);
        ss = vnorm2(n, s);
        A(ctx, 1, s, r);
        double rr_new = vnorm2(n, r);
        double beta = rr_new / rr;
        rr = rr_new;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) p[j] = r[j] + beta * p[j];
        k++;
    }
    /* true residual */
    A(ctx, 0, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) q[j] = b[j] - q[j];
    *relres = sqrt(vnorm2(n, q) / bb);
    *iters = k;
    free(s); free(r); free(p); free(q);
    return (sqrt(ss / bb) <= tol) ? 0 : 1;
}

/* BiCGStab (van der Vorst 1992) on M x = b, stop when |r|/|b| <= tol. */
static int bicgstab(op_fn A, const void* ctx, int64_t n, const cplx* b, cplx* x, double tol, int maxiter,
                    int* iters, double* relres) {
    cplx* r = malloc(n * sizeof(cplx));
    cplx* rhat = malloc(n * sizeof(cplx));
    cplx* p = malloc(n * sizeof(cplx));
    cplx* v = malloc(n * sizeof(cplx));
    cplx* s = malloc(n * sizeof(cplx));
    cplx* t = malloc(n * sizeof(cplx));
    memset(x, 0, n * sizeof(cplx));
    memcpy(r, b, n * sizeof(cplx));
    memcpy(rhat, b, n * sizeof(cplx));
    memset(p, 0, n * sizeof(cplx));
    memset(v, 0, n * sizeof(cplx));
    double bb = vnorm2(n, b);
    cplx rho = 1, alpha = 1, omega = 1;
    double rr = bb;
    int k = 0, status = 0;
    while (k < maxiter && sqrt(rr / bb) > tol) {
        cplx rho_new = vdot(n, rhat, r);
        if (cabs(rho_new) == 0.0) { status = 2; break; }
        cplx beta = (rho_new / rho) * (alpha / omega);
        rho = rho_new;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) p[j] = r[j] + beta * (p[j] - omega * v[j]);
        A(ctx, 0, p, v);
        alpha = rho / vdot(n, rhat, v);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) s[j] = r[j] - alpha * v[j];
        A(ctx, 0, s, t);
        omega = vdot(n, t, s) / vdot(n, t, t);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) {
            x[j] += alpha * p[j] + omega * s[j];
            r[j] = s[j] - omega * t[j];
        }
        rr = vnorm2(n, r);
        k++;
    }
    A(ctx, 0, x, t);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) t[j] = b[j] - t[j];
    *relres = sqrt(vnorm2(n, t) / bb);
    *iters = k;
    free(r); free(rhat); free(p); free(v); free(s); free(t);
    if (status) return status;
    return (sqrt(rr / bb) <= tol) ? 0 : 1;
}

int or_wilson_cgnr(const or_wilson* p, const double* b, double* x, double tol, int maxiter, int* iters,
                   double* relres) {
    init_gamma();
    int64_t n = (int64_t)p->L[0] * p->L[1] * p->L[2] * p->L[3] * 12;
    return cgnr(wilson_op, p, n, (const cplx*)b, (cplx*)x, tol, maxiter, iters, relres);
}

int or_wilson_bicgstab(const or_wilson* p, const double* b, double* x, double tol, int maxiter, int* iters,
                       double* relres) {
    init_gamma();
    int64_t n = (int64_t)p->L[0] * p->L[1] * p->L[2] * p->L[3] * 12;
    return bicgstab(wilson_op, p, n, (const cplx*)b, (cplx*)x, tol, maxiter, iters, relres);
}

/* Threads of the OpenMP loops over sites (timing on a stated number of cores). */
void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int or_get_threads(void) { return omp_get_max_threads(); }

/* A fixed number of CGNR iterations (for timing a bounded sample). */
double or_wilson_cgnr_fixed(const or_wilson* p, const double* b, double* x, int niter) {
    init_gamma();
    int64_t n = (int64_t)p->L[0] * p->L[1] * p->L[2] * p->L[3] * 12;
    int it;
    double rel;
    cgnr(wilson_op, p, n, (const cplx*)b, (cplx*)x, 0.0, niter, &it, &rel);
    return rel;
}

int or_hisq_cgnr(const or_hisq* p, const double* b, double* x, double tol, int maxiter, int* iters,
                 double* relres) {
    int64_t n = (int64_t)p->L[0] * p->L[1] * p->L[2] * p->L[3] * 3;
    return cgnr(hisq_op, p, n, (const cplx*)b, (cplx*)x, tol, maxiter, iters, relres);
}

/* Multi-shift CG (Jegerlehner) for (A + sigma_i) x_i = b with A hermitian
 * positive definite and sigma_0 <= sigma_i. One Krylov space, that of
 * A + sigma_0; the other shifts follow from the collinearity of the residuals
 * r_i = zeta_i r:
 *   init: x_i = 0, p_i = r = b, zeta_i = zeta_i^prev = 1, alpha_prev = 1, beta_prev = 0;
 *   q = (A + sigma_0) p_0, alpha = (r,r)/(p_0,q);
 *   zeta_i' = zeta_i zeta_i^prev alpha_prev /
 *             [alpha beta_prev (zeta_i^prev - zeta_i) + zeta_i^prev alpha_prev (1 + (sigma_i - sigma_0) alpha)];
 *   alpha_i = alpha zeta_i'/zeta_i;  x_i += alpha_i p_i;  r -= alpha q;
 *   beta = (r',r')/(r,r);  p_0 = r' + beta p_0;  p_i = zeta_i' r' + beta (zeta_i'/zeta_i)^2 p_i.
 * Shift i is converged when |zeta_i| |r| / |b| <= tol. */
static int multishift_cg(void (*apply_A)(const void*, const cplx*, cplx*), const void* ctx, int64_t n,
                         int nshift, const double* sigma, const cplx* b, cplx** x, double tol, int maxiter,
                         int* iters) {
    cplx* r = malloc(n * sizeof(cplx));
    cplx* q = malloc(n * sizeof(cplx));
    cplx** p = malloc(nshift * sizeof(cplx*));
    double* zeta = malloc(nshift * sizeof(double));
    double* zeta_prev = malloc(nshift * sizeof(double));
    int* active = malloc(nshift * sizeof(int));
    for (int i = 0; i < nshift; i++) {
        p[i] = malloc(n * sizeof(cplx));
        memcpy(p[i], b, n * sizeof(cplx));
        memset(x[i], 0, n * sizeof(cplx));
        zeta[i] = zeta_prev[i] = 1.0;
        active[i] = 1;
    }
    memcpy(r, b, n * sizeof(cplx));
    double bb = vnorm2(n, b), rr = bb;
    double alpha_prev = 1.0, beta_prev = 0.0;
    int k = 0;
    while (k < maxiter && sqrt(rr / bb) > tol) {
        apply_A(ctx, p[0], q);
        vaxpy(n, sigma[0], p[0], q);
        double alpha = rr / creal(vdot(n, p[0], q));
        double zeta_new[64];
        for (int i = 1; i < nshift; i++) {
            double d = sigma[i] - sigma[0];
            double den = alpha * beta_prev * (zeta_prev[i] - zeta[i]) +
                         zeta_prev[i] * alpha_prev * (1.0 + d * alpha);
            zeta_new[i] = zeta[i] * zeta_prev[i] * alpha_prev / den;
        }
        vaxpy(n, alpha, p[0], x[0]);
        for (int i = 1; i < nshift; i++)
            if (active[i]) vaxpy(n, alpha * zeta_new[i] / zeta[i], p[i], x[i]);
        vaxpy(n, -alpha, q, r);
        double rr_new = vnorm2(n, r);
        double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) p[0][j] = r[j] + beta * p[0][j];
        for (int i = 1; i < nshift; i++) {
            if (active[i]) {
                double zr = zeta_new[i] / zeta[i];
#pragma omp parallel for schedule(static)
                for (int64_t j = 0; j < n; j++) p[i][j] = zeta_new[i] * r[j] + beta * zr * zr * p[i][j];
            }
            zeta_prev[i] = zeta[i];
            zeta[i] = zeta_new[i];
            if (fabs(zeta[i]) * sqrt(rr_new / bb) <= tol) active[i] = 0;
        }
        rr = rr_new;
        alpha_prev = alpha;
        beta_prev = beta;
        k++;
    }
    *iters = k;
    for (int i = 0; i < nshift; i++) free(p[i]);
    free(p); free(r); free(q); free(zeta); free(zeta_prev); free(active);
    return sqrt(rr / bb) <= tol ? 0 : 1;
}

/* A = H^+ H for the staggered hopping term (hermitian, positive semi-definite) */
static void hisq_normal(const void* ctx, const cplx* in, cplx* out) {
    const or_hisq* p = (const or_hisq*)ctx;
    int64_t n = (int64_t)p->L[0] * p->L[1] * p->L[2] * p->L[3] * 3;
    cplx* t = malloc(n * sizeof(cplx));
    or_hisq_hop(p, 0, (const double*)in, (double*)t);
    or_hisq_hop(p, 1, (const double*)t, (double*)out);
    free(t);
}

/* Solves D_i x_i = b with D_i = m_i + s_h H for every mass m_i at once.
 * Multi-shift CG on A = H^+ H with shifts m_i^2 gives y_i = (H^+ H + m_i^2)^{-1} b;
 * then x_i = D_i^+ y_i. This is D_i^{-1} b exactly when D_i D_i^+ = H^+ H + m_i^2,
 * i.e. when H is anti-hermitian (H^+ = -H), a property of Eq. 4 that the tests
 * check separately. The true residual |b - D_i x_i|/|b| of every mass is
 * recomputed and returned in relres. Masses must be sorted ascending. */
int or_hisq_multishift(const or_hisq* p, int nmass, const double* masses, const double* b, double** x,
                       double tol, int maxiter, int* iters, double* relres) {
    int64_t n = (int64_t)p->L[0] * p->L[1] * p->L[2] * p->L[3] * 3;
    if (nmass < 1 || nmass > 64) return 3;
    double sigma[64];
    cplx* y[64];
    for (int i = 0; i < nmass; i++) {
        sigma[i] = masses[i] * masses[i];
        y[i] = malloc(n * sizeof(cplx));
    }
    int st = multishift_cg(hisq_normal, p, n, nmass, sigma, (const cplx*)b, y, tol, maxiter, iters);
    cplx* t = malloc(n * sizeof(cplx));
    for (int i = 0; i < nmass; i++) {
        or_hisq pi = *p;
        pi.m = masses[i];
        or_hisq_apply(&pi, 1, (const double*)y[i], x[i]);
        or_hisq_apply(&pi, 0, x[i], (double*)t);
        const cplx* bc = (const cplx*)b;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) t[j] = bc[j] - t[j];
        relres[i] = sqrt(vnorm2(n, t) / vnorm2(n, bc));
        free(y[i]);
    }
    free(t);
    return st;
}
