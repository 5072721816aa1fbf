/*
 * lq.h -- C ABI of the B300 lattice Dirac-operator library.
 *
 * The library applies the lattice Dirac operators of arXiv:2201.09004
 * ("Performance of the GPU inverters with Chroma+QUDA for various fermion
 * actions") and solves D x = b with them, on one CUDA GPU:
 *   - Wilson twisted mass, optional clover term: Sec. 2.1, Eq. 1-3;
 *   - HISQ staggered with fat one-hop and long three-hop links: Sec. 2.2, Eq. 4.
 * The paper's own contribution is an interface through which an application
 * calls GPU inverters for several actions (Sec. 1, Sec. 3); this header is that
 * interface for this library.
 *
 * Conventions (the paper is silent or garbled on these; every entry point uses them):
 *   Geometry: dims = {Lx, Ly, Lz, Lt}, all even and >= 2. Site index
 *     i = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) & 1, even = 0.
 *     Periodic in space; in time the boundary sign t_boundary (+1 or -1)
 *     multiplies each hop once per crossing of t = Lt-1 -> 0.
 *   Links: U_mu(x) transports from x+mu to x; the backward hop uses U_mu(x-mu)^+.
 *   Gamma matrices: DeGrand-Rossi basis, g5 = g1 g2 g3 g4 = diag(1,1,-1,-1).
 *   Wilson operator (Sec. 2.1 Eq. 2 with an overall sign -1):
 *     M = (4+m) + i mu g5 + C - H,
 *     H psi(x) = 1/2 sum_mu [(1+g_mu) U_mu(x) psi(x+mu) + (1-g_mu) U_mu(x-mu)^+ psi(x-mu)].
 *     The complex mass of Sec. 2.1 Eq. 1 is m + i mu g5 (twisted reading).
 *   Clover (Sec. 2.1 Eq. 3): C = c_sw (i/2) sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu},
 *     sigma = (i/2)[g_mu, g_nu], Fhat = (Q - Q^+)/8 traceless, Q = sum of the
 *     four plaquette leaves at x.
 *   Staggered/HISQ (Sec. 2.2 Eq. 4): D = m + H,
 *     H psi(x) = 1/2 sum_mu eta_mu(x) [V_mu(x) psi(x+mu) - V_mu(x-mu)^+ psi(x-mu)
 *                 + c_naik (W_mu(x) psi(x+3mu) - W_mu(x-3mu)^+ psi(x-3mu))],
 *     MILC phases eta_1 = (-1)^t, eta_2 = (-1)^(t+x), eta_3 = (-1)^(t+x+y), eta_4 = 1.
 *
 * Canonical layouts (FP64 complex, interleaved re/im, C order) used by every
 * pointer argument below unless stated otherwise:
 *   gauge    [mu][t][z][y][x][3][3]        (4*V*9 complex)
 *   spinor   [t][z][y][x][spin 4][colour 3] (V*12 complex)
 *   colour   [t][z][y][x][colour 3]         (V*3 complex)
 *   clover   [t][z][y][x][12][12]           (V*144 complex, index 3*spin+colour)
 *
 * Errors: every function returns an lq_status; LQ_OK is 0. No C++ exception
 * crosses this boundary. lq_last_error() gives a thread-local message for the
 * last failure on the calling thread.
 *
 * Memory: the library copies what it is given (gauge, clover) into its own
 * device memory, which lives until lq_destroy_lattice. Caller buffers (sources,
 * solutions) stay owned by the caller; loc says whether a pointer is host or
 * device memory. Nothing returned by the library must be freed by the caller.
 *
 * Threads: a lattice handle may be used by one thread at a time. The server
 * functions are thread-safe.
 */
#ifndef LQ_H
#define LQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lq_lattice_s* lq_lattice;
typedef struct lq_server_s* lq_server;
typedef struct lq_field_s* lq_field;

typedef enum {
    LQ_OK = 0,
    LQ_EINVAL = 1,      /* bad argument (odd extent, null pointer, unknown enum, missing gauge) */
    LQ_ENOMEM = 2,      /* device or host allocation failed, or over the server's HBM budget */
    LQ_ENOTCONV = 3,    /* solver hit maxiter; x holds the best iterate, info is filled */
    LQ_EBREAKDOWN = 4,  /* Krylov breakdown (non-positive curvature) */
    LQ_ENAN = 5,        /* NaN or Inf in the source or during the solve */
    LQ_EAGAIN = 6,      /* lq_poll: the request is not finished yet */
    LQ_ETIMEOUT = 7,    /* lq_wait timed out */
    LQ_ECUDA = 8,       /* a CUDA runtime call failed; see lq_last_error */
    LQ_EBUSY = 9        /* server is shutting down or the queue is full */
} lq_status;

/* F16 = 16-bit fixed point + per-site norm, FP32 arithmetic. F32X2 = "double-float":
 * each real is a pair of FP32 numbers (hi + lo, ~48 significant bits) stored in 8
 * bytes and computed on the FP32 pipes; the mixed-precision solvers use it for
 * their FP64-accuracy steps because B300's FP64 rate is 1/64 of its FP32 rate. */
typedef enum { LQ_F64 = 0, LQ_F32 = 1, LQ_F16 = 2, LQ_F32X2 = 3 } lq_prec;
/* Link compression, for SU(3) links (thin Wilson links, HISQ long links; fat links
 * are always R18). R12: rows 0 and 1, row 2 = conj(row0 x row1). R8: u01, u02, u10
 * and the phases of u00 and u20; the rest follows from unitarity and det = 1
 * (LQ_F32 / LQ_F16 only; undefined where |u00| = 1, e.g. a unit gauge field, which
 * the packing step rejects with LQ_EINVAL). */
typedef enum { LQ_R18 = 18, LQ_R12 = 12, LQ_R8 = 8 } lq_recon;
typedef enum { LQ_THIN = 0, LQ_FAT = 1, LQ_LONG = 2 } lq_gauge_kind;
typedef enum { LQ_HOST = 0, LQ_DEVICE = 1 } lq_loc;
typedef enum { LQ_WILSON_TM = 0, LQ_WILSON_TM_CLOVER = 1, LQ_HISQ = 2 } lq_action;
/* The paper's complex mass m_cri + omega (Sec. 2.1 Eq. 1) read as the twisted mass
 * i mu g5 (default), or literally as the scalar i mu. */
typedef enum { LQ_TWIST_GAMMA5 = 0, LQ_TWIST_SCALAR = 1 } lq_twist;
typedef enum { LQ_CGNR = 0, LQ_MIXED_CGNR = 1, LQ_MULTISHIFT_CG = 2, LQ_BICGSTAB = 3, LQ_GCR = 4 } lq_solver;
typedef enum { LQ_OP_FULL = 0, LQ_OP_SCHUR = 1 } lq_op_form;
typedef enum { LQ_WILSON_FIELD = 0, LQ_STAGGERED_FIELD = 1 } lq_field_kind;
typedef enum { LQ_EVEN = 0, LQ_ODD = 1 } lq_parity;

/* Operator parameters. For Wilson actions m and mu are the real and twisted
 * mass (M = (4+m) + i mu g5 + C - H, or M = (4+m) + i mu + C - H with
 * twist_mode = LQ_TWIST_SCALAR); c_sw is used only for
 * LQ_WILSON_TM_CLOVER and must match the c_sw of lq_load_clover. For LQ_HISQ,
 * m is the staggered mass and c_naik the coefficient of the three-hop term
 * (tree level: -1/24). */
typedef struct {
    int action;      /* lq_action */
    double m;
    double mu;
    double c_sw;
    double c_naik;
    int recon;       /* lq_recon of the thin / long links in lq_dslash_apply, lq_dslash_apply_noalloc
                        and lq_operator_apply at LQ_F32 / LQ_F16 (0 = LQ_R12; LQ_F64 and LQ_F32X2
                        always use LQ_R18). The solvers take recon_sloppy instead. */
    int twist_mode;  /* lq_twist (Wilson actions); the Wilson multi-shift solve needs LQ_TWIST_GAMMA5 */
} lq_op_params;

/* Solver parameters.
 *   LQ_CGNR:          CG on the normal equations of the even-odd Schur operator
 *                     (plain CG on the hermitian Schur operator for HISQ),
 *                     everything in prec_sloppy (LQ_F64 gives the FP64 solver).
 *   LQ_MIXED_CGNR:    same, with the Krylov vectors and operator in prec_sloppy
 *                     and reliable updates in FP64 whenever the iterated residual
 *                     falls below delta times its maximum since the last update.
 *   LQ_BICGSTAB:      Wilson actions; BiCGStab (van der Vorst) directly on the
 *                     even-odd Schur operator (no normal equations; the CPU
 *                     solver of the paper's Table 2), in prec_sloppy with the same
 *                     FP64 reliable updates as LQ_MIXED_CGNR (delta; none for
 *                     prec_sloppy = LQ_F64). A vanishing BiCGStab denominator ends
 *                     that right-hand side with LQ_EBREAKDOWN.
 *   LQ_GCR:           Wilson actions; restarted GCR (generalised conjugate
 *                     residual: each new direction is the current residual, its
 *                     image under the operator made orthogonal to the earlier
 *                     ones) directly on the even-odd Schur operator, in
 *                     prec_sloppy, keeping `restart` directions (0 = 12, at most
 *                     16); at every restart, and whenever the residual fell below
 *                     delta times its value at the last restart, the solution is
 *                     accumulated and the residual recomputed in FP64 accuracy.
 *   LQ_MULTISHIFT_CG: HISQ only; one Krylov space for all nshift masses
 *                     masses[0..nshift-1] (ascending) in prec_sloppy, then each
 *                     mass refined by the mixed-precision CG; x gets nrhs*nshift
 *                     solutions, x[rhs*nshift + shift].
 * tol is the target of the FP64 true residual |b - D x|/|b| of the full system. */
typedef struct {
    int solver;       /* lq_solver */
    double tol;
    double delta;     /* reliable-update threshold (0.1) */
    int maxiter;
    int prec_sloppy;  /* lq_prec */
    int recon_sloppy; /* lq_recon for thin/long links in the sloppy operator (0 = LQ_R18) */
    int nshift;
    const double* masses;
    int graph_iters;  /* Krylov iterations captured per CUDA graph and replayed with one
                         launch: 0 = the library's choice (1), < 0 = no graphs */
    int restart;      /* LQ_GCR: directions kept before a restart (0 = 12, at most 16) */
    int persistent;   /* LQ_MIXED_CGNR, Wilson clover, prec_sloppy LQ_F16, recon_sloppy LQ_R12, one
                         right-hand side: > 0 runs that many CG iterations per launch of one persistent
                         cooperative kernel (grid-wide barriers between the operator, vector and
                         reduction phases) instead of separate kernels and graphs; 0 = off. Other
                         configurations ignore it. */
    double update_f32_below; /* LQ_MIXED_CGNR with sloppy FP32 or FP16: once the true residual of the
                         last reliable update is below this fraction of |bhat| (for every right-hand
                         side), a reliable update forms the new residual in correction form,
                         s = s_prev - Mhat (x - x_prev), with the FP32 operator (x - x_prev, the sloppy
                         solution, is exact in FP32; the error of the product, ~1e-7 of |s_prev|, stays
                         below the target once |s_prev| is small); the solution still accumulates in
                         FP64 accuracy and the final residual is recomputed from b in FP64 accuracy.
                         0 = off: every update recomputes b - Mhat x in FP64 accuracy (Sec. 1,
                         mixed-precision solvers). */
} lq_solve_params;

typedef struct {
    int status;               /* lq_status of this right-hand side */
    int iters;                /* Krylov iterations */
    int reliable_updates;
    int operator_applications;
    double true_rel_residual; /* FP64 |b - D x|/|b| on the full lattice (max over shifts) */
    double seconds;           /* device time of the solve (CUDA events on its stream) */
} lq_solve_info;

/* ------------------------------------------------------------------ errors */

/* Message of the last failure on the calling thread ("" if none). The pointer
 * stays valid until the next failing call on the same thread.
 * Paper: no counterpart (error reporting of this library). */
const char* lq_last_error(void);

/* --------------------------------------------------------------- lattices */

/* Creates a lattice of extents dims[4] = {Lx, Ly, Lz, Lt} (each even, >= 2) with
 * time boundary sign t_boundary (+1 periodic, -1 antiperiodic), on the current
 * CUDA device. *out receives the handle. LQ_EINVAL for odd or too small extents.
 * Paper: Sec. 2.1-2.2 (the four-dimensional lattice on which the operators of
 * Eq. 2-4 act, with the site and parity conventions stated above) and Table 1
 * (the ensembles' volumes L^3 x T, whose shapes the synthetic fields take). */
int lq_create_lattice(const int dims[4], int t_boundary, lq_lattice* out);

/* Frees every device buffer of the lattice. Accepts NULL.
 * Paper: no counterpart (resource management of this library). */
int lq_destroy_lattice(lq_lattice lat);

/* Device bytes the lattice currently holds (links, clover, caches, and the
 * solver work buffers it keeps between solves).
 * Paper: no counterpart (memory accounting of this library). */
int lq_lattice_bytes(lq_lattice lat, size_t* bytes);

/* Frees the solver work buffers the lattice keeps between solves (device
 * fields, staging buffers, pinned host scalars) that no running solve uses.
 * *freed (may be NULL) receives the device bytes released. A later solve
 * allocates them again. Not part of the paper's method: a memory-management
 * call of this library.
 * Paper: no counterpart. */
int lq_lattice_release_workspace(lq_lattice lat, size_t* freed);

/* Loads links in the canonical gauge layout (host or device, FP64). kind
 * selects the thin links of the Wilson actions, or the fat / long links of
 * HISQ (Sec. 2.2). The library packs them into its even-odd layout in every
 * precision it needs; the caller may free its buffer after the call.
 * Paper: Sec. 2.1 Eq. 2 (the links U_mu of the Wilson hopping term) and Sec. 2.2
 * Eq. 4 with the HISQ action's fat one-hop and long three-hop links. */
int lq_load_gauge(lq_lattice lat, int kind, int loc, const double* links);

/* Clover term of Sec. 2.1 Eq. 3. clover == NULL builds it on the device from
 * the thin links already loaded, with coefficient c_sw; otherwise clover is a
 * canonical 12x12-per-site array (host or device) that must be hermitian and
 * commute with g5 (its two 6x6 chiral blocks are used).
 * Paper: Sec. 2.1 Eq. 3 (the clover term), and Sec. 2.1's remark that the
 * twisted-mass clover inverse has a complex diagonal, so the whole clover term
 * and its inverse are computed on the GPU itself (built here on the device,
 * the inverse per (m, mu) on first use). */
int lq_load_clover(lq_lattice lat, int loc, const double* clover, double c_sw);

/* ----------------------------------------------------- operator application */

/* Hopping term H restricted to output parity `parity` (0/1): out(x) = (H in)(x)
 * for x of that parity and 0 elsewhere; dagger = 1 applies H^+. For LQ_HISQ it
 * is the staggered H of Eq. 4. in/out are canonical spinors (colour vectors for
 * HISQ) in FP64, at loc; the operator runs in precision prec (inputs are
 * rounded to it). stream is a cudaStream_t or NULL for the default stream;
 * the call returns after the result is in out.
 * Paper: Sec. 2.1 Eq. 2 (the Wilson hopping term: the sum over mu and the
 * projectors (1 +- g_mu)) and Sec. 2.2 Eq. 4 (the staggered hopping term with
 * the phases of the spin diagonalisation); the hopping kernel is the "dslash
 * kernel" on which Sec. 2.3 builds the overlap operator. */
int lq_dslash_apply(lq_lattice lat, const lq_op_params* op, int parity, int dagger, int prec, int loc,
                    const double* in, double* out, void* stream);

/* lq_dslash_apply for callers that cannot allocate device memory (an
 * application whose memory pool owns the GPU, a fixed memory budget, a loop
 * that must not trigger the implicit synchronisation of cudaMalloc/cudaFree).
 * The paper has no counterpart; this is a service of the library. Same result
 * as lq_dslash_apply with loc = LQ_DEVICE (in/out are canonical FP64 device
 * arrays), but the two internal packed fields live in a fixed scratch array of
 * 32 MiB compiled into the library (held on every GPU that loads it until the
 * process exits) and nothing is allocated. Limits and rules:
 *   - LQ_EINVAL if the two packed fields need more than 32 MiB (FP64 Wilson:
 *     up to 174762 sites, e.g. 16^3x32; FP32 twice that);
 *   - LQ_EINVAL if the lattice's links are not yet packed in this precision:
 *     one earlier lq_dslash_apply with the same action and precision does it;
 *   - the first call on a device looks up the scratch array's device address,
 *     so make it before any stream capture;
 *   - all calls share the scratch array: calls that can overlap on the GPU
 *     (other streams or threads) race, so the caller must order them.
 * The call synchronises `stream` and returns after the result is in out. */
int lq_dslash_apply_noalloc(lq_lattice lat, const lq_op_params* op, int parity, int dagger, int prec,
                            const double* in, double* out, void* stream);

/* Whole operator. form = LQ_OP_FULL: out = D in (D = M for Wilson, m + H for
 * HISQ) on the full lattice. form = LQ_OP_SCHUR: the even-odd Schur operator
 * on even sites, Mhat = A_ee - H_eo A_oo^{-1} H_oe for Wilson (A = 4+m+i mu g5+C)
 * and m^2 - H_eo H_oe for HISQ; only the even sites of in are read and only
 * the even sites of out are written (odd sites of out are set to 0).
 * Paper: Sec. 2.1 Eq. 1-3 (D_w(m_cri + omega) with the clover term, in the
 * twisted reading of omega) and Sec. 2.2 Eq. 4 (D = m + H); the even-odd Schur
 * form is the preconditioning of the GPU inverters whose timings Tables 2-3
 * report. */
int lq_operator_apply(lq_lattice lat, const lq_op_params* op, int form, int dagger, int prec, int loc,
                      const double* in, double* out, void* stream);

/* ------------------------------------------------------------------ solves */

/* Solves D x_k = b_k for k < nrhs (Wilson: M; HISQ: m + H, and for
 * LQ_MULTISHIFT_CG every mass of params->masses). rhs[k] and x[k] are canonical
 * FP64 arrays at loc (x must hold nrhs*nshift arrays for multi-shift). info
 * (may be NULL) receives one entry per right-hand side. Right-hand sides are
 * solved together with the multi-right-hand-side operator.
 * Returns LQ_OK if every system reached tol, LQ_ENOTCONV if any did not.
 * Paper: the inverters whose propagator timings Tables 2-3 report.
 *   LQ_CGNR, LQ_MIXED_CGNR: the QUDA CG the paper calls (Sec. 2.2, Table 3's
 *     GPU CG), in mixed precision with reliable updates after the
 *     mixed-precision solvers of Clark et al. cited in Sec. 1;
 *   LQ_BICGSTAB: Table 2's CPU solver (BiCGStab, Sec. 2.1);
 *   LQ_GCR: Table 2's GPU solver (GCR, Sec. 2.1);
 *   LQ_MULTISHIFT_CG: the multi-mass algorithm (Jegerlehner) of Sec. 2.3,
 *     here for HISQ's several masses and, without clover, twisted masses. */
int lq_solve(lq_lattice lat, const lq_op_params* op, const lq_solve_params* params, int nrhs,
             const double* const* rhs, double* const* x, int loc, lq_solve_info* info, void* stream);

/* ----------------------------------------------------------- device fields */

/* A spinor or colour field resident on the device in the library's internal
 * even-odd layout and precision, for callers that keep data on the GPU across
 * calls (and for timing the kernels alone): nrhs fields of one parity.
 * Paper: no counterpart (residency of the spinor fields on the GPU between
 * calls, the data movement that the GPU inverters of Sec. 1 avoid). */
int lq_field_create(lq_lattice lat, int kind, int prec, int nrhs, lq_field* out);
/* Paper: no counterpart. */
int lq_field_destroy(lq_field f);
/* copy canonical FP64 data (host or device; only sites of `parity` are read)
 * into right-hand side k of the field, and back (sites of the other parity in
 * `canonical` are left untouched)
 * Paper: no counterpart (layout conversion of this library). */
int lq_field_import(lq_field f, int k, int parity, int loc, const double* canonical, void* stream);
/* Paper: no counterpart (layout conversion of this library). */
int lq_field_export(lq_field f, int k, int parity, int loc, double* canonical, void* stream);

/* out = H_{parity, 1-parity} in on resident fields, all right-hand sides of the
 * field at once (multi-right-hand-side kernel). Asynchronous on stream.
 * Paper: Sec. 2.1 Eq. 2 / Sec. 2.2 Eq. 4 (hopping term), applied to the columns
 * of a propagator together (Table 2's 12-column, Table 3's 3-column ones). */
int lq_dslash_field(lq_lattice lat, const lq_op_params* op, int parity, int dagger, lq_field in,
                    lq_field out, void* stream);
/* out = Mhat in (Schur operator, even parity) on resident fields; tmp is a
 * scratch field of the same shape used for the odd sites. Asynchronous on stream.
 * Paper: Sec. 2.1 Eq. 1-3 in even-odd form, as in lq_operator_apply. */
int lq_schur_field(lq_lattice lat, const lq_op_params* op, int dagger, lq_field in, lq_field out,
                   lq_field tmp, void* stream);

/* ----------------------------------------------------------- instrumentation */

/* When enabled, every kernel launch of the library is bracketed with CUDA
 * events on its own stream; lq_profile_query returns, for kernels whose name
 * contains `name`, the number of launches and their summed device time since
 * the last reset (this synchronises the recorded events). */
/* Paper: no counterpart (instrumentation of this library). */
int lq_profile_enable(int on);
/* Paper: no counterpart. */
int lq_profile_reset(void);
/* Paper: no counterpart. */
int lq_profile_query(const char* name, int64_t* launches, double* total_ms);
/* number of kernel launches the library issued since the last reset
 * Paper: no counterpart. */
int64_t lq_launch_count(void);

/* Autotuner controls (the tuner times each candidate launch configuration of a
 * kernel on its first call for a given shape and keeps the fastest).
 * lq_tune_reset forgets every tuned choice. lq_tune_force(code) restricts later
 * tuning to the candidate with that code where a kernel offers it (code = block
 * size; 1000 + block size for the FP32/FP16 Wilson kernel built with its
 * registers capped at 85 per thread; 2000 + block size for its single-RHS build
 * with two hops of gathers in flight); 0 lifts the restriction. For tests and diagnostics;
 * not part of the paper's method.
 * Paper: Sec. 2.3's remark on the speed of the Wilson kernel, credited to
 * QUDA's auto-tuning (the tuner itself); the controls have no counterpart. */
int lq_tune_reset(void);
/* Paper: Sec. 2.3 (QUDA's auto-tuning), as lq_tune_reset; the restriction itself
 * has no counterpart. */
int lq_tune_force(int code);

/* Test of the bounded grid-wide barrier that the persistent CG kernel uses: one
 * cooperative launch of `blocks` blocks (<= 64) meets `rounds` times at a barrier
 * that waits for `expect` blocks (blocks <= expect <= 64). With expect == blocks
 * every barrier completes (LQ_OK, *failed = 0); with expect > blocks the first wait
 * runs out after about half a second, the kernel returns and the call gives
 * LQ_ETIMEOUT with *failed = 1. No GPU state is left behind either way.
 * Paper: no counterpart (a diagnostic of this library). */
int lq_barrier_selftest(int blocks, int expect, int rounds, int* failed);

/* ----------------------------------------------------------------- overlap */

/* Building blocks of the overlap operator (Sec. 2.3):
 *   D_ov = (1/rho) (1 + g5 eps(H_w)),  H_w = g5 D_w(-rho),  rho ~ 1.5,
 * eps the sign function. Fields are full-lattice Wilson spinors in the canonical
 * layout (host or device per loc); prec is LQ_F64, LQ_F32X2 or LQ_F32. The
 * lattice needs its thin links; clover and twisted mass are not used. */
typedef struct {
    int order;             /* Chebyshev terms used */
    double max_deviation;  /* max |1 - x P(x^2)| over lambda_min/lambda_max <= x <= 1 */
} lq_sign_info;

/* out = g5 D_w(-rho) in, with g5 fused into the operator kernel's epilogue.
 * Paper: Sec. 2.3 (the kernel that combines g5 and D_w to save bandwidth, and the
 * 50 D_w applications timed there). */
int lq_gamma5_dw_apply(lq_lattice lat, double rho, int prec, int loc, const double* in, double* out,
                       void* stream);

/* Coefficients of the sign approximation eps(x) ~ x P(x^2) for eps = lambda_min /
 * lambda_max in (0, 1): P(y) = sum_k c_k T_k((2y - eps^2 - 1)/(1 - eps^2)) (c_0 with
 * its factor 1/2 applied) interpolates 1/sqrt(y) at the Chebyshev nodes of
 * [eps^2, 1]; the order is the smallest whose |1 - x P(x^2)| stays <= delta on
 * [eps, 1] (dense sampling). The paper refines its fit at the error's extrema
 * instead (a Remez-like exchange); node interpolation is within a small factor of
 * that minimax error. coeffs (may be NULL) receives *order values, at most
 * max_order; LQ_EINVAL if more are needed. Host only.
 * Paper: Sec. 2.3 (the Chebyshev approximation of the sign function and its
 * error, Fig. 2). */
int lq_chebyshev_sign(double eps, double delta, int max_order, double* coeffs, int* order, double* max_deviation);

/* out ~ eps(H_w) in on the part of the spectrum with lambda_min <= |lambda| <=
 * lambda_max: (H_w/lambda_max) P((H_w/lambda_max)^2) in, P from lq_chebyshev_sign,
 * evaluated by the Clenshaw recurrence (two H_w applications per term). lambda_max
 * must bound the spectrum (|4 - rho| + 8 always does: eight hops of norm one);
 * outside [-lambda_max, lambda_max] the polynomial grows without bound. The paper
 * projects out the lowest modes first (lq_overlap_sign_apply_deflated); here the
 * caller chooses lambda_min below the spectrum it passes. info (may be NULL) gets
 * the order and the deviation bound.
 * Paper: Sec. 2.3 (eps(H_w) by the Chebyshev polynomial in the overlap operator). */
int lq_overlap_sign_apply(lq_lattice lat, double rho, double lambda_min, double lambda_max, double delta, int prec,
                          int loc, const double* in, double* out, lq_sign_info* info, void* stream);

/* Low modes of H_w (Sec. 2.3, the eigensolver of the overlap operator): the nev
 * eigenpairs with the smallest |lambda|. A Chebyshev polynomial T_d of
 * w(H_w^2) = (2 H_w^2 - a - b)/(b - a), [a, b] = [lambda_cut^2, lambda_max^2], keeps
 * the eigenvectors and makes the modes below lambda_cut the largest eigenvalues;
 * a thick-restart Arnoldi iteration (full re-orthogonalisation) finds them, and a
 * Rayleigh-Ritz step with H_w itself gives the eigenvalues (with their sign) and
 * checks |H_w z - lambda z| <= tol. Arithmetic in double-float (FP64 accuracy). */
typedef struct {
    int nev;            /* eigenpairs wanted, 1..48 */
    int nkv;            /* Krylov basis size, nev + 2 .. 64 (0 = min(2 nev + 8, 64)) */
    int degree;         /* degree of the Chebyshev filter, rounded up to even (0 = 24) */
    double lambda_cut;  /* filter edge: above the nev-th |lambda|, below lambda_max */
    double lambda_max;  /* bound on |H_w| (|4 - rho| + 8 always is one) */
    double tol;         /* absolute residual bound on |H_w z - lambda z| (|z| = 1) */
    int max_restarts;   /* 0 = 100 */
} lq_eig_params;

typedef struct {
    int converged;               /* 1 if every residual met tol */
    int restarts;
    int operator_applications;   /* H_w applications */
    double max_residual;
    double seconds;
} lq_eig_info;

/* evals (host, nev) in ascending |lambda|; evecs (may be NULL): nev canonical FP64
 * full-lattice Wilson spinors (host or device per loc), unit norm, each fixed up to
 * a phase. LQ_ENOTCONV if max_restarts passed first (the best pairs are returned). */
/* Paper: Sec. 2.3 and Table 4 (low eigenvectors of g5 D_w by a Chebyshev-accelerated
 * restarted Arnoldi method). */
int lq_hw_eigensolve(lq_lattice lat, double rho, const lq_eig_params* p, int loc, double* evals, double* const* evecs,
                     lq_eig_info* info, void* stream);

/* lq_overlap_sign_apply deflated by nev eigenpairs of H_w (evals and unit evecs as
 * lq_hw_eigensolve returns them, in the canonical layout per loc): their part of
 * in gets its exact sign, the polynomial acts on the rest, so lambda_min only has
 * to lie below the remaining spectrum. Computed in double-float.
 * Paper: Sec. 2.3 (the low modes projected out before the polynomial; the
 * deflation used for the overlap propagators). */
int lq_overlap_sign_apply_deflated(lq_lattice lat, double rho, double lambda_min, double lambda_max, double delta,
                                   int nev, const double* evals, const double* const* evecs, int loc,
                                   const double* in, double* out, lq_sign_info* info, void* stream);

/* ----------------------------------------------------------------- serving */

/* A request server for continuous batching of solves: requests are queued,
 * admitted while their estimated device memory fits in hbm_budget_bytes (next
 * to the lattices they use), at most max_slots at once. Admission takes the
 * first queued request, in arrival order, that fits: one that does not fit yet
 * is overtaken by later ones that do, at most 2 * max_slots times, after which
 * nothing behind it is admitted before it (no starvation). Each admitted request
 * runs on its own worker thread and CUDA stream, so solves that arrive while
 * others are on the GPU start as soon as a slot and memory free up and then
 * overlap with them on the device. Lattices (gauge and clover fields) are
 * created and loaded by the caller and stay resident across requests. */
typedef struct {
    lq_lattice lat;           /* resident lattice; must outlive the request */
    lq_op_params op;
    lq_solve_params solve;    /* solve.masses is copied at submission */
    int nrhs;
} lq_request;

typedef struct {
    double submitted;  /* seconds since server creation */
    double admitted;
    double finished;
} lq_request_times;

/* Paper: Sec. 1 and Sec. 3 (one interface through which an application calls
 * the GPU inverters of several actions, here for a stream of propagator
 * requests); the serving loop itself (admission by memory, continuous batching)
 * is this library's addition and has no counterpart in the paper. */
int lq_server_create(size_t hbm_budget_bytes, int max_slots, lq_server* out);
/* stops the workers after the admitted requests finish; queued ones are dropped
 * Paper: no counterpart. */
int lq_server_destroy(lq_server s);
/* rhs: nrhs canonical FP64 host arrays, copied before the call returns.
 * LQ_ENOMEM if the request alone can never fit in the budget.
 * Paper: Sec. 1 and Sec. 3 (the inverter call of the uniform interface, queued). */
int lq_submit(lq_server s, const lq_request* req, const double* const* rhs, uint64_t* ticket);
/* LQ_EAGAIN until done; then copies nrhs*max(1,nshift) solutions into x (host
 * arrays), per-rhs info and the timestamps (either may be NULL), forgets the
 * ticket and returns the solve's status
 * Paper: Sec. 1 and Sec. 3 (the result of that inverter call). */
int lq_poll(lq_server s, uint64_t ticket, double* const* x, lq_solve_info* info, lq_request_times* times);
/* blocks up to timeout_ms for the ticket to finish; LQ_ETIMEOUT otherwise
 * Paper: no counterpart. */
int lq_wait(lq_server s, uint64_t ticket, int timeout_ms);
/* device bytes the server reserves for this request while it runs (its solver
 * work fields and staging, not counting the resident lattice)
 * Paper: no counterpart. */
int lq_request_bytes(const lq_request* req, size_t* bytes);
/* requests queued, running, and device bytes currently reserved by running requests
 * Paper: no counterpart. */
int lq_server_stats(lq_server s, int* queued, int* running, size_t* reserved_bytes);

#ifdef __cplusplus
}
#endif
#endif /* LQ_H */
