/*
 * tpcg.h -- C ABI of the GB300 (sm_103a) Truncated Preconditioned Conjugate Gradient library for
 * isogeometric Poisson problems in Tucker format (Montardini, Sangalli, Tani, "A low-rank
 * isogeometric solver based on Tucker tensors").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: TPCG_OK (0) or one of the TPCG_E_* codes below.  Invalid arguments are reported
 *    before anything is enqueued.  TPCG_E_CUDA means a CUDA call failed; tpcg_last_error() gives text.
 *  - All compute entry points are stream-ordered and asynchronous on the given cudaStream_t
 *    (passed as void*; NULL = the legacy default stream).  Scalars produced on the device are written
 *    to device pointers; read them after synchronising the stream.
 *  - Layout: every direction has the same number n of degrees of freedom.  A factor matrix is n x cols,
 *    column-major with leading dimension n.  A dense core r1 x r2 x r3 is column-major (mode 1 fastest),
 *    matching vec() of Sec. 2.3.  Floating-point data is double (TPCG_F64) or float (TPCG_F32), chosen per
 *    context; CG scalars are always double.
 *  - Ownership: tucker_t buffers are allocated and owned by the caller (e.g. PyTorch); the library owns
 *    tpcg_ctx (workspace) and tpcg_problem (operator, right-hand side, preconditioner tables) and frees
 *    them in the matching destroy call.
 *  - Ranks live on the device (tucker_t.desc), so consecutive calls need no host synchronisation and the
 *    whole sequence can be captured in a CUDA graph.
 */
#ifndef TPCG_H
#define TPCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------------------ status codes */
#define TPCG_OK 0
#define TPCG_E_INVALID 1        /* bad argument (sizes, ranks, capacities, dtype mismatch)          */
#define TPCG_E_NOMEM 2          /* device allocation failed                                          */
#define TPCG_E_NOT_CONVERGED 3  /* TPCG reached max_it before ||r|| <= tol ||f||                     */
#define TPCG_E_RANK_CAP 4       /* a rank cap forced a truncation error above the requested tolerance */
#define TPCG_E_TIMEOUT 5        /* a device-side wait gave up (persistent scheduler)                 */
#define TPCG_E_CUDA 6           /* a CUDA runtime call failed                                        */
#define TPCG_E_BREAKDOWN 7      /* NaN/Inf or a non-positive curvature p.q in the CG scalars          */

#define TPCG_F64 0
#define TPCG_F32 1
#define TPCG_MIXED 2          /* problems/contexts: FP64 tensors and outer loop, FP32 inner TPCG (see tpcg_solve) */

#define TPCG_MAX_BLOCKS 128     /* core blocks of an unrounded Tucker tensor                          */
#define TPCG_DESC_BYTES 8192    /* bytes of device memory a tucker_t.desc must provide                */

/* ------------------------------------------------------------------------------------ Tucker tensors */
/* A Tucker vector x = (U3 (x) U2 (x) U1) vec(core) (eq. Tucker, Sec. 2.3).
 * Rounded ("plain") tensors have one dense core.  Unrounded results of tucker_apply, tucker_residual,
 * tucker_axpby and fd_precond_apply have a block-diagonal core (Sec. 2.3 sum and eq. tt_product) kept as
 * a list of scaled dense blocks that POINT AT the cores of their inputs: those input cores must stay
 * unchanged until the unrounded tensor has been rounded (tucker_round) or is no longer needed. */
typedef struct {
    int dtype;          /* TPCG_F64 or TPCG_F32                                                       */
    int n;              /* dofs per direction                                                        */
    int cap;            /* column capacity of each factor buffer                                     */
    long long core_cap; /* element capacity of the core buffer                                        */
    void* U[3];         /* device, n x cap each, column-major, ld = n                                */
    void* core;         /* device, core_cap elements                                                 */
    void* desc;         /* device, TPCG_DESC_BYTES bytes: ranks and block list (library-managed)     */
} tucker_t;

typedef struct tpcg_ctx_s* tpcg_ctx;          /* workspace for one solve stream                     */
typedef struct tpcg_problem_s* tpcg_problem;  /* operator A~, rhs f~, preconditioner P~ on the device */

/* ------------------------------------------------------------------------------------ problem setup */
#define TPCG_GEOM_CUBE 0    /* identity map, f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z); with Neumann faces
                               f = 3 w^2 s(x) s(y) s(z), s(t) = sin(w t + k0 pi/2), w = (1 - k0/2 - k1/2) pi */
#define TPCG_GEOM_TWIST 1   /* quarter annulus rho in [1,2], theta in [0,pi/2], extruded along z, with the
                               cross-section rotated about its centroid by amp sin(pi z); f = 1       */

typedef struct {
    int kind;           /* TPCG_GEOM_*                                                               */
    double amp;         /* twist amplitude (radians), TPCG_GEOM_TWIST only                            */
    double eps_geo;     /* relative tolerance of the low-rank coefficient approximation (App. A); 0 = 1e-8 */
    double eps_prec;    /* relative tolerance of the preconditioner, eq. prec_bound; 0 = 0.1         */
    int k0, k1;         /* boundary conditions on the faces eta_t = 0 (k0) and eta_t = 1 (k1) of every
                           direction t: 0 homogeneous Dirichlet, 1 homogeneous Neumann (App. B's flags).
                           (0,0), (0,1) or (1,0); (1,1) would leave the constant in the kernel           */
} tpcg_geometry;

/* Host FP64 setup (App. A, App. B, Prop. 1) followed by upload: B-spline matrices, low-rank Chebyshev
 * approximation of Q(eta) and omega(eta) folded into a Kronecker sum A~ = sum_j w_j K3^j (x) K2^j (x) K1^j,
 * the Tucker rhs f~ (rounded losslessly), and the low-rank FD tables with the exponential sums chosen by
 * TPCG_OPT_EXPSUM_BEST (by default the best sums, R_P of eq. estimate_prec_rel as in Table 1).  n dofs per
 * direction, degree p, n_el = n - p + 2 - k0 - k1 > p: a Neumann end keeps its end function (the natural
 * condition), and the preconditioner takes App. B's Neumann variant.  dtype selects the precision of the device copies.  *out is
 * owned by the caller and released with tpcg_problem_destroy. */
int tpcg_setup(const tpcg_geometry* geo, int degree, int n, int dtype, tpcg_problem* out);

/* Problem from explicit host arrays (all double, column-major):
 *   R terms: weights w[R]; bands[((j*3 + t)*(2p+1) + d)*n + i] = K_t^j[i, i + d - p] (zero outside);
 *   rhs: core f_core (rf1 x rf2 x rf3), factors f_U[t] (n x rf_t);
 *   preconditioner (Alg. 4 with the eigenvector factorisation of App. B):
 *     lam[n]      : Lambda~ (first n1 entries omega_j^2, omega_j = (j - k0/2 - k1/2) pi, then Lambda2),
 *     mu[n1]      : sine-basis scaling, U~[:, :n1] = W U_dft diag(1/mu),
 *     W (n x n1)  : sparse, given in CSR: w_rowptr[n+1], w_col[nnz], w_val[nnz],
 *     v2u2 (n x n2): V2 U2 dense,
 *     RP exponential-sum pairs omega[RP], alpha[RP], lambda_min,
 *     k0, k1      : Neumann flags of the two ends (the same in every direction; (1,1) is refused).
 *   The sine transform is U_dft[l,j] = sqrt2 sin(omega_j x_l + k0 pi/2), l, j = 1..n1, on the interpolation
 *   points x_l of App. B: the breakpoints i/n_el without the Dirichlet ends for odd p (n_el = n1 + 1 - k0 -
 *   k1), the span midpoints (l - 1/2)/n1 for even p.  With k0 = k1 = 0 it is DST-I (odd p) or DST-II (even p). */
typedef struct {
    int n, p, R, dtype;
    const double* w;
    const double* bands;
    int rf[3];
    const double* f_core;
    const double* f_U[3];
    int n1, n2, RP, w_nnz;
    const double* lam;
    const double* mu;
    const int* w_rowptr;
    const int* w_col;
    const double* w_val;
    const double* v2u2;
    const double* omega;
    const double* alpha;
    double lambda_min;
    int k0, k1;
} tpcg_problem_arrays;

/* Returns TPCG_E_INVALID, before any device work, for inconsistent sizes or a NaN/Inf in any table. */
int tpcg_problem_create(const tpcg_problem_arrays* a, tpcg_problem* out);

typedef struct {
    int n, p, R, RP, n1, n2, rf[3], dtype;
    double lambda_min, lambda_max, MP, norm_f;
    int w_nnz;          /* non-zeros of W */
    int k0, k1;         /* Neumann flags of the ends */
} tpcg_problem_info;

int tpcg_problem_get_info(tpcg_problem pb, tpcg_problem_info* out);

/* Host copies of the setup data, laid out as in tpcg_problem_arrays (buffers provided by the caller,
 * sized from tpcg_problem_get_info; any pointer may be NULL to skip it).  f_U[t] gets n x rf[t]. */
int tpcg_problem_export(tpcg_problem pb, double* w, double* bands, double* f_core, double* f_U0, double* f_U1,
                        double* f_U2, double* lam, double* mu, double* v2u2, double* omega, double* alpha);
/* Host-only form of tpcg_setup: the same FP64 setup (App. A, App. B, Prop. 1), its tables copied into caller-owned
 * host buffers laid out as in tpcg_problem_arrays and tpcg_problem_export, without any GPU call.  info receives
 * the sizes (dtype and norm_f are 0); any buffer may be NULL (skipped), so a first call with NULL buffers returns
 * the sizes.  f_Ut: n x rf[t]; w_rowptr n + 1; w_col, w_val w_nnz.  Errors as tpcg_setup. */
int tpcg_setup_host(const tpcg_geometry* geo, int degree, int n, tpcg_problem_info* info, double* w, double* bands,
                    double* f_core, double* f_U0, double* f_U1, double* f_U2, double* lam, double* mu, double* v2u2,
                    double* omega, double* alpha, int* w_rowptr, int* w_col, double* w_val);
/* W of the sine factorisation in CSR (rowptr n+1, col/val w_nnz); NULL pointers are skipped. */
int tpcg_problem_export_w(tpcg_problem pb, int* rowptr, int* col, double* val);
void tpcg_problem_destroy(tpcg_problem pb);

/* ------------------------------------------------------------------------------------ workspace */
/* Workspace for rounding, dots and TPCG on tensors with n dofs per direction, at most max_cols factor
 * columns before rounding and rank at most rank_cap after rounding. */
int tpcg_ctx_create(int n, int max_cols, int rank_cap, int dtype, tpcg_ctx* out);
/* Device bytes such a context holds once it has run a solve (workspace and the solver's tensors). */
size_t tpcg_ctx_bytes(int n, int max_cols, int rank_cap, int dtype);
void tpcg_ctx_destroy(tpcg_ctx c);

/* ------------------------------------------------------------------------------------ Tucker ops */
/* Mark t as a plain tensor of multilinear rank (r1, r2, r3) whose core and factors the caller filled. */
int tucker_set_plain(tucker_t* t, int r1, int r2, int r3, void* stream);
/* Ranks and number of core blocks (synchronises the stream). */
int tucker_get_ranks(const tucker_t* t, int* r3_out, int* nblk_out, void* stream);

/* y = A~ x (eq. tt_product): factors [K_t^1 X_t, ..., K_t^R X_t], core superdiag(w) (x) G_x (blocks).
 * x must be plain; y needs cap >= R * rank(x). */
int tucker_apply(tpcg_problem pb, const tucker_t* x, tucker_t* y, void* stream);
/* y = f~ - A~ x (Alg. 5 step 11 before truncation); y needs cap >= rf + R * rank(x). */
int tucker_residual(tpcg_problem pb, const tucker_t* x, tucker_t* y, void* stream);
/* z = a x + b y (Sec. 2.3 sum): concatenated factors, block-diagonal core.  a and b are host doubles,
 * or, when a_dev / b_dev are non-NULL, device doubles read at execution time. */
int tucker_axpby(double a, const double* a_dev, const tucker_t* x, double b, const double* b_dev,
                 const tucker_t* y, tucker_t* z, void* stream);
/* *out_dev = <x, y> (Sec. 2.3 scalar product), both plain.  out_dev: device double.  Outside a stream capture
 * the call reads both descriptors (synchronising the stream) and returns TPCG_E_INVALID for a block
 * (unrounded) tensor or a rank above the context's rank_cap; inside a capture it cannot, and writes NaN for
 * such inputs instead. */
int tucker_dot(tpcg_ctx c, const tucker_t* x, const tucker_t* y, double* out_dev, void* stream);
/* <x, y> exactly as tucker_dot, without a context and without allocating device memory (the paper has no
 * counterpart: this serves callers that may not allocate, e.g. code running under another party's stream
 * capture or inside allocator callbacks).  Its scratch is one fixed device array of about 4.3 MB inside the
 * library, sized for ranks <= 64: x->cap or y->cap above 64 returns TPCG_E_INVALID (nothing launched); block tensors are refused as in
 * tucker_dot (outside a capture).
 * x, y: plain tensors of the same n and dtype (TPCG_F64 or TPCG_F32); out_dev: device double.
 * The first call on a device looks up the array's address (cudaGetSymbolAddress); make that call before
 * any stream capture that is to contain it.  All callers share the array: calls that overlap on the
 * device (other streams, other host threads) race and must be serialised by the caller. */
int tucker_dot_static(const tucker_t* x, const tucker_t* y, double* out_dev, void* stream);
/* In-place relative truncation, Alg. 1: y <- T_rel(y, eps) with ST-HOSVD split eps^2/3 per mode, ranks
 * clipped to rank_cap (<= 0: the context's cap).  Factors come out orthonormal, so ||y|| = ||core||.
 * If info_dev is non-NULL it receives 6 doubles: ||y||^2 before, the discarded squared norm, the new
 * ranks (3, as doubles) and a flag: 0 ok, 1 the new core did not fit the tensor's core_cap, 2 the input's
 * blocks need more Z-formation workspace than the context holds (sum over blocks of r1 min(n, k2) r3 above
 * max_cols n rank_cap; y is then left with rank 0); TPCG_E_RANK_CAP is not raised here (check info).
 * Grams of order above 128 are first reduced to the Rayleigh-Ritz matrix Q^T G Q of an orthonormal basis Q of
 * at most 128 pivoted-Cholesky columns of G (stopped once the Schur complement holds 1% (FP32) or 1e-8 (FP64)
 * of the mode's budget) in FP32 contexts with n > 128 and in FP64 contexts with n > 256 and rank_cap <= 112:
 * the error bound of Alg. 1 holds exactly, and the ranks are the exact rule's up to that fraction unless 128
 * columns do not reach it (such a Gram then keeps at most 128 directions). */
int tucker_round(tpcg_ctx c, tucker_t* y, double eps, const double* eps_dev, int rank_cap, double* info_dev,
                 void* stream);
/* v = P~^{-1} s, Alg. 4 steps 5-9: factors [U~ D_(t,1) U~^T S_t, ..., U~ D_(t,RP) U~^T S_t], core
 * superdiag(omega / lambda_min) (x) G_s (blocks).  s plain; v needs cap >= RP * rank(s). */
int fd_precond_apply(tpcg_problem pb, tpcg_ctx c, const tucker_t* s, tucker_t* v, void* stream);

/* ------------------------------------------------------------------------------------ solver */
typedef struct {
    double tol;         /* relative residual tolerance, ||r_k|| <= tol ||f~||             (1e-6)  */
    double eps0;        /* initial dynamic-truncation tolerance                           (0.1)   */
    double eps_min;     /* minimum dynamic tolerance; <= 0: tol ||f~|| / 10 (Sec. 5)              */
    double alpha;       /* reduction factor of Alg. 2                                      (0.5)   */
    double delta;       /* update-ratio threshold of Alg. 2                                (1e-3)  */
    double beta_trunc;  /* beta of eq. rel_tol_iterates                                    (0.1)   */
    int max_it;         /* iteration cap                                                   (500)   */
    int rank_cap;       /* rank cap of every truncation; <= 0: the context's cap                   */
    double inner_tol;   /* mixed form: relative tolerance of each FP32 inner solve          (2e-2)  */
    int max_outer;      /* mixed form: cap on FP64 residual refinements (at most 64)        (12)    */
    double refine_keep; /* mixed form: relative accuracy to which each correction is kept in x  (3e-2) */
} tpcg_params;

typedef struct {
    int iters;              /* TPCG iterations                                                      */
    int status;             /* TPCG_OK, TPCG_E_NOT_CONVERGED, TPCG_E_BREAKDOWN                      */
    double rel_res;         /* ||r_k|| / ||f~|| of the truncated residual at exit                   */
    int rank[3];            /* multilinear rank of the solution                                      */
    double mem_compression; /* eq. mem_comp, percent                                                */
    int dt_trials;          /* total Alg. 2 truncations                                             */
    int max_rank_seen;      /* largest rank of any rounded iterate                                  */
    int outer_iters;        /* mixed form: FP64 residual refinements (0 for the single-precision forms) */
    double true_rel_res;    /* mixed form: ||f - A x|| / ||f|| of the FP64 residual before the last stop test */
} tpcg_stats;

void tpcg_params_default(tpcg_params* p);

/* Per-iteration scalars of the last Alg. 5 run on context c (no counterpart in the paper; for inspection and
 * tests).  Row k (k = 0 the state after the set-up steps of Alg. 5, k >= 1 after iteration k) holds
 * TPCG_HIST_COLS doubles: ||r_k|| / ||f~||, omega_{k-1}, beta_{k-1}, xi_k = p_k . q_k, the dynamic-truncation
 * tolerance eps_new after the Alg. 2 call of iteration k, the last update ratio v of that call, the number
 * of Alg. 2 truncations in iteration k, and eta_k of eq. rel_tol_iterates.  Up to max_rows rows are copied
 * to out (host, row-major); *rows receives the number recorded.  In the mixed form the inner FP32 solves
 * run on the context's FP32 companion, so c records nothing for them. */
#define TPCG_HIST_COLS 8
int tpcg_ctx_history(tpcg_ctx c, double* out, int max_rows, int* rows);

/* Alg. 5 with x_0 = 0: x receives the low-rank solution (plain, caller buffers with cap >= rank_cap and
 * core_cap >= rank_cap^3).  Synchronises the stream once per iteration for the stopping test.
 * Mixed form (problem and context created with TPCG_MIXED; x is FP64): iterative refinement around Alg. 5.
 * Each outer step forms the residual f - A x in FP64 (banded products and the Z formation of Alg. 1 in
 * FP64, so the cancellation is exact to FP64 and ||Z|| is the true residual norm) and truncates it in FP32
 * to 0.1 inner_tol relative, or to beta tol ||f~|| / 2 absolute when that is looser (the relaxation of
 * eq. rel_tol_iterates carried over to the outer loop).  It then solves A d = r by Alg. 5 in FP32 to
 * max(inner_tol, tol ||f~|| / (2 ||r||)) (dynamic-truncation floor a tenth of that, at most 12 iterations)
 * and sets x <- T_rel(x + d, refine_keep ||d|| / ||x + d||) in FP64.  A looser refine_keep drops the FP32
 * rounding noise of the corrections (which later FP32 corrections cannot resolve) instead of accumulating it.  x is plain throughout, so the FP64 residual refers to the returned tensor.
 * The stopping test uses the true FP64 residual. */
int tpcg_solve(tpcg_problem pb, tpcg_ctx c, const tpcg_params* prm, tucker_t* x, tpcg_stats* st, void* stream);

/* count independent solves at once (no counterpart in the paper; many-solve throughput).  Solve i is
 * tpcg_solve(pbs[i], ctxs[i], &prms[i], &xs[i], &sts[i], streams[i]) on a host thread of its own, so the
 * solves' kernels overlap on the device.  Every solve needs its own context and its own stream; a NULL
 * entry runs that solve on a non-blocking stream owned by its context (created on first use).  Problems may be
 * shared: a solve only reads its problem (its capacity-error flags live in its own context).  statuses[i] receives each
 * solve's status; the return value is TPCG_OK, else the first hard error, else TPCG_E_NOT_CONVERGED.
 * Results do not depend on what runs beside them (no shared scratch).  Turn profiling off first. */
/* The non-blocking stream owned by a context (created on first use, destroyed with the context; no counterpart
 * in the paper).  Concurrent solves must not share a stream: the solver replays CUDA graphs captured on its
 * stream, and a capture in progress on a shared stream would take in another solve's work.  Callers that
 * draw streams from a recycling pool (torch keeps 32 per priority) should use this one instead. */
int tpcg_ctx_stream(tpcg_ctx c, void** out);
int tpcg_solve_batch(int count, const tpcg_problem* pbs, const tpcg_ctx* ctxs, const tpcg_params* prms, tucker_t* xs,
                     tpcg_stats* sts, void* const* streams, int* statuses);

/* ------------------------------------------------------------------------------------ elasticity */
/* Compressible linear elasticity (Sec. 5.3), b(u, v) = 2 mu (eps(u), eps(v)) + lambda (div u, div v) on the
 * mapped cube, homogeneous Dirichlet conditions on every face and a constant body force.  The system is the
 * 3 x 3 block matrix [A_ij] (eq. block-system-elasticity): block A_ij (test component i, trial component j) is
 * a Kronecker sum built from the coefficients C^{ij}_{kl} = det J [mu delta_ij (G G^T)_kl + mu G_ki G_lj +
 * lambda G_kj G_li], G = J^-1, exactly as the Poisson operator is built from Q (App. A).  A block vector is
 * an array of three tucker_t (components 1, 2, 3); products, sums, scalar products and truncations act per
 * block.  The preconditioner is block diagonal: block i is Alg. 4 for mu (K M M + M K M + M M K) +
 * (lambda + mu) (K in direction i), i.e. the FD with direction weights c_t = mu + (lambda + mu) delta_ti.
 * Forms: TPCG_F64 and TPCG_F32. */
typedef struct tpcg_elast_s* tpcg_elast;

/* Host FP64 setup of all nine blocks (force: 3 host doubles, the constant body force), then upload.
 * geo->k0 / geo->k1 = 1 make the faces eta_t = 0 / eta_t = 1 of every direction traction-free (the natural
 * condition: their end functions stay in the space of every component), 0 clamps them; (1,1) is refused. */
int tpcg_elast_setup(const tpcg_geometry* geo, int degree, int n, double lame_lambda, double lame_mu,
                     const double* force, int dtype, tpcg_elast* out);
/* The same from caller tables: blocks[3 i + j] describes A_ij (its rhs fields give f_i; the preconditioner
 * tables of the diagonal blocks are used).  All nine share n, p and dtype. */
int tpcg_elast_create(const tpcg_problem_arrays* blocks, double lame_lambda, double lame_mu, tpcg_elast* out);
/* R[9]: Kronecker terms of every block; RP: exponential-sum length; norm_f: ||[f_1; f_2; f_3]|| (host). */
int tpcg_elast_get_info(tpcg_elast e, int* R, int* RP, double* norm_f);
/* y_i = sum_j A_ij x_j (unrounded; the blocks of A_ij x_j are appended to y_i's block list).  x, y: 3 tensors;
 * y_i needs cap >= sum_j R_ij rank(x_j) and at most 128 blocks. */
int tpcg_elast_apply(tpcg_elast e, const tucker_t* x, tucker_t* y, void* stream);
/* y_i = f_i - sum_j A_ij x_j (unrounded). */
int tpcg_elast_residual(tpcg_elast e, const tucker_t* x, tucker_t* y, void* stream);
/* v_i = P~_i^-1 s_i (Alg. 4 with the direction weights of block i); s plain, v_i needs cap >= R_P rank(s_i). */
int tpcg_elast_precond(tpcg_elast e, tpcg_ctx c, const tucker_t* s, tucker_t* v, void* stream);
/* Alg. 5 on block vectors with x_0 = 0; x: 3 caller tensors (cap >= rank_cap, core_cap >= rank_cap^3).
 * Uses 21 of the context's solver tensors (context: same n and dtype, max_cols >= max_i (rf_i + sum_j R_ij
 * rank_cap) and >= R_P rank_cap).  stats: iterations, the largest rank per mode over the components,
 * memory compression as defined in Sec. 5.3, and the true relative residual of the returned x. */
int tpcg_elast_solve(tpcg_elast e, tpcg_ctx c, const tpcg_params* prm, tucker_t* x, tpcg_stats* st, void* stream);
void tpcg_elast_destroy(tpcg_elast e);

/* ------------------------------------------------------------------------------------ tuning */
/* Launch-shape options (no counterpart in the paper), process-wide:
 *   TPCG_OPT_GEMM_CTAS_PER_SM: CTA budget per SM of the grouped GEMM launches (0 = one CTA per output tile
 *   and argument group; 1..64 caps the grid and the kernel strides over the groups; default 2, measured best
 *   with 32 solves at once: 4.0 against 3.6 solves/s uncapped). */
#define TPCG_OPT_GEMM_CTAS_PER_SM 1
/*   TPCG_OPT_EXPSUM_BEST: which exponential sums (Prop. 1) tpcg_setup / tpcg_elast_setup build for the FD
 *   preconditioner: 1 (default) the best sums of tpcg_expsum_best, whose R_P reproduces Table 1; 0 the
 *   sinc-quadrature sums found by a search (R_P about twice Table 1's).  Problems set up earlier keep their
 *   sums. */
#define TPCG_OPT_EXPSUM_BEST 2
/*   TPCG_OPT_EIG: eigensolver of the FP32 mode Grams of ST-HOSVD (Alg. 1 step 3) up to 128 x 128: 1 (default) a
 *   pivoted Cholesky G = L L^T followed by one-sided Jacobi on the columns of L, whose normalised columns are the
 *   eigenvectors (the pivoted Cholesky of G = Z Z^T is the column-pivoted QR of Z^T, the preconditioner of
 *   Drmac and Veselic's one-sided Jacobi SVD); 0 the two-sided cyclic Jacobi on G with accumulated rotations. */
#define TPCG_OPT_EIG 3
/*   TPCG_OPT_DST: how the preconditioner applies the sine block U_dft of App. B (Alg. 4): 1 (default) batched FFTs,
 *   O(n1 log n1) per column, by Bluestein's chirp-z identity for any n1 <= 1024 (power-of-two FFTs of size
 *   >= 2 n1 - 1 in shared memory); 0 the dense n1 x n1 product with the stored sine matrix. */
#define TPCG_OPT_DST 4
/*   TPCG_OPT_TC: where the FP32 contractions (Alg. 1 Z formation, mode Grams, projections and factor updates, the
 *   scalar products) run: 1 on the tensor cores (tcgen05, 3xTF32 products with FP32 accumulation in tensor
 *   memory), 0 (default) on the FP32 SIMT units.  FP64 contractions always use the FP64 units. */
#define TPCG_OPT_TC 5
/*   TPCG_OPT_RR: 1 (default) contexts created afterwards (FP32 with n > 128; FP64 with n > 256 and rank_cap <=
 *   112) reduce mode Grams of order above 128 to a Rayleigh-Ritz matrix of at most 128 pivoted-Cholesky columns
 *   before the eigensolver (see tucker_round); 0 they give every Gram to the one-CTA Jacobi eigensolvers, whose
 *   FP32 variant above order 128 tracks the eigenvalues by rotation updates and can misjudge the discarded
 *   energy by more than the FP32 Gram's resolution. */
#define TPCG_OPT_RR 6
/*   TPCG_OPT_GRAM_MIN_K: the mode Grams of ST-HOSVD (Alg. 1 step 3) are split-K reductions into at most 64 partial
 *   Grams summed in a fixed order; a value k > 0 gives every partial at least k of the reduction (fewer, longer
 *   partials: less partial traffic and block start-up, which pays when many solves share the device), 0 (default)
 *   always uses the most partials.  Read when a truncation is launched or captured. */
#define TPCG_OPT_GRAM_MIN_K 7
/*   TPCG_OPT_GEMM_KIND: the FP32 SIMT contractions: 2 (default) 128 threads per 64 x 64 output tile, 8 x 4 outputs
 *   per thread (16-byte shared loads, 32 FMAs per 3 loads), operands copied by cp.async through three shared
 *   stages; 1 the same tile staged through registers and two stages; 0 256 threads, 4 x 4 outputs per thread. */
#define TPCG_OPT_GEMM_KIND 8
/*   TPCG_OPT_ROUND_RULE: the FP64 truncation rule of tucker_round (Alg. 1 step 3 on mode Grams): -1 (default)
 *   automatic, strict below eps = 1e-7 (every discarded Gram eigenvalue charged its rounding uncertainty
 *   4 eps_machine trace, so nothing the Gram cannot resolve is dropped); 0 plain (clamped eigenvalues as they
 *   are); 1 strict; 2 resolved below eps = 1e-8 (two passes: the part one Gram resolves, rounded at 1e-7, then
 *   the remainder rounded with the absolute budget eps ||y||, whose own Grams resolve it; the two merged
 *   losslessly), which meets ||y - y~|| <= eps ||y|| with ranks close to those of an SVD.  tpcg_solve chooses
 *   its own rule. */
#define TPCG_OPT_ROUND_RULE 9
/*   TPCG_OPT_RESOLVED: 1 (default) FP64 solves (the FP64 form's Alg. 2 truncations of x, the mixed form's
 *   correction update of x) take the resolved rule whenever their tolerance is below 1e-8 and the context holds
 *   3 rank_cap columns; 0 one Gram pass with the plain rule. */
#define TPCG_OPT_RESOLVED 10
int tpcg_set_option(int key, long long value);

/* Best exponential sum s_R(lambda) = sum_j omega_j exp(-alpha_j lambda) for 1/lambda on [1, M] in the maximum
 * norm (Prop. 1, eq. estimate_approx_diag), with R the smallest number of terms meeting E_R(M) <= eps_prec / M
 * (the R_P of eq. estimate_prec_rel when M = M_P).  Computed on the host (no GPU call) by the Remez exchange on
 * the alternation points of the error.  omega, alpha: caller-owned host arrays of at least rmax entries;
 * *R_out = R; *E_out (may be NULL) = E_R(M).  Returns TPCG_E_INVALID for a null output, rmax < 1, M < 1,
 * eps_prec <= 0, or when no R <= rmax meets the bound.  Takes seconds for M up to ~1e6. */
int tpcg_expsum_best(double M, double eps_prec, int rmax, double* omega, double* alpha, int* R_out, double* E_out);

/* ------------------------------------------------------------------------------------ profiling */
/* Kernel classes timed with CUDA events on the launching stream while profiling is on:
 *   0 fused last-mode GEMM of Alg. 1 step 2 (Z formation)   1 per-block mode products of step 2
 *   2 mode Grams of ST-HOSVD (split-K GEMM + reduction)       3 eigensolver + truncation rule
 *   4 ST-HOSVD projections   5 Householder QR   6 banded matvec (apply/residual)   7 FD application
 *   8 Tucker dot   9 whole tucker_round   10 reserved   11 one-CTA Jacobi sweeps (flops field: sweeps,
 *   bytes field: Grams; no time).
 * flops/bytes are the algorithmic work of the launches (accumulated on the device from the actual ranks). */
#define TPCG_PROF_KINDS 16
int tpcg_profile_enable(int on);
int tpcg_profile_reset(void);
int tpcg_profile_get(int kind, double* ms_total, long long* count, double* flops, double* bytes);
/* Number of kernels this library has launched since load (host counter, no synchronisation). */
long long tpcg_launch_count(void);

/* ------------------------------------------------------------------------------------ misc */
const char* tpcg_last_error(void);
const char* tpcg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TPCG_H */
