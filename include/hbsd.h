/*
 * hbsd.h -- C ABI of the GB300 LABPSD library: block preconditioned steepest descent with
 * the hybrid (global + locally accelerated) preconditioner of Cai, Bai, Pask and Sukumar
 * (Sec. 3 "LABPSD" outline and remarks; Sec. 4 implementation of step 6).
 *
 * Problem (Eq. ghep): lowest nev eigenpairs of H x = lambda S x, H Hermitian, S Hermitian
 * positive definite, H and S sparse with one shared pattern (Sec. 4 footnote).
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, HBSD_NOT_CONVERGED (1) when the outer iteration cap was hit
 *     (outputs then hold the best iterate), HBSD_BUSY (2) from hbsd_poll while a request
 *     runs, and a negative HBSD_ERR_* code on error.  No exception or abort crosses the ABI;
 *     hbsd_last_error() returns a thread-local message for the last failing call.
 *   - Block vectors on the device are ROW-MAJOR: entry (i, j) of an n x k block with leading
 *     dimension ld (ld >= k, in elements) sits at ptr[i * ld + j].  Every device pointer
 *     must be 16-byte aligned and every ld even, so that a row pair of doubles is one
 *     16-byte access.  ld >= k is checked (HBSD_ERR_ARG); alignment and evenness are the
 *     caller's contract.
 *   - Host arrays (hbsd_csr, X0, outputs of hbsd_solve) are plain C arrays; the caller owns
 *     them; the library copies what it keeps.  Device buffers passed to step-level entry
 *     points are owned by the caller; the library never frees them.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = legacy default
 *     stream).  Step-level calls are asynchronous on that stream unless stated otherwise.
 *   - The library holds no torch or Python types; a caller may hand in device pointers of
 *     any allocator.
 */
#ifndef HBSD_H
#define HBSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------ */
#define HBSD_OK               0
#define HBSD_NOT_CONVERGED    1
#define HBSD_BUSY             2
#define HBSD_ERR_ARG        (-1)   /* invalid argument (sizes, NULL, layout)               */
#define HBSD_ERR_OOM        (-2)   /* device allocation failed or admission refused        */
#define HBSD_ERR_NOT_SPD    (-3)   /* factorisation of H - sigma_bar S met a pivot <= 0:   */
                                   /* sigma_bar is not below the spectrum (Sec. 5)         */
#define HBSD_ERR_RR_RANK    (-4)   /* search space rank below the number of wanted pairs   */
#define HBSD_ERR_TIMEOUT    (-5)   /* a device-side wait gave up                           */
#define HBSD_ERR_CUDA       (-6)   /* CUDA runtime error; see hbsd_last_error()            */
#define HBSD_ERR_UNSUPPORTED (-7)  /* valid request for a feature the library lacks        */

/* ---- problem description ----------------------------------------------------------- */

/* Sparse matrix in CSR form (host memory).  row_ptr has n+1 int64 entries, col_idx nnz
 * int32 column indices sorted within each row, val nnz doubles (is_complex = 0) or 2*nnz
 * interleaved (re, im) doubles (is_complex = 1).  H and S given to hbsd_create must have
 * identical n, row_ptr and col_idx (Sec. 4 footnote: one pattern). */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const double* val;
    int is_complex;
} hbsd_csr;

/* Geometry of the discretisation (host memory), used to order the sparse factorisation of
 * the global preconditioner (Sec. 4, Eq. ldl) by nested dissection of the periodic node
 * grid.  dof_node[i] in [0, grid[0]*grid[1]*grid[2]) is the mesh node carrying dof i, with
 * node index ix + grid[0]*(iy + grid[1]*iz); dof_cluster[i] is the atom cluster of an
 * enrichment dof or -1 (informational). */
typedef struct {
    const int32_t* dof_node;
    const int32_t* dof_cluster;
    int32_t grid[3];
} hbsd_local_blocks;

#define HBSD_PRECISION_FP64   0   /* every step in FP64                                  */
#define HBSD_PRECISION_MIXED  1   /* step 6(a) and MINRES's operator products in FP32 on the
                                     scaled pencil; steps 3/7, 8 and 10-11 in double-float
                                     (options minres_f32, spmm_df64); residual norms,
                                     Rayleigh-Ritz and the convergence test in FP64         */

#define HBSD_PRECOND_HYBRID   0   /* steps 6(a) + 6(b) (Sec. 3 hybrid scheme)           */
#define HBSD_PRECOND_GLOBAL   1   /* step 6(a) only (Eq. globalprecond)                  */
#define HBSD_PRECOND_LOCAL    2   /* step 6(b) only (Sec. 5 "local" comparison): P = -R,
                                     localized columns refined by MINRES from zero; no
                                     global factor is built                              */

/* Step 6(b) solvers (hbsd_options.local_solver) */
#define HBSD_LOCAL_MINRES     0   /* MINRES (Sec. 4, Eq. indls; Paige-Saunders)             */
#define HBSD_LOCAL_ONESTEP    1   /* first-order one-step iteration with the residual-
                                     minimising step (Sec. 6): p -= alpha d, d = A p + r,
                                     alpha = (A d . d) / (A d . A d); same stopping rule  */

/* Solver options.  hbsd_options_default() fills the paper's defaults (Sec. 5):
 * tau1 = tau2 = 0.1 (remark 4), eta = 0.25, max_minres = 20, max_outer = 1000,
 * m0 = -1 (= max(3, ceil(nev/10)), remark 1), sigma0 = NaN (= sigma_bar), tc_update = 0,
 * update_hs = -1, minres_f32 = 1, spmm_df64 = 1. */
typedef struct {
    double sigma_bar;   /* global shift eps_bar of K = (H - eps_bar S)^{-1}; must lie below the spectrum */
    double sigma0;      /* shift making H - sigma0 S positive definite (Sec. 5); NaN -> sigma_bar        */
    int m0;             /* guard vectors (remark 1); -1 -> default                                       */
    double tau1, tau2;  /* localisation thresholds (remark 4)                                           */
    double eta;         /* inexact-solve tolerance (Eq. approxp)                                        */
    int max_minres;     /* MINRES step cap per refinement                                               */
    int max_outer;      /* BPSD iteration cap                                                           */
    int precision;      /* HBSD_PRECISION_*                                                             */
    int precond;        /* HBSD_PRECOND_*                                                               */
    uint64_t seed;      /* seed of the SplitMix64 normals used when X0 is NULL                           */
    int local_solver;   /* HBSD_LOCAL_* (default MINRES)                                                */
    int tc_update;      /* mixed form, experimental: 1 runs steps 10-11 on the tensor cores from exact
                           bf16 slices (as hbsd_update_oz) while q <= 640; 0 (default) in double-float
                           on the FP32 pipes.  The slices are fixed point against each row's largest
                           entry, and the rows of the search blocks span many orders of magnitude
                           across their columns: with 1 the solves of the synthetic workloads stall
                           above 1e-8.  The FP64 form ignores it.                                       */
    int update_hs;      /* 1: Psi_H and Psi_S are updated with W like Psi (steps 10-11 as printed);
                           0: they are recomputed from the updated Psi by the fused SpMM of steps 3/7
                           (the same blocks up to rounding; one SpMM costs less than two block updates
                           when q is large); -1 (default): 1 in the FP64 form, which follows the
                           printed outline step for step; in the mixed form 0 for an update of width
                           q with q n > 1.5 nnz when the products are double-float (spmm_df64: 2 nnz
                           double-float multiply-adds per column against the two block updates' 2 n q),
                           q n > 3.5 nnz when they are FP64, else 1                                    */
    int minres_f32;     /* mixed form: 1 (default) computes the operator products of the MINRES steps
                           of 6(b) from the FP32 scaled pencil, (Hs - e S) v = D^-1 [(D Hs D) - e (D S
                           D)] (D^-1 v) with v, the Lanczos and Givens recurrences and the solution in
                           FP64; 0 in FP64 throughout.  The FP64 form ignores it.                      */
    int spmm_df64;      /* mixed form: 1 (default) computes the products of steps 3 and 7 and the
                           recomputation of Psi_H, Psi_S as hbsd_spmm_pair_df64 does, and checks
                           convergence on FP64 products; 0 in FP64.  Double-float sums carry about
                           48 bits: where the terms of H x, or of the Gram and update sums, cancel
                           strongly, the residuals stop short of tol.  So when the best Res_max has
                           not halved in 10 outer iterations once below 1e4 tol (or in 30 at any
                           level), the mixed form recomputes Psi_H and Psi_S in FP64 and runs the
                           products in FP64 from then on (hbsd_stats.fp64_from_iter); after a
                           further stall, the Gram and the update too (fp64_gram_from_iter).  The
                           FP64 form ignores it.                                                     */
} hbsd_options;

/* Statistics of one solve (all counts cumulative over the solve). */
typedef struct {
    int iters;               /* outer BPSD iterations (steps 4-11)                         */
    int iters_fp64;          /* of which with FP64 residuals and Rayleigh-Ritz (all, in    */
                             /* both forms)                                                */
    int64_t minres_steps;    /* total MINRES steps over all refined columns (M_s)          */
    int64_t precond_cols;    /* total columns through step 6(a)                            */
    int64_t local_cols;      /* total columns through step 6(b)                            */
    int rr_fallbacks;        /* Rayleigh-Ritz calls that took the rank-revealing branch    */
    double res_max;          /* final Res_max (Eq. res1), recomputed in FP64               */
    double t_factor_ms;      /* factorisation time of hbsd_create (host clock)            */
    double t_solve_ms;       /* hbsd_solve wall time                                       */
    int64_t nnz_L;           /* stored entries of the supernodal factor                    */
    int n_supernodes;
    int gpu_launches;        /* kernels launched by the last hbsd_solve                     */
    /* device time per LABPSD step class over the last solve (CUDA events on the session
     * stream), the breakdown of Sec. 5.3 / Fig. 8: */
    double t_matvec_ms;      /* steps 3 and 7: fused SpMM (H X, S X)                        */
    double t_resid_ms;       /* steps 4-5: residuals and norms                              */
    double t_precond_ms;     /* step 6(a): supernodal triangular solves                     */
    double t_local_ms;       /* step 6(b): MINRES refinement (shifted SpMM included)        */
    double t_gram_ms;        /* step 8                                                      */
    double t_rr_ms;          /* step 9                                                      */
    double t_update_ms;      /* steps 10-11                                                 */
    int64_t matvec_cols;     /* columns through steps 3 and 7                              */
    int64_t minres_spmm_cols;/* columns through the shifted SpMM of step 6(b)              */
    int precond_calls;       /* applications of step 6(a)                                   */
    int64_t local_calls;     /* launches of step 6(b) (one fused kernel per iteration with
                                localized columns)                                          */
    int64_t neg_pivots;      /* negative pivots of the LDL^T factor of H_loc - eps_bar S: the
                                number of eigenvalues of the local pencil below eps_bar
                                (Sylvester's inertia; 0 when eps_bar lies below the spectrum) */
    double gram_fma;         /* algorithmic multiply-adds of step 8 over the solve: n q (q+1)
                                per call (both reduced matrices, one triangle each)            */
    double update_fma;       /* algorithmic multiply-adds of steps 10-11: 3 n q w per call     */
    int fp64_from_iter;      /* mixed form: the outer iteration from which the products of
                                steps 3/7 ran in FP64 because Res_max had stalled in double-
                                float (no halving of its best value in 10 iterations once below
                                1e4 tol, or in 30); -1: never                                   */
    int fp64_gram_from_iter; /* mixed form: the same for the Gram and the update (a second
                                stall after the first switch); -1: never                       */
} hbsd_stats;

typedef struct hbsd_handle hbsd_handle;

void hbsd_options_default(hbsd_options* opt);

/* Create a solver session: copies H and S to the device, builds the SELL-C-sigma pattern
 * with interleaved (h, s) values (Sec. 4 footnote: one pattern), and factorises
 * H - sigma_bar S once (Sec. 4, Eq. ldl; remark: computed once and reused).  lb is required
 * (the ordering of the factorisation); opt may be NULL (defaults, sigma_bar must then be
 * set by hbsd_set_sigma, else HBSD_ERR_ARG).  stream: cudaStream_t as void* for all work of
 * the session (NULL = a stream the session creates).  The factor is a Cholesky when
 * sigma_bar lies below the spectrum; otherwise (a non-positive pivot) the factorisation is
 * redone as LDL^T with 1 x 1 pivots in the same order (Eq. ldl without 2 x 2 blocks), whose
 * negative pivots (hbsd_stats.neg_pivots) count the eigenvalues below sigma_bar; sigma0 must then
 * be set below the spectrum.  Returns HBSD_ERR_NOT_SPD if a pivot is zero or not finite.
 *
 * Complex Hermitian input (Sec. 2: H Hermitian, S Hermitian positive definite, complex at a
 * Bloch vector k != 0): H and S both with is_complex = 1 (HBSD_ERR_ARG if only one is).  The
 * session then holds the real symmetric pencil ([Hr, -Hi; Hi, Hr], [Sr, -Si; Si, Sr]) of size
 * 2n, equivalent to the complex one (every eigenvalue twice: x and i x), with the real and
 * imaginary part of each dof stored next to each other (real dof 2i is Re x_i, 2i+1 is Im x_i)
 * and factorised as above (both halves of a dof share its mesh node).  hbsd_solve and
 * hbsd_solve_device take and return complex blocks (see there); every step-level entry point
 * acts on the real-equivalent pencil, with 2n rows in that order.  hbsd_n returns n. */
int hbsd_create(const hbsd_csr* H, const hbsd_csr* S, const hbsd_local_blocks* lb,
                const hbsd_options* opt, void* stream, hbsd_handle** out);

/* Replace H's values (same pattern) for an SCF follow-up; the global factor keeps the
 * first H (Sec. 4: K built from H^(1) and reused through the SCF).  H_val: nnz doubles, or
 * 2 nnz interleaved (re, im) doubles on a complex session. */
int hbsd_update_H(hbsd_handle* h, const double* H_val);

/* Nonlocal term of the Hamiltonian (Sec. 4, Eq. fgf): from now on the session's H is
 * H_loc + F G F^T, with H_loc the CSR values given to hbsd_create / hbsd_update_H.
 * F: host, row-major n x k (leading dimension ldf >= k), the projector matrix; only its
 * nonzero entries are stored, so projectors of compact support make its products cheap.
 * G: host, row-major k x k, symmetric (HBSD_ERR_ARG if |G_lm - G_ml| > 1e-14 max|G|).
 * Both are copied; k = 0 removes the term (F, G may then be NULL).  k <= 4096.
 * Every product with H (steps 3 and 7, the MINRES operator of step 6(b), hbsd_spmm_pair,
 * hbsd_spmm_shifted, the FP32 entry points on the scaled pencil) adds F (G (F^T X)); the
 * global preconditioner becomes the Sherman-Morrison-Woodbury inverse of
 * H_loc^(1) - eps_bar S + F G F^T (Sec. 4, steps 1-6): Fhat = K F and M = (I + G F^T Fhat)^{-1} G
 * are formed on first use with the factor of the local part and kept until the next call.
 * HBSD_ERR_ARG there if I + G F^T Fhat is singular.  The factor itself is unchanged (it is
 * that of the local part).  Waits for the session's stream; not to be called during a solve.
 * HBSD_ERR_UNSUPPORTED for k > 0 on a complex session. */
int hbsd_set_nonlocal(hbsd_handle* h, int k, const double* F, int64_t ldf, const double* G);

/* LABPSD (Sec. 3 outline, steps 1-12): lowest nev eigenpairs to Res_max <= tol (remark 2).
 * X0: host, row-major n x (nev + m0) start block (remark 1), or NULL for seed-normal draws,
 * or the previous solve's block if warm != 0 (X0 must then be NULL).  lambda: host, nev
 * unshifted eigenvalues ascending.  X: host, row-major n x nev S-orthonormal eigenvectors, or
 * NULL.  iters, st: nullable.  Synchronous.
 *
 * Complex session: X0 is n x (nev + m0) complex (2 doubles per entry, re then im; NULL draws
 * the real parts from the SplitMix64 normals of stream 2 and the imaginary parts from stream 6
 * of opt.seed) and X is n x nev complex, S-orthonormal in x^H S y.  The solve runs LABPSD on the
 * real-equivalent pencil for 2 nev pairs with 2 m0 guard columns from the start block whose
 * columns are the realified x_c and J x_c (J: multiplication by i), whose span every step keeps
 * invariant under J: it is the complex iteration of the outline in real arithmetic, and iters
 * and hbsd_stats count its iterations.  From the 2 nev real eigenvectors, nev complex
 * directions are then selected on the GPU in ascending eigenvalue order and S-orthonormalised
 * (HBSD_ERR_RR_RANK if fewer than nev are independent).  nev <= 512.  The nonlocal term is not
 * available on complex sessions. */
int hbsd_solve(hbsd_handle* h, int nev, double tol, const double* X0, int warm,
               double* lambda, double* X, int* iters, hbsd_stats* st);

/* Same as hbsd_solve with device buffers: X0_dev row-major n x (nev+m0), ld = ldx0 (or NULL),
 * lambda_dev nev doubles, X_dev row-major n x nev with ld = ldx (or NULL).  On a complex
 * session X0_dev and X_dev are complex (re, im doubles per entry) and ldx0, ldx count complex
 * entries. */
int hbsd_solve_device(hbsd_handle* h, int nev, double tol, const double* X0_dev, int64_t ldx0,
                      double* lambda_dev, double* X_dev, int64_t ldx, int* iters, hbsd_stats* st);

/* Res_max = max_i Res_i (Eq. res1) at every convergence test (step 5) of the session's last
 * solve, in order: entry 0 follows the Rayleigh-Ritz on the start block, the last is the value
 * that stopped the solve.  Writes at most cap values to out (host; NULL if cap = 0) and returns
 * how many there are. */
int hbsd_res_history(const hbsd_handle* h, double* out, int cap);

/* The stall test of the mixed form's precision escalation (hbsd_options.spmm_df64), on a history
 * of Res_max values (host, len doubles, in order): 1 when more than win entries follow index mark
 * (the history length at the last switch), the best value before the last win entries is below
 * `below`, and the best of the last win entries is above half of it; else 0.  The solve applies it
 * with (win, below) = (10, 1e4 tol) and (30, +inf).  HBSD_ERR_ARG for len < 0, mark outside
 * [0, len], win < 1 or a NULL hist with len > 0.  Host only. */
int hbsd_res_stalled(const double* hist, int len, int mark, int win, double below);

void hbsd_destroy(hbsd_handle* h);
const char* hbsd_status_string(int status);
const char* hbsd_last_error(void);
int64_t hbsd_n(const hbsd_handle* h);
int hbsd_is_complex(const hbsd_handle* h);   /* 1 for a session created from complex input */
double hbsd_sigma0(const hbsd_handle* h);
void hbsd_get_stats(const hbsd_handle* h, hbsd_stats* st);

/* ---- step-level entry points (device pointers, the session's stream) -------------------
 * Each runs one step of the LABPSD outline exactly as hbsd_solve does, so that each step can
 * be checked on its own.  All block vectors are row-major FP64 with the ld given. */

/* Steps 3 and 7: HX = (H - sigma0 S) X and SX = S X for an n x k block X. */
int hbsd_spmm_pair(hbsd_handle* h, const double* X, int64_t ldx, int k,
                   double* HX, int64_t ldhx, double* SX, int64_t ldsx);

/* Operator of step 6(b): Y(:,j) = (H - sigma0 S - e_j S) X(:,j), e (device, k doubles)
 * shifts relative to sigma0. */
int hbsd_spmm_shifted(hbsd_handle* h, const double* X, int64_t ldx, int k, const double* e,
                      double* Y, int64_t ldy);

/* Steps 3 and 7 in double-float arithmetic (the mixed form's products): HX = Hs X and SX = S X
 * computed as D^-1 [(D Hs D)(D^-1 X)] and D^-1 [(D S D)(D^-1 X)], D = diag(S)^{-1/2}, with the
 * scaled values and D^-1 X split into float pairs and every product and sum in double-float
 * (about 2^-44 relative to |Hs||X| per entry; on the scaled pencil, whose entries are O(1), no
 * value falls below the float range).  FP64 device blocks as in hbsd_spmm_pair; the nonlocal term
 * is added in FP64. */
int hbsd_spmm_pair_df64(hbsd_handle* h, const double* X, int64_t ldx, int k, double* HX, int64_t ldhx,
                        double* SX, int64_t ldsx);

/* FP32 forms on the scaled pencil (hbsd_precond_apply_f32 is step 6(a) of HBSD_PRECISION_MIXED;
 * hbsd_spmm_pair_f32 is a step-level product on the FP32 copy of the matrix).  They act on the
 * diagonally scaled pencil (D Hs D, D S D), D = diag(S)^{-1/2} (hbsd_dscale returns D, host,
 * n doubles): hbsd_spmm_pair_f32 gives (D Hs D) X and (D S D) X; hbsd_precond_apply_f32 gives
 * P = -(D (H - sigma_bar S) D)^{-1} R from the FP32 copy of the factor panels.  Blocks are
 * row-major FP32 with ld a multiple of 4 and 16-byte aligned pointers. */
int hbsd_spmm_pair_f32(hbsd_handle* h, const float* X, int64_t ldx, int k, float* HX, int64_t ldhx,
                       float* SX, int64_t ldsx);
int hbsd_precond_apply_f32(hbsd_handle* h, const float* R, int64_t ldr, int k, float* P, int64_t ldp);
int hbsd_dscale(const hbsd_handle* h, double* d_host);

/* Steps 4-5 (Eq. res1): for j < m, r_j = PsiH(:,j) - PsiS(:,j) E_j and
 * res[j] = ||r_j|| / ||PsiH(:,j)|| (device outputs: R n x m with ldr, res m doubles). */
int hbsd_residual(hbsd_handle* h, const double* PsiH, int64_t ldh, const double* PsiS,
                  int64_t lds, const double* E, int m, double* R, int64_t ldr, double* res);

/* Step 6(a) (Eq. k1p): P = -(H - sigma_bar S)^{-1} R for an n x k block, by the
 * supernodal factor of hbsd_create. */
int hbsd_precond_apply(hbsd_handle* h, const double* R, int64_t ldr, int k, double* P,
                       int64_t ldp);

/* Step 6(b) (Eq. indls, Eq. approxp): for each column j of the n x k block P, MINRES on
 * (H - sigma0 S - e_j S) y = -r_j from y0 = P(:,j), stopped when the recurrence residual is
 * <= eta ||r_j|| or after max_minres steps; P(:,j) := y.  steps (device, k ints): steps
 * taken per column. */
int hbsd_minres(hbsd_handle* h, const double* R, int64_t ldr, const double* e, int k,
                double eta, int max_minres, double* P, int64_t ldp, int* steps);

/* The first-order one-step refinement (Sec. 6) with the arguments and the stopping rule of
 * hbsd_minres: for column j, d = (Hs - e_j S) P(:, j) + R(:, j), P(:, j) -= alpha d with
 * alpha = (A d . d) / (A d . A d), until ||d|| <= eta ||R(:, j)|| or max_steps steps (steps[j]
 * steps taken, device, nullable).  Device pointers; synchronous. */
int hbsd_onestep(hbsd_handle* h, const double* R, int64_t ldr, const double* e, int k,
                 double eta, int max_steps, double* P, int64_t ldp, int* steps);

/* Step 8: H_R = Z^T ZH and S_R = Z^T ZS (q x q, row-major, ld q), made exactly symmetric
 * as (A + A^T)/2; Z, ZH, ZS are n x q row-major blocks. */
int hbsd_gram(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS,
              int64_t ldzs, int64_t n, int q, double* HR, double* SR, void* stream);

/* Steps 10-11 on the tensor cores: Y = [Z0 Z1] W with FP64 operands and result, computed from
 * exact bf16 slices (8 six-bit digits per entry, against the largest entry of each row of Z0, of
 * each row of Z1 and of each column of W's two row blocks) whose products of equal weight are
 * summed exactly in FP32 tensor-memory accumulators (tcgen05.mma); products of weight below 2^-48
 * are dropped.  Error per entry about 2^-46 (max|Z_g(i,:)| sum_k |W_g(k,j)| + sum_k |Z_g(i,k)|
 * max|W_g(:,j)|) summed over the two blocks g: the accuracy of FP64 relative to each row's and
 * column's largest entry (fixed point), where FP64 itself is relative per product.  Z0 n x q0 (ld0), Z1 n x q1 (ld1; q1 may be 0), W
 * (q0 + q1) x k row-major (ld k), Y n x k (ldy), all device; Y must not overlap Z0 or Z1.
 * 1 <= q0 <= 640, 0 <= q1 <= 640 (HBSD_ERR_ARG otherwise).  Synchronous. */
int hbsd_update_oz(const double* Z0, int64_t ld0, int q0, const double* Z1, int64_t ld1, int q1,
                   int64_t n, const double* W, int k, double* Y, int64_t ldy, void* stream);

/* Tensor-core building block of the split-slice products: D = A B^T with A (M x K) and B (N x K)
 * row-major bf16 (uint16 bit patterns), D (M x N) row-major FP32, all device pointers; one CTA per
 * 128 rows of D issues tcgen05.mma (kind::f16, FP32 accumulation in tensor memory) on shared-memory
 * tiles of 16 K-columns.  M a multiple of 128, N a multiple of 16 in [16, 256], K a multiple of 16
 * (HBSD_ERR_ARG otherwise).  variant 0 is the operand layout the products use; variant 1 describes
 * the same tiles with the descriptor's two core-matrix offsets exchanged (a layout check).
 * HBSD_ERR_TIMEOUT if an MMA completion wait gives up (2 s).  Synchronous.  The paper has no
 * counterpart: its products run on CPU BLAS. */
int hbsd_tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K, int variant,
                      void* stream);

/* Allocation-free form of hbsd_gram, for callers that must not allocate device memory:
 * a serving loop whose per-request path may not call cudaMalloc / cudaFree (both can
 * synchronise the whole device and stall the requests already in flight), or a host whose
 * memory pool owns all device memory up front.  It computes what hbsd_gram computes, the same
 * result up to rounding (for large q it sums fewer row chunks, so the order of the partial sums
 * differs), but its scratch is a file-scope device array of 2^21 doubles (16 MiB) that every
 * device which loads the library holds until the process exits; the paper has no counterpart.
 * Sizes: q <= 1024 (2 q^2 scratch doubles per row chunk); a larger q returns HBSD_ERR_ARG
 * before any other argument check.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it, so make that first call
 * before any stream capture, and do not use the library across a cudaDeviceReset (the array may
 * then live at another address).  All calls share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller; each call overwrites every scratch element it reads, so nothing
 * carries over from the previous call.  Asynchronous on stream; no allocation, no free. */
int hbsd_gram_noalloc(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh,
                      const double* ZS, int64_t ldzs, int64_t n, int q, double* HR, double* SR,
                      void* stream);

/* Step 9: lowest k eigenpairs of H_R W = S_R W Theta (q x q inputs row-major, ld q, device).
 * Diagonal scaling D = diag(S_R)^{-1/2}, Cholesky of D S_R D, symmetric eigensolve of
 * L^{-1} D H_R D L^{-T}; if the Cholesky breaks down or a pivot is below 1e-14 the
 * eigen-directions of D S_R D below 1e-14 * max are dropped instead.  Outputs (device):
 * theta k doubles ascending, W q x k row-major (ld k), info[0] = 1 if that fallback was
 * taken, info[1] = rank used.  Returns HBSD_ERR_RR_RANK if the rank is below k.  The
 * workspace is internal.  Synchronous (reads back info). */
int hbsd_rayleigh_ritz(const double* HR, const double* SR, int q, int k, double* theta,
                       double* W, int* info, void* stream);

/* Steps 10-11: Z(:, 0:k) := Z(:, 0:q) W in place, row by row, for an n x q block Z and a
 * q x k matrix W (row-major, ld k, device), k <= q. */
int hbsd_update(double* Z, int64_t ldz, int64_t n, int q, const double* W, int k, void* stream);

/* ---- Served form (continuous batching of solve requests on one GPU) ------------------------
 *
 * A server runs up to max_slots requests at a time, each on its own CUDA stream, so the kernels
 * of different solves overlap on the device.  Requests are taken in arrival order, except that
 * one that cannot run yet (its session busy with an earlier request, or not enough device
 * memory under hbm_budget_bytes) does not hold back later ones.  A new problem is copied at
 * submission and factorised when it runs; its session (matrix, factor, last block) then stays
 * resident for follow-up requests (SCF steps, Sec. 3: new H values on the same pattern, warm
 * start from the previous block; the factor of the session's first H is kept, reading R2).
 * Idle sessions are evicted least-recently-used first when memory is short, or released by the
 * caller.  Admission reserves a per-problem estimate of device memory (from n, nnz and nev,
 * scaled by the largest ratio of a request's peak device allocation to its estimate seen so
 * far, at least 1.25); once a request ends,
 * its session's measured footprint (the device memory its create and solves left allocated)
 * replaces the reservation.  A request whose allocation still fails on the device frees every
 * idle session and retries once before it reports HBSD_ERR_OOM.  All functions are
 * thread-safe. */
typedef struct {
    size_t hbm_budget_bytes;  /* device memory the server may hold; 0 = 80% of the free memory */
    int max_slots;            /* requests running at once (1..64), default 4                   */
} hbsd_server_opts;

typedef struct {
    /* new problem: H, S, lb and opt (copied at submission); session_id = -1 */
    const hbsd_csr* H;
    const hbsd_csr* S;
    const hbsd_local_blocks* lb;
    const hbsd_options* opt;
    /* follow-up: session_id >= 0 (from an earlier result); H_val = new H values (nnz
     * doubles, copied) or NULL to keep H */
    int64_t session_id;
    const double* H_val;
    int nev;
    double tol;
    const double* X0;   /* host, n x (nev + m0) row-major, copied; or NULL (seeded start) */
    int warm;           /* follow-up only: start from the session's last block (X0 = NULL) */
    /* new problem only: nonlocal term F G F^T as in hbsd_set_nonlocal (nl_k = 0: none);
     * F n x nl_k row-major with leading dimension nl_ldf, G nl_k x nl_k; both copied.  A
     * follow-up keeps its session's term. */
    int nl_k;
    const double* nl_F;
    int64_t nl_ldf;
    const double* nl_G;
} hbsd_request;

typedef struct {
    uint64_t ticket;
    int status;          /* HBSD_OK, HBSD_NOT_CONVERGED or an error code of the solve       */
    int iters;
    int64_t session_id;  /* the session the request ran in (-1 if a new problem failed)     */
    double res_max;      /* final max relative residual                                     */
    double latency_ms;   /* submission to completion                                        */
    double queue_ms;     /* submission to start                                             */
    double run_ms;       /* start to completion (factorisation included for a new problem)  */
} hbsd_result;

typedef struct hbsd_server hbsd_server;

void hbsd_server_opts_default(hbsd_server_opts* opts);
/* Starts the worker threads.  HBSD_ERR_ARG for max_slots outside [1, 64]. */
int hbsd_server_create(const hbsd_server_opts* opts, hbsd_server** out);
/* Queues a request and returns at once with its ticket.  lambda_out (nev doubles) and X_out
 * (n x nev, row-major, or NULL) are host buffers the caller keeps valid until the result has
 * been polled.  A complex problem (H and S with is_complex = 1, Bloch phases) runs as in
 * hbsd_solve on a complex session: X0, X_out and the H_val of its follow-ups are complex
 * (re, im doubles per entry), and it is admitted by the footprint of its real pencil of size
 * 2n; the nonlocal term is not available for it (HBSD_ERR_UNSUPPORTED).  HBSD_ERR_OOM if the problem alone exceeds the memory budget, HBSD_ERR_ARG for
 * an unknown session or malformed input. */
int hbsd_submit(hbsd_server* sv, const hbsd_request* rq, double* lambda_out, double* X_out, uint64_t* ticket);
/* HBSD_BUSY while the request is queued or running; HBSD_OK once, with the result (the ticket
 * is then forgotten); HBSD_ERR_ARG for an unknown ticket. */
int hbsd_poll(hbsd_server* sv, uint64_t ticket, hbsd_result* out);
/* Frees an idle session now (HBSD_BUSY while a request of it runs). */
int hbsd_session_release(hbsd_server* sv, int64_t session_id);
/* Waits for the running requests, stops the workers and frees every session; queued requests
 * are dropped. */
void hbsd_server_destroy(hbsd_server* sv);

/* ---- Batched form (many resident sessions solved in one call) --------------------------------
 *
 * Independent problems of uneven size -- k-points, SCF runs, configurations (Sec. 5: each is a
 * separate eigenproblem of the same method) -- created beforehand with hbsd_create, each with
 * its own stream, and solved together: worker threads take the sessions longest-first by the
 * estimated cost nev' (nnz + n nev') with nev' the block width, and run each solve on its
 * session's stream, so that the kernels of different sessions overlap on the device.  Before
 * that, each session that has not been tuned for its block width is tuned (hbsd_autotune).
 *
 * Autotuner: for one session and block width w, times the candidate launch shapes of the two
 * steps whose best shape depends on the problem's size, on seeded data on the session's stream,
 * and keeps the fastest for the session's later solves:
 *   - the fused SpMM of steps 3/7 (in the session's precision form; w columns): the most lanes
 *     per matrix row, 4, 8, 16 or 32 (fewer lanes per row put more rows in a CTA and more
 *     column chunks in a lane);
 *   - the cooperative MINRES launch of step 6(b) (min(w, 32) columns, 10 steps): its CTA count,
 *     the whole GPU or 1/2 ... 1/32 of it; the smallest count within 10% of the fastest is kept
 *     (cheaper grid barriers, and SMs left to the other sessions of a batch).
 * Results of sessions with equal precision form, block width and n, nnz within 20% are shared
 * (a process-wide table), so a batch of similar problems is timed once per size class.  Tuning
 * changes the order of floating-point sums in those two steps only; a tuned session solved alone
 * gives bit for bit the results it gives in a batch. */
typedef struct {
    int width;                 /* block width tuned for                                         */
    int spmm_lanes;            /* chosen most lanes per row of the fused SpMM                   */
    int minres_ctas;           /* chosen CTA count of the MINRES launch                          */
    int minres_ctas_full;      /* the whole-GPU CTA count                                        */
    int from_table;            /* 1: taken from an earlier session of the same size class       */
    double spmm_ms[4];         /* time per candidate (4, 8, 16, 32 lanes), ms; 0 if not timed    */
    double minres_ms[6];       /* time per candidate (full, 1/2, ..., 1/32 of the CTAs), ms     */
} hbsd_tune;

/* Tune session h for solves of block width `width` (nev + m0, or 2 (nev + m0) on a complex
 * session; see hbsd_solve).  Synchronous; allocates and frees scratch blocks of n x width.
 * out: nullable.  HBSD_ERR_ARG for width < 1. */
int hbsd_autotune(hbsd_handle* h, int width, hbsd_tune* out);

typedef struct {
    hbsd_handle* h;            /* a session; each at most once per call                          */
    int nev;
    double tol;
    const double* X0_dev;      /* as hbsd_solve_device: device start block or NULL              */
    int64_t ldx0;
    double* lambda_dev;        /* device, nev doubles                                            */
    double* X_dev;             /* device, n x nev row-major (ld = ldx), or NULL                  */
    int64_t ldx;
    /* out */
    int status;                /* of this session's solve: HBSD_OK, HBSD_NOT_CONVERGED, error   */
    int iters;
    double res_max;
    double run_ms;             /* wall time of this session's solve                             */
    double start_ms;           /* its start, from the call's start                              */
} hbsd_batch_item;

typedef struct {
    int max_concurrent;        /* sessions solved at once (1..64); default 8                     */
    int autotune;              /* 1 (default): tune untuned sessions first; 0: built-in shapes  */
    int longest_first;         /* 1 (default): by estimated cost; 0: in the given order          */
} hbsd_batch_opts;

void hbsd_batch_opts_default(hbsd_batch_opts* opts);
/* Solves every item; returns HBSD_OK when every item's status is HBSD_OK, else the first item's
 * status (in item order) that is not.  HBSD_ERR_ARG (nothing run) for a NULL or repeated
 * handle, count < 0, max_concurrent outside [1, 64]. */
int hbsd_solve_batch(hbsd_batch_item* items, int count, const hbsd_batch_opts* opts);

/* Double-float forms of hbsd_gram and hbsd_update, the ones the mixed form (HBSD_PRECISION_MIXED)
 * runs: FP64 inputs and outputs, products and short sums in pairs of floats (about 48 bits per
 * term, TwoProd / TwoSum), the Gram sums accumulated in FP64 across 128-row tiles.  hbsd_gram_df64
 * computes the entries a <= b of Z^T ZH and Z^T ZS and mirrors them (no averaging).  Arguments,
 * layouts and errors as hbsd_gram / hbsd_update; FP64 values enter the products with ~47 bits
 * above 2^-96 in magnitude, at least 24 bits down to 2^-126, and as zero below.  hbsd_update_df64
 * takes q <= 3520 (8 rows of q pairs staged in 220 KB of shared memory; HBSD_ERR_ARG otherwise). */
int hbsd_gram_df64(const double* Z, int64_t ldz, const double* ZH, int64_t ldzh, const double* ZS,
                   int64_t ldzs, int64_t n, int q, double* HR, double* SR, void* stream);
int hbsd_update_df64(double* Z, int64_t ldz, int64_t n, int q, const double* W, int k, void* stream);

/* The start-block generator used when hbsd_solve gets X0 = NULL (host only, no GPU needed):
 * count standard normals from SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based
 * generator (draw t = mix(key + (t+1) * 0x9E3779B97F4A7C15), key = mix((seed ^ stream *
 * 0x9E3779B97F4A7C15) + 0x9E3779B97F4A7C15)), uniforms from the top 53 bits, Box-Muller on
 * consecutive pairs.  hbsd_solve uses stream 2 and the options' seed; entry (i, j) of the
 * n x (nev + m0) block is draw i * (nev + m0) + j.  The paper has no counterpart (its start
 * vectors come from the previous SCF step, remark 1). */
int hbsd_seed_normals(uint64_t seed, uint64_t stream, int64_t count, double* out);

/* ---- measurement ------------------------------------------------------------------
 * Sustained FMA throughput of the SIMT pipes on the current device (which = 0: FP64, 1: FP32),
 * in FLOP/s (an FMA counts 2), from one timed launch of independent FMA chains on every SM.
 * The paper has no counterpart; it supplies the ALU peak that the FP64 rooflines divide by.
 * Synchronous. */
int hbsd_probe_peak(int which, void* stream, double* flops_per_s);

/* Failure path of the device-side waits (no counterpart in the paper): launches the bounded grid
 * barrier of the fused MINRES kernel on two blocks that wait for a third arrival that never
 * comes, with a wait limit of limit_s seconds (clamped to [1 ms, 5 s]).  Both blocks give up,
 * raise the error flag and return, and the call returns HBSD_ERR_TIMEOUT -- the status a solve
 * reports when a MINRES barrier times out; the CUDA context stays usable.  Any other outcome
 * returns HBSD_ERR_CUDA.  Synchronous. */
int hbsd_probe_barrier_timeout(double limit_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HBSD_H */
