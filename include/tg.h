/*
 * tg.h - C ABI of the two-grid deflated Krylov solver for sm_103a (GB300).
 *
 * Method: Morgan, Whyte, Wilcox, Yang, "Two-grid deflated Krylov methods for linear
 * equations".  A x = b from a PDE discretisation (Section 1) is solved in three phases:
 *   1. GMRES-DR(m,k) on a coarse grid (Section 2.1; Section 3 box, phase 1) solves the
 *      coarse problem and finds k approximate eigenvectors;
 *   2. the eigenvectors and the coarse solution are moved to the fine grid (Section 3
 *      box, phase 1: "move the approximate eigenvectors to the fine grid");
 *   3. restarted BiCGStab (Section 4.1 box, BiCGStab(ncyc)-Proj(k)) or GMRES (Section 2.2,
 *      GMRES(m)-Proj(k)) with a projection over those vectors between cycles.
 *
 * Conventions for every entry point:
 *   - Vector arguments are DEVICE pointers owned by the caller unless stated otherwise;
 *     they must stay valid until the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t (passed as void*); NULL means the legacy default stream.
 *     Calls queue their kernels on it.  Calls that return results to host memory
 *     (tg_stats, cycle counts) synchronise that stream before returning.
 *   - Handles (tg_op, tg_defl) own their device workspaces; they are not thread safe.
 *   - Errors are returned as a status code (TG_OK = 0).  No entry point traps, aborts or
 *     prints; a CUDA error is reported as TG_CUDA_ERROR and the handle stays destroyable.
 *   - Grid vectors are x-fastest lexicographic: 2D index (j-1)*N + (i-1); 3D index
 *     (i-1) + N*((j-1) + N*(k-1)), 1 <= i, j, k <= N, h = 1/(N+1), zero Dirichlet values
 *     outside.  Lattice vectors: site x0 + L*(x1 + L*(x2 + L*x3)), complex128 stored as
 *     interleaved (re, im) doubles.
 *   - Real vectors are float64 in TG_F64 mode; in TG_F32_IR mode the right-hand side and
 *     solution stay float64 (the outer refinement) and only the inner iteration is float32.
 *   - Multi-column arrays (bases, multiple right-hand sides) are column-major with
 *     leading dimension n: column c starts at c * n elements.
 */
#ifndef TG_H
#define TG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- status codes */
#define TG_OK            0  /* success                                                   */
#define TG_NOT_CONVERGED 1  /* tolerance not reached within max_mvps / max_cycles        */
#define TG_BREAKDOWN     2  /* BiCGStab breakdown that restarting could not cure          */
#define TG_NAN           3  /* a NaN/Inf appeared in a residual norm or reduction         */
#define TG_BAD_ARG       4  /* invalid argument (message from tg_last_error)              */
#define TG_OOM           5  /* device allocation failed                                   */
#define TG_CUDA_ERROR    6  /* a CUDA runtime call failed (message from tg_last_error)    */
#define TG_SYNC_TIMEOUT  7  /* a bounded device-side wait gave up                          */

/* ----------------------------------------------------------------------- enumerations */
enum { TG_CD2D = 0, TG_CD3D = 1, TG_U1_4D = 2, TG_VARK2D = 3, TG_EXP2D = 4 };  /* operator kinds */
enum { TG_BICGSTAB = 0, TG_GMRES = 1 };                            /* fine-grid method   */
enum { TG_PROJ_MINRES = 0, TG_PROJ_GALERKIN = 1 };                 /* projection kind    */
enum { TG_F64 = 0, TG_F32_IR = 1 };                                /* precision mode     */
enum { TG_FINE = 0, TG_COARSE = 1 };                               /* grid level         */

typedef struct tg_op tg_op;       /* fine + coarse operator, grid maps, workspaces       */
typedef struct tg_defl tg_defl;   /* deflation basis Y, A Y factored, projection data     */
typedef struct tg_batch tg_batch; /* many instances x 8 right-hand sides (added form)    */

/* Per-solve statistics (host memory, filled by the solvers). */
typedef struct tg_stats {
    int64_t mvps;           /* fine-grid operator applications (the paper's "mvp")      */
    int64_t coarse_mvps;    /* coarse-grid operator applications                         */
    int64_t vops;           /* length-n vector operations (cost model of Example 1)      */
    int32_t cycles;         /* restarted cycles (fine solve) or GMRES-DR cycles (coarse)  */
    int32_t status;         /* TG_* status of this solve                                 */
    double  relres;         /* ||b - A x|| / ||b||, recomputed in float64 at exit        */
    double  coarse_relres;  /* coarse least-squares residual / ||b_c|| (GMRES-DR)        */
    int32_t kk;             /* number of deflation vectors produced (k or k+1)           */
    int32_t eig_converged;  /* harmonic Ritz pairs meeting rtolev at the last cycle       */
    double *history;        /* optional host buffer of 3*history_cap doubles: per cycle   */
                            /* (||r||/||b|| after the projection, rticyc, mvps so far)   */
    int32_t history_cap;
    int32_t history_len;    /* entries written                                           */
    int32_t fp64_cycles;    /* TG_F32_IR: cycles finished in float64 after a float32      */
                            /* correction failed to lower the float64 residual            */
    int32_t reserved;
} tg_stats;

/* Human-readable text of a status code, and of the last error on this thread. */
const char *tg_status_string(int status);
const char *tg_last_error(void);

/* ------------------------------------------------------------------ operator set-up
 * Builds the fine operator and its coarse partner (Section 3: the coarse problem is the
 * same PDE at h_c = 2h, Example 1 and Example 4; for the lattice, the Galerkin product
 * P^H A P of the 2^4 block-transport prolongation).
 *   kind   TG_CD2D   -u_xx - u_yy + beta[0] u_x + c u, 5-point centred, dims = {N}, N odd
 *          TG_CD3D   -Lap u + beta . grad u + c u, 7-point centred, dims = {N}, N odd, beta[3]
 *          TG_EXP2D  -exp(beta[2] x y)(u_xx + u_yy) + beta[0] u_x + beta[1] u_y + c u,
 *                    5-point centred at x = i h, y = j h, dims = {N}, N odd, beta[3]
 *                    (Example 1: beta = {40, 40, 5}, c = 0)
 *          TG_VARK2D -div(kappa grad u) + beta[0] u_x, dims = {N}, N odd;
 *                    coeffs = device float64 kappa on the (N+2)^2 node grid, index
 *                    j*(N+2)+i; faces use the arithmetic mean of their two nodes
 *          TG_U1_4D  (m+8) psi(x) - sum_mu [U_mu(x) psi(x+mu) + conj(U_mu(x-mu)) psi(x-mu)],
 *                    dims = {L}, L even, periodic; *mass = m; coeffs = device complex128
 *                    links U[mu][site], mu = 0..3
 *   mass   lattice: the mass m (required); TG_CD2D / TG_CD3D / TG_EXP2D: the reaction
 *          coefficient c (NULL means 0; Example 4's Helmholtz operator -Lap u - 100^2 u is
 *          TG_CD2D with beta = 0, c = -1e4), on the coarse level too; TG_VARK2D: NULL or 0
 *   ndim   1 (all kinds take one size; the grid dimension follows from kind)
 *   coarse_factor must be 2.
 * The coefficient arrays are copied; the caller may free them after the call.
 * Returns TG_BAD_ARG for an unknown kind, an even N (grids), an odd L (lattice) or
 * N < 3.  Any beta is accepted: |beta h / 2| >= 1 (no closed-form spectrum) is fine.   */
int tg_setup_operator(tg_op **op, int kind, const int64_t *dims, int ndim,
                      const double *beta, const double *mass, const void *coeffs,
                      int coarse_factor, void *stream);
int tg_destroy_op(tg_op *op);

/* Sizes of the fine (level 0) and coarse (level 1) problems. */
int64_t tg_op_size(const tg_op *op, int level);

/* y = A x (transpose = 0) or y = A^T x (transpose = 1; the conjugate transpose for the
 * lattice, which is Hermitian) on the given level.  precision TG_F64: float64 (complex128
 * lattice) vectors; TG_F32_IR: float32 vectors, coefficients rounded to float32.
 * One operator application; x and y must not overlap.                                 */
int tg_apply(const tg_op *op, int level, int transpose, int precision,
             const void *x, void *y, void *stream);

/* Grid transfer (Section 3, phase 1).  Prolongation coarse -> fine of ncols columns:
 * bilinear (2D) / trilinear (3D) with a fixed summation order (pairs along x, then y,
 * then z; the weight applied last), so results are reproducible bit for bit; lattice:
 * psi(x) = (1/4) conj(W(x)) psi_c(X), W the link product on the path from the block
 * corner 2X to x in mu order.  Restriction fine -> coarse: full weighting P^T / 2^d
 * (grids) or P^H (lattice).                                                            */
int tg_prolong(const tg_op *op, const void *coarse, void *fine, int ncols, void *stream);
int tg_restrict(const tg_op *op, const void *fine, void *coarse, int ncols, void *stream);

/* Interpolation used by every prolongation of this operator (tg_prolong, the moved
 * eigenvectors and x0 of tg_coarse_gmresdr, the batched set-up).  TG_INTERP_LINEAR (the
 * default): bilinear / trilinear as above.  TG_INTERP_CUBIC: fourth-order interpolation in
 * place of the paper's splines (Section 3, phase 1 "we generally use spline
 * interpolation"): a fine point halfway between coarse nodes a, a+1 takes (-1, 9, 9, -1)/16
 * of nodes a-1..a+2, with the grid function continued oddly beyond the Dirichlet boundary
 * (node -1 = -u(1), node Nc+2 = -u(Nc)); tensor product in x, then y, then z, each sum
 * rounded in a fixed order, so results are reproducible bit for bit.  Grid kinds only
 * (TG_BAD_ARG for the lattice or an unknown value).  The restriction is unchanged.     */
#define TG_INTERP_LINEAR 0
#define TG_INTERP_CUBIC  1
int tg_op_set_interp(tg_op *op, int interp);

/* ------------------------------------------------------------------ phase 1: coarse solve
 * GMRES-DR(m,k) (Section 2.1) on the coarse operator (transpose = 1: on A_c^T, giving
 * left eigenvectors for the adjoint solve), right-hand side b_c = restrict(b_fine)
 * (b_fine: device, fine size).  Stops when the least-squares residual is
 * <= rtol ||b_c|| and the nev smallest harmonic Ritz pairs have residual
 * ||A y - theta y|| <= rtolev |theta| (checked at the end of each cycle, Example 1), or
 * after max_cycles.  Writes the coarse solution to xc_out (device, coarse size; may be
 * NULL) and creates *defl_out (may be NULL): the orthonormal basis of the final cycle's
 * k harmonic Ritz vectors (k+1 if k would split a complex pair), prolonged to the fine
 * grid, A Y formed on the fine grid (k products) and factored for the projection `proj`
 * (MinRes: CholQR2 of A Y; Galerkin: CholQR2 of Y, H = V^T A V and its LU).
 * precision TG_F64: the whole coarse phase in float64 (complex128 lattice).  TG_F32_IR
 * (real operators): the Arnoldi basis, the coarse operator products and the CGS2
 * orthogonalisation run in float32; the Hessenberg matrix, the restart step (least
 * squares, harmonic Ritz pairs, recombination matrices), ||b_c|| and the outputs (xc_out,
 * Y, A Y and its factors) are float64, and the handle also carries float32 copies for
 * float32 inner cycles.  The coarse solution is then accurate to about float32 rounding
 * times the coarse condition number (it only serves as the fine initial guess).
 * Each cycle is captured as a CUDA graph on the second use of its shape and replayed
 * (not while tg_profile_enable is on); results are identical to direct launches.
 * 1 <= k < m <= 128.  Synchronises `stream`.                                           */
int tg_coarse_gmresdr(tg_op *op, int transpose, const void *b_fine, int m, int k, int nev,
                      double rtolev, double rtol, int max_cycles, void *xc_out,
                      tg_defl **defl_out, int proj, int precision, tg_stats *stats,
                      void *stream);

/* A deflation handle from a caller-supplied fine basis Y (n x k, column-major, device,
 * float64 / complex128), e.g. a basis saved from an earlier run (the basis is reused
 * across right-hand sides, Section 4.1 Example 2, Figure 4.2).  Forms A Y (or A^T Y)
 * and factors it as in tg_coarse_gmresdr.  Y is copied.                                */
int tg_defl_from_basis(tg_op *op, int transpose, const void *Y, int k, int proj,
                       int precision, tg_defl **defl_out, void *stream);
int tg_destroy_defl(tg_defl *defl);

/* Deflation data for inspection or saving (float64 / complex128, column-major):
 *   what 0: Y (n x kk)   1: Q (MinRes) or V (Galerkin) (n x kk)
 *        2: A Y (n x kk) 3: R (MinRes, kk x kk upper triangular, A Y = Q R) or
 *                           H = V^H A V (Galerkin, kk x kk).
 * *kk_out receives the number of columns; dst may be NULL to query it.                */
int tg_defl_copy(const tg_defl *defl, int what, void *dst, int *kk_out, void *stream);

/* One projection (Section 2.2 box, step 2-4, or its MinRes variant), float64: x += Y d,
 * r -= A Y d with d minimising ||r - A Y d|| (MinRes) or V^H (r - A V d) = 0 (Galerkin).
 * x and r: device, fine size.                                                           */
int tg_project(const tg_op *op, const tg_defl *defl, void *x, void *r, void *stream);

/* ------------------------------------------------------------------ phase 3: fine solve
 * Restarted method with projection over defl between cycles (defl = NULL: no deflation,
 * the k = 0 case of Example 3).  method TG_BICGSTAB: BiCGStab(ncyc)-Proj(k), Section 4.1:
 * for icyc = 1..ncyc: project; rticyc = min((rtol ||b|| / ||r||)^(1/(ncyc-icyc+1)),
 * (||b|| / ||r||) rtol^(icyc/ncyc)); BiCGStab to rticyc (checked at half and full steps);
 * stop when ||r|| <= rtol ||b||.  If the ncyc scheduled cycles end above rtol (the paper's
 * box stops at icyc = ncyc and is silent on this case), later cycles aim at
 * rticyc = rtol ||b|| / ||r|| (the step-3b value at icyc = ncyc) until convergence or
 * max_mvps.  ncyc = 0 selects fixed-length restarting: cycles of at most restart_mvps
 * products (Example 2); with ncyc > 0, restart_mvps > 0 also caps every cycle.  method TG_GMRES: GMRES(m3)-Proj(k), Section
 * 2.2.  The true residual b - A x is recomputed in float64 at every restart.
 * precision TG_F32_IR: each cycle solves the correction equation in float32 (projection
 * included) and adds the correction to the float64 x (iterative refinement).  A cycle
 * whose correction does not lower the float64 residual (float32 rounding times the
 * condition number near 1) is undone and the solve finishes in float64 cycles
 * (stats.fp64_cycles counts them).  A BiCGStab cycle also stops when its residual
 * has grown 1e8-fold (divergence).
 * b, x: device, n x nrhs column-major (x: in x0, out solution).  Each right-hand side
 * is solved in turn; stats (host, may be NULL) must hold nrhs entries.
 * Returns TG_OK if every right-hand side converged, else the first failure status.
 * Synchronises `stream`.                                                               */
int tg_solve_proj(tg_op *op, const tg_defl *defl, int method, int precision,
                  const void *b, void *x, int nrhs, double rtol, int ncyc,
                  int restart_mvps, int m3, int64_t max_mvps, tg_stats *stats,
                  void *stream);

/* IDR(ncyc)-Proj(k) (Section 4.1: the box's step 3 runs "BiCGStab or IDR"; the paper's
 * IDR is van Gijzen and Sonneveld's biorthogonal IDR(s), default s = 4): the schedule of
 * tg_solve_proj (projection, rticyc, cycles past ncyc, true residual at every restart) with
 * cycles of IDR(s).  Each cycle starts from e = 0 with G = U = 0, M = I, omega = 1; omega
 * is the residual-minimising <t, r> / <t, t>, enlarged by kappa / |rho| when the cosine
 * |rho| = |<t, r>| / (||t|| ||r||) is below kappa (0.7 is the published default; 0 turns
 * the safeguard off).  Convergence (||r|| <= rticyc ||r_cycle_start||) and the product cap
 * are checked after every residual update.
 *   s   shadow-space dimension, 1..8 (and < n)
 *   P   device, n x s column-major (float64 / complex128): the shadow columns, linearly
 *       independent (random normal is the usual choice); the library orthonormalises them
 *       by CholQR2 (the QR factor with a positive-diagonal R) and uses the same space in
 *       every cycle.  TG_BAD_ARG when they are numerically dependent.
 * precision TG_F64 (float64 / complex128), or TG_F32_IR for the real operators: each
 * cycle solves the correction equation in float32 IDR(s) (the orthonormalised shadow space
 * rounded once to float32, a float32 projection with the handle's float32 copies, which
 * must then exist) with float64 refinement of x and of the true residual; a correction
 * that does not lower the float64 residual is undone and float64 IDR(s)-Proj cycles finish
 * (stats.fp64_cycles).  b and x are float64 in both forms.  Other arguments, stats and the
 * return value as for tg_solve_proj.  Synchronises `stream`.                             */
int tg_solve_idr(tg_op *op, const tg_defl *defl, int precision, const void *b, void *x, int nrhs,
                 double rtol, int ncyc, int restart_mvps, int s, const void *P, double kappa,
                 int64_t max_mvps, tg_stats *stats, void *stream);

/* ------------------------------------------------------------------ phase 2: improvement
 * Arnoldi-E improvement of the moved eigenvectors on the fine grid (Section 3 box and
 * Section 4.1 box, step 2; Example 7: "Arnoldi-E(150,100) ... with the 10 smallest
 * approximate eigenvectors used as starting vectors"; Example 8: "targeting only the
 * smallest five").  With k = the handle's kk:
 *   0. Rayleigh-Ritz on span(Y): the Ritz pairs of Y^H A Y, ordered like the harmonic
 *      Ritz values of tg_coarse_gmresdr (|theta|, Re, Im >= 0 first), k kept;
 *   cycle c = 0..cycles-1: S = span{u, A u, ..., A^(m-k) u} + span(Y), u the Ritz vector
 *      number (c mod nstart) of the previous Rayleigh-Ritz step (smallest first; its
 *      largest coefficient made real and positive, real problems take its real part),
 *      dimension m (u lies in span(Y): the dependent direction is dropped); Rayleigh-Ritz
 *      on S (the same ordering, k kept, k + 1 when a complex pair would split), Y <- an
 *      orthonormal real basis of the kept span;
 *   stop after `cycles`, or once the nev smallest pairs have ||A y - theta y|| <=
 *      rtolev |theta| (rtolev > 0).
 * The handle's basis is replaced by the improved one and A Y and its factorisation (and the
 * float32 copies of a TG_F32_IR handle) are rebuilt.  kk < m <= 256, 1 <= nstart <= kk.
 * theta_out (host, may be NULL): 2 kk doubles, the kept Ritz values (re, im) in order.
 * stats (host, may be NULL): cycles run, fine products (mvps), kk, pairs converged.
 * Synchronises `stream`.                                                                */
int tg_improve_defl(tg_op *op, tg_defl *defl, int m, int cycles, int nstart, int nev, double rtolev,
                    double *theta_out, tg_stats *stats, void *stream);

/* ------------------------------------------------------------------ adjoint (added form)
 * Not in the paper: the gradient of a loss L(x) through the solve A(kappa) x = b for
 * TG_VARK2D.  Solves A^T lambda = g with the same two-grid deflated BiCGStab using a
 * deflation handle built on A^T (tg_coarse_gmresdr with transpose = 1), then, if dkappa
 * is not NULL, writes dL/dkappa on the (N+2)^2 nodes:
 *   dkappa_p = -1/2 sum over faces f touching p of (lambda_a - lambda_b)(x_a - x_b)/h^2
 * (lambda = x = 0 on the boundary).  g, lambda, x: device, fine size float64;
 * lambda is also the initial guess (zero it for a cold start).                         */
int tg_adjoint_solve(tg_op *op, const tg_defl *defl_left, const void *g, void *lambda,
                     const void *x, void *dkappa, double rtol, int ncyc, int restart_mvps,
                     int precision, tg_stats *stats, void *stream);

/* dkappa from given x and lambda (the contraction step alone). */
int tg_kappa_gradient(const tg_op *op, const void *x, const void *lambda, void *dkappa,
                      void *stream);

/* ------------------------------------------------------------------ batched form (added)
 * Not in the paper: many independent 2D convection-diffusion instances (TG_CD2D, sizes Ns[i]
 * odd, convection betas[i]), each with nrhs = 8 right-hand sides sharing one deflation
 * basis (the paper reuses the basis across right-hand sides, Section 4.1, Example 2).
 * Right-hand sides and solutions are float64, concatenated by instance, each instance's
 * n_i x 8 block point-major: element (point j, column q) of instance i at
 * offset_i + j * 8 + q (tg_batch_layout gives offset_i and n_i).
 * tg_batch_setup: per instance, coarse GMRES-DR(m,k) on the restriction of its column 0,
 *   prolongation, A Y and CholQR2 with float32 copies (1 <= k <= 32); stats: count entries.
 * tg_batch_solve: per instance, float32-inner / float64-refinement BiCGStab(ncyc)-Proj(k)
 *   on the 8 columns together (one read of the basis serves all 8), each column with its
 *   own cycle tolerance and stopping test.  x holds the initial guesses.
 * Both phases advance all instances together in lock-step cycles, one kernel launch per
 *   phase for all of them (blocks of instance i take its points): tg_batch_setup runs the
 *   instances' coarse GMRES-DR cycles with one batched restart launch per cycle (m <= 62;
 *   larger m falls back to one instance per host thread), then prolongs and factors each
 *   basis on `threads` host threads; tg_batch_solve replays the 8-iteration BiCGStab
 *   sequence of all instances as one CUDA graph until every column of the cycle has
 *   finished.  The graph's blocks per instance are chosen on the first solve of a handle
 *   by timing the candidates 8, 16, 32, 64, 128 on the first cycle (tg_batch_tuning).
 *   A float32 correction that raises a column's float64 residual more than 4-fold is undone
 *   and that column's cycle cap halved; a column that no float32 cycle can advance finishes
 *   with float64 BiCGStab(-Proj) cycles on its instance's operator and basis
 *   (stats.fp64_cycles, per instance).
 *   Both calls wait for `stream` first and return when all work is done (they run on a
 *   private stream).  stats: count (setup) / count * 8 (solve) entries.
 * Returns TG_OK when every column converged, else the first failing status.           */
int tg_batch_create(tg_batch **out, int count, const int64_t *Ns, const double *betas, int nrhs,
                    void *stream);
int tg_batch_layout(const tg_batch *b, int i, int64_t *offset, int64_t *n);
int tg_batch_setup(tg_batch *b, const void *rhs, int m, int k, int nev, double rtolev, double rtol,
                   int max_cycles, int proj, int threads, tg_stats *stats, void *stream);
int tg_batch_solve(tg_batch *b, const void *rhs, void *x, double rtol, int ncyc, int restart_mvps,
                   int64_t max_mvps, int threads, tg_stats *stats, void *stream);
int tg_destroy_batch(tg_batch *b);
/* The autotuner's choice for the batched iteration graph: blocks per instance and its
 * time per iteration (microseconds, all instances and columns), and every candidate's
 * (ncand entries of cand_blocks / cand_us, at most 8; any pointer may be NULL).  Zero
 * blocks before the first tg_batch_solve of the handle.                               */
int tg_batch_tuning(const tg_batch *b, int *blocks_per_instance, double *us_per_iteration, int *ncand,
                    int *cand_blocks, double *cand_us);

/* ------------------------------------------------------------------ small dense step
 * The single-CTA float64 kernel of GMRES-DR's restart (Section 2.1), exposed for tests:
 * for an (m+1) x m upper-Hessenberg-plus-dense-leading-block Hbar (device, column-major,
 * leading dimension m+1), computes all harmonic Ritz values theta (eigenvalues of
 * H_m + |h_{m+1,m}|^2 f e_m^T, H_m^H f = e_m), orders them by |theta|, Re, Im >= 0 first,
 * keeps k (k+1 if a complex pair would split) and returns an orthonormal m x kk basis of
 * their span (real arithmetic for real Hbar; complex = 1 for complex128 Hbar).
 * theta_out: device, 2*m doubles (re, im) in the sorted order; basis_out: device, m x kk
 * (m x kk complex for complex = 1); eres_out: device, kk doubles, ||Hbar g - theta [g;0]||
 * for unit g; kk_out: host.                                                            */
int tg_harmonic_ritz(const void *Hbar, int m, int k, int complex_, void *theta_out,
                     void *basis_out, void *eres_out, int *kk_out, void *stream);

/* The same step as tg_harmonic_ritz (same arguments, same results), for callers that
 * cannot allocate device memory: callers that own all device memory through their own
 * allocator or a fixed pre-reserved pool (a cudaMalloc inside the library would bypass
 * the pool, or fail once it holds the memory), and latency-critical loops that cannot take
 * the device-wide synchronisation cudaMalloc / cudaFree may cause.  The paper has no
 * counterpart; this is a deployment variant.
 * No device memory is allocated or freed: all scratch lives in one fixed 2 MiB device
 * array of the library, reserved on every GPU that loads it and held until the process
 * exits.  Limit: m <= 128 (TG_BAD_ARG with a message beyond it).  The first call on a
 * device (with that device current) looks up the array's device address; make that first
 * call before any stream capture.  Every call uses the same array: two calls whose work
 * overlaps on the GPU (different streams, or several host threads) race and corrupt each
 * other's results; serialise them.  Synchronises `stream`.                             */
int tg_harmonic_ritz_noalloc(const void *Hbar, int m, int k, int complex_, void *theta_out,
                             void *basis_out, void *eres_out, int *kk_out, void *stream);

/* ------------------------------------------------------------------ instrumentation
 * Not part of the method: measurement hooks for benchmarks.
 * tg_profile_enable(1) starts recording a CUDA event pair around every kernel the
 * library launches (on the launch's stream), tagged with its kernel class and the
 * algorithmic bytes and float64-equivalent flops of that launch; tg_profile_enable(0)
 * stops recording.  tg_profile_read writes the per-class totals as a JSON object
 *   {"<class>": {"launches": L, "ms": T, "bytes": B, "flops": F}, ...}
 * into json (cap bytes; TG_BAD_ARG if too small); it waits for the recorded events.
 * tg_launch_count: number of kernels this process has launched through the library.
 * Not thread safe.                                                                    */
int tg_profile_enable(int on);
int tg_profile_read(char *json, int cap);
int64_t tg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TG_H */
