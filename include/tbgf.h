/*
 * tbgf: GB300 (sm_103a) library for the generalized shifted linear equations
 *
 *     (z S - H) x = b                                  (Eq. 2, Sec. 3)
 *
 * for many complex energies z and unit right-hand sides b = e_j, solved by a
 * shifted COCG (the first solver named in Sec. 3), and for the reduction of
 * the resulting Green's-function entries G_ij(z) = e_i^T (z S - H)^{-1} e_j to
 * local densities of states and density-matrix elements (the Green's-function
 * based quantities of Sec. 2).  H and S are the sparse real-symmetric
 * Hamiltonian and overlap of an atom-orbital (LCAO) basis, S positive definite
 * with unit diagonal (Sec. 2 Eq. 1, Sec. 8).
 *
 * Conventions for every entry point:
 *  - Plain C types only.  Complex numbers are two doubles (re, im), arrays of
 *    them are interleaved, row-major.
 *  - Array arguments are owned by the caller.  Unless an entry point says
 *    otherwise each array may live in host memory or in device memory of the
 *    current CUDA device; the library detects which (cudaPointerGetAttributes)
 *    and stages host arrays through its own device buffers, copying host
 *    outputs back before it returns.
 *  - Work is queued on the CUDA stream passed in (NULL = legacy default
 *    stream).  With device-resident outputs an entry point may return before
 *    the work finishes; synchronise the stream before reading them.  With any
 *    host-resident output it synchronises before returning.
 *  - Indices are 0-based.  Row indices are int64, block-column indices int32.
 *  - Every entry point returns an int status: 0 = success, negative = error
 *    (nothing useful was written), positive = warnings (bit mask, see below).
 *    Nothing throws across the boundary.  tb_status_string() names a status.
 */
#ifndef TBGF_H
#define TBGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define TB_OK 0
#define TB_ERR_ARG (-1)         /* an argument is invalid                           */
#define TB_ERR_CUDA (-2)        /* a CUDA call failed (see tb_last_error)           */
#define TB_ERR_ALLOC (-3)       /* device or host allocation failed                 */
#define TB_ERR_UNSUPPORTED (-4) /* a valid request this build does not implement    */
#define TB_ERR_SIZE (-5)        /* a size exceeds an internal limit                 */
#define TB_ERR_STRUCTURE (-6)   /* a matrix structure is malformed                  */

/* positive return values of shifted_cocg_solve: OR of these over columns */
#define TB_WARN_MAX_ITER 1
#define TB_WARN_BREAKDOWN 2
#define TB_WARN_NONFINITE 4

/* per-column status written by shifted_cocg_solve */
#define TB_COL_CONVERGED 0 /* every shift met the tolerance                     */
#define TB_COL_MAX_ITER 1  /* max_iter reached with some shift above tolerance  */
#define TB_COL_BREAKDOWN 2 /* rho_n = r^T S r or mu_n = p^T (z_s S - H) p is 0  */
#define TB_COL_NONFINITE 3 /* a recurrence scalar became inf or NaN             */

/* ------------------------------------------------------------- context */
typedef struct tb_ctx tb_ctx;

/* Create a context bound to the current CUDA device.  It owns the library's
 * device workspace (grown on demand, freed by tb_ctx_destroy).  One context
 * must not be used from two host threads at once. */
int tb_ctx_create(tb_ctx **out);
int tb_ctx_destroy(tb_ctx *ctx);
const char *tb_status_string(int status);
/* The message of the last failure recorded in ctx (never NULL). */
const char *tb_last_error(const tb_ctx *ctx);
/* Library version, e.g. 10100 for 1.1.0. */
int tb_version(void);

/* ------------------------------------------------------ system builder */
/* Synthetic tight-binding systems with the structure Sec. 8 states for the
 * LCAO matrices: H, S real symmetric, S_ii = 1, |S_ij| < 1, S positive
 * definite (checked by Gershgorin dominance), nearest-neighbour sparsity.   */
#define TB_LATTICE_SC_PERIODIC 0 /* L^3 simple cubic, periodic, 6 NN; L >= 3    */
#define TB_LATTICE_FCC_CLUSTER 1 /* n_sites FCC sites nearest the origin, open  */

#define TB_ONSITE_UNIFORM 0     /* u * I, u ~ U[onsite_lo, onsite_hi] per atom       */
#define TB_ONSITE_DIAG_NORMAL 1 /* diag(onsite_diag) + (N + N^T)/2, N ~ N(0,sigma)   */
#define TB_HOP_CONST 0          /* hop_t * I on every NN pair                        */
#define TB_HOP_NORMAL 1         /* X ~ N(0, hop_sigma) per pair, X_ji = X_ij^T       */
#define TB_S_IDENTITY 0         /* S = I (no S matrix is produced)                   */
#define TB_S_NORMAL 1           /* S = I + symmetric NN blocks N(0, s_param)         */
#define TB_S_CONST 2            /* S = I + s_param * I on every NN pair              */

typedef struct {
    int32_t lattice;
    int32_t L;              /* SC edge length                                      */
    int64_t n_sites;        /* FCC: sites kept before vacancies and slab           */
    int32_t bdim;           /* orbitals per atom = block edge, 1..16               */
    int32_t onsite_mode;
    double onsite_lo, onsite_hi, onsite_sigma;
    double onsite_diag[16];
    int32_t hop_mode;
    double hop_t, hop_sigma;
    int32_t s_mode;
    double s_param;
    double vacancy_frac;    /* FCC only: fraction of sites removed                 */
    int32_t slab;           /* FCC only: remove sites above a random z cut         */
    double subst_frac;      /* fraction of atoms whose onsite block gets + shift*I */
    double subst_shift;
} tb_system_spec;

/* Block-sparse row matrix with bdim x bdim blocks.
 *   row_ptr int64[n_brows+1], col_idx int32[nnzb] ascending within each block
 *   row with the diagonal block present, val double[nnzb*bdim*bdim] with each
 *   block row-major.  bdim = 1 is plain CSR. */
typedef struct {
    int64_t n_brows;
    int32_t bdim;
    int64_t nnzb;
    int64_t *row_ptr;
    int32_t *col_idx;
    double *val;
} tb_bsr;

/* Build H (and S unless s_mode is TB_S_IDENTITY) for `spec` from `seed`.
 * Host memory only.  Two phases: with H->row_ptr == NULL only n_brows, bdim
 * and nnzb of H (and S) are filled; then call again with row_ptr, col_idx and
 * val allocated to those sizes.  S may be NULL when s_mode is TB_S_IDENTITY.
 * Random values come from Philox4x32-10 keyed by the seed, counter
 * (index, stream); *overlap_seed (optional) receives the seed the overlap
 * draws used (seed + k when the first k draws failed the dominance check).
 * Integer structure is a deterministic function of spec (bit-exact).
 * Errors: TB_ERR_ARG for an invalid spec (e.g. L < 3), TB_ERR_SIZE when
 * the structure does not fit int32 block-column indices. */
int tb_build_bsr(const tb_system_spec *spec, uint64_t seed, tb_bsr *H, tb_bsr *S,
                 uint64_t *overlap_seed);
/* tb_build_bsr for bdim = 1 (scalar CSR); TB_ERR_ARG if spec->bdim != 1. */
int tb_build_csr(const tb_system_spec *spec, uint64_t seed, tb_bsr *H, tb_bsr *S,
                 uint64_t *overlap_seed);

/* ---------------------------------------------------------- sparse product */
#define TB_PREC_FP64 0  /* all vectors and arithmetic in FP64                      */
#define TB_PREC_MIXED 1 /* FP32 vectors, SpMM and updates with FP32 accumulation;
                           FP64 recurrence scalars, dot products, convergence
                           tests, projected solutions and reductions           */
#define TB_PREC_DF64 2  /* vectors, SpMM and updates in double-float (hi + lo
                           FP32 pairs, ~48 bits) on the FP32 pipes; FP64
                           scalars, projections and reductions as above.  With
                           S, the inner solve S r = rt is iterative refinement:
                           the residual t = rt - S y is kept in df, FP32 CG
                           sweeps solve S c = t (FP32 vectors, FP32 values of S,
                           two-float dot products) and each sweep's c is added
                           to y in df, t -= S c with a df product (an FP32 one
                           once every ||t|| <= 5e4 inner_tol ||rt||, where its
                           error stays below inner_tol ||rt|| / 20), until
                           ||t|| <= inner_tol ||rt||                            */

/* Y = A X for a real BSR matrix A (n = n_brows*bdim rows) and a complex panel
 * X of ncols columns: X, Y complex double [n][ncols] (row-major, interleaved).
 * precision TB_PREC_MIXED rounds A and X to FP32 and accumulates in FP32;
 * TB_PREC_DF64 computes in double-float.
 * ncols in {1..64}.  The sparse product shared by every shift in each COCG
 * iteration (Sec. 3); exposed for measurement and tests. */
int tb_bsr_spmm(tb_ctx *ctx, const tb_bsr *A, const double *X, int32_t ncols, double *Y,
                int32_t precision, void *stream);

/* Time the block-sparse product kernel of tb_bsr_spmm alone: the matrix is
 * converted and a panel of width panel(ncols) in the working precision is
 * filled once with test values in the library's workspace; then one untimed
 * launch and `reps` launches, each between CUDA events on `stream` after a
 * 256 MB write that evicts the operands from L2 (cold-L2 time).
 * *ms_per_launch = average milliseconds per product (the measurement behind
 * the SpMM bandwidth figure; Sec. 3's shared product).  Allocates only the
 * context's workspace; TB_ERR_ARG / TB_ERR_UNSUPPORTED as tb_bsr_spmm. */
int tb_bsr_spmm_profile(tb_ctx *ctx, const tb_bsr *A, int32_t ncols, int32_t precision, int32_t reps,
                        void *stream, double *ms_per_launch);

/* ------------------------------------------------------ shifted COCG solve */
typedef struct {
    double tol;          /* stop a shift when ||b - (zS-H)x|| <= tol ||b|| (recurrence
                            residual), default 1e-10                              */
    int32_t max_iter;    /* outer iterations, default 100000                        */
    int32_t precision;   /* TB_PREC_FP64 (default), TB_PREC_MIXED or TB_PREC_DF64 */
    int32_t panel_w;     /* columns solved together; 0 = autotuned: with >= 128
                            columns the library times one iteration of its
                            kernels for each width 8..64 and 2 or 3 CTAs per SM
                            and keeps the fastest per column (cached per shape
                            in the context); fewer columns use a heuristic     */
    int32_t seed_shift;  /* index of the seed shift; -1 = median Re z (default)    */
    double inner_tol;    /* S != I: relative tolerance ||S r - rt|| <= inner_tol ||rt||
                            of the inner solve on S; 0 = max(1e-3 tol, 1e-13) FP64,
                            max(1e-3 tol, 1e-7) mixed, max(1e-5 tol, 1e-12) DF64   */
    int32_t inner_max;   /* S != I: inner iterations per outer iteration (DF64: per
                            FP32 sweep), 0 = 40                                   */
    int32_t ctas_per_sm; /* resident CTAs per SM for the panel kernels, 0 = 3;
                            the FP32 sweep update of the DF64 refinement runs
                            one fewer (at least 1)                              */
    void *stream;        /* cudaStream_t to queue work on                         */
    int32_t solver;      /* TB_SOLVER_COCG (default) or TB_SOLVER_QMR                */
    int64_t *stats;      /* optional host array [4]: outer iterations, inner
                            iterations, and (DF64 with S) refinement passes and
                            of those the ones that took S c in FP32 (written
                            before returning)                                     */
} tb_solve_opts;

/* Solvers of Sec. 3 for Eq. 2:
 * TB_SOLVER_COCG  generalized shifted COCG: each shift stops when its residual
 *                 ||rt|| / |pi^m| <= tol (resid is that residual);
 * TB_SOLVER_QMR   generalized shifted QMR: the quasi-minimal residual iterates
 *                 of the same Krylov space, obtained from the COCG iterates by
 *                 QMR smoothing (1/tau_n^2 = 1/tau_{n-1}^2 + 1/omega_n^2,
 *                 xq_n = xq_{n-1} + (tau_n / omega_n)^2 (x_n - xq_{n-1}), omega_n =
 *                 sqrt|r_n^T S r_n| / |pi^m_n|, the quasi-norm of the shift's COCG
 *                 residual; equal in exact arithmetic to QMR on the unconjugated
 *                 Lanczos process); a shift stops when its quasi-residual
 *                 tau_n / tau_0 <= tol (resid is that ratio).  No df64 restarts. */
#define TB_SOLVER_COCG 0
#define TB_SOLVER_QMR 1

/* Fill `opts` with the defaults above. */
void tb_solve_opts_default(tb_solve_opts *opts);

/* Solve (z_m S - H) x = e_j for every shift z_m (m < n_z) and every column
 * j = rhs_rows[c] (c < n_rhs), keeping x on the rows asked for:
 *
 *   G[(out_row_ptr[c] + k) * n_z + m] = e_i^T (z_m S - H)^{-1} e_j,
 *       i = out_rows[out_row_ptr[c] + k],  0 <= k < out_row_ptr[c+1]-out_row_ptr[c]
 *
 * H and S (S = NULL means S = I) are BSR with the same bdim and n_brows, their
 * arrays in device memory or host memory (staged).  z: complex [n_z].
 * Outputs: G complex [out_row_ptr[n_rhs]][n_z]; iters int32[n_rhs] (outer
 * iterations run); resid double[n_rhs][n_z] (final recurrence residual
 * ||rt_n|| / |pi^m_n| relative to ||b||); status int32[n_rhs] (TB_COL_*).
 * Method: one seed COCG per column in the S-bilinear form <u,v> = u^T S v
 * (Sec. 3's generalized shifted COCG): p = r + beta p, u = (z_s S - H) p,
 * alpha = r^T S r / p^T u, S r <- S r - alpha u, r = S^-1 (S r) by an inner CG;
 * every shift z_m follows through collinear residuals r_m = r / pi_m, with
 * pi_{n+1} = (1 + alpha_n (z_m - z_s)) pi_n + (alpha_n beta_{n-1} /
 * alpha_{n-1}) (pi_n - pi_{n-1}) and x_m += (alpha_n pi_n / pi_{n+1}) p_m
 * kept on the requested rows only; columns batched into panels so that one block
 * sparse product per iteration serves every column and every shift.  When
 * every diagonal block of S is the identity (orthonormal orbitals on each
 * site; checked on the device per call) the S products add those blocks'
 * operand instead of multiplying by them, with the same result bits.
 * TB_PREC_DF64 restart: once a column's seed residual ||S r|| is below 1e-10,
 * its worst unconverged shift residual is checked every 512 outer
 * iterations; if it fell by less than 1 % since the previous check, the
 * column restarts with that shift as its new seed: converged shifts keep
 * their results, every unconverged shift starts again from x = 0, and the
 * restart itself takes one outer iteration.  At most two restarts per
 * column; iters counts every iteration run, before and after restarts.
 * Returns TB_OK, or a positive OR of TB_WARN_* when some column did not
 * converge, or a negative error. */
int shifted_cocg_solve(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z,
                       int32_t n_z, const int64_t *rhs_rows, int64_t n_rhs,
                       const int64_t *out_row_ptr, const int64_t *out_rows,
                       const tb_solve_opts *opts, double *G, int32_t *iters, double *resid,
                       int32_t *status);

/* Times the kernels of one solver iteration (the Sec. 3 step sequence) for
 * the first panel of the given problem (same arguments and options as
 * shifted_cocg_solve, no outputs).  After the panel is initialised, the
 * sequence  A, B, [IC_A, IC_B], C  (the bracketed pair and C only when
 * S != NULL) is launched `reps` times as ordinary launches on opts->stream,
 * each kernel bracketed by CUDA events (with S, a first inner pair runs
 * untimed before the timed one, so IC_A/IC_B are timed in their steady
 * state with a previous search direction).  ms[k] (k < 8) receives the average
 * milliseconds per launch of kernel k: 0 A (H product, shifted steps),
 * 1 B (residual update; with S also the S product of the inner start),
 * 2 IC_A (S product of the inner CG), 3 IC_B (inner CG update), 4 C (rho),
 * 5 R (DF64 with S: refinement pass with S c in df), 6 R with S c in FP32;
 * unused entries are 0.  These are the kernels the solve's graph runs. */
int shifted_cocg_profile(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z,
                         const int64_t *rhs_rows, int64_t n_rhs, const int64_t *out_row_ptr,
                         const int64_t *out_rows, const tb_solve_opts *opts, int32_t reps, double *ms);

/* ------------------------------------------------ local subspaces (order N) */
/* Hop-shell subspaces (Sec. 2: order-N locality): for column c the atoms
 * within radii[c] hops of the atom owning row rhs_rows[c] in the
 * nearest-neighbour graph of A's block pattern, ascending.  Host memory only.
 * Two phases: with sub_atoms == NULL only sub_ptr[0..n_rhs] (CSR offsets) is
 * written; then call again with sub_atoms sized sub_ptr[n_rhs].  radii in
 * 0..64.  Errors: TB_ERR_ARG (ranges, or sub_ptr changed between the calls),
 * TB_ERR_STRUCTURE (column index out of range). */
int tb_local_subspaces(const tb_bsr *A, const int64_t *rhs_rows, const int32_t *radii, int64_t n_rhs,
                       int64_t *sub_ptr, int32_t *sub_atoms);

/* shifted_cocg_solve on truncated problems: column c solves
 * (z_m S_OO - H_OO) x = e_j on the principal submatrices over the block rows
 * O_c = sub_atoms[sub_ptr[c] .. sub_ptr[c+1]) (ascending, containing the atom
 * of j = rhs_rows[c]; at most 32767 atoms) and keeps the rows out_rows (rows
 * outside O_c give 0).  S (NULL = I) must have H's block pattern.  `order`
 * (optional, a permutation of 0..n_rhs-1) is the order in which columns are
 * taken from the device work queue: each CTA solves one column at a time in
 * shared memory and takes the next as soon as it finishes.  When the vectors
 * of the largest subspace do not fit one CTA's shared memory they are placed
 * in a device workspace of (grid x vectors) instead (read through L2).
 * opts->panel_w is ignored; n_z <= 1024.  Outputs and status as
 * shifted_cocg_solve.  TB_ERR_SIZE when even the per-shift states and the
 * local block structure do not fit shared memory. */
int shifted_cocg_solve_local(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const double *z, int32_t n_z,
                             const int64_t *rhs_rows, int64_t n_rhs, const int64_t *sub_ptr,
                             const int32_t *sub_atoms, const int64_t *out_row_ptr, const int64_t *out_rows,
                             const int64_t *order, const tb_solve_opts *opts, double *G, int32_t *iters,
                             double *resid, int32_t *status);

/* ------------------------------------------------- learned scheduler inputs */
/* 32 FP32 numbers per column describing its local problem (the paper has no
 * learned component; the scheduler's predictor reads these).  Column c uses
 * the subspace sub_atoms[sub_ptr[c]..sub_ptr[c+1]) of radius radii[c] around
 * the atom of rhs_rows[c] (as tb_local_subspaces gives them).  Layout of
 * out[c*32 + q]: 0 R/5; 1 log(n_atoms)/log(1000); 2..6 atoms at hop distance
 * 1..5 / 100; 7 nearest neighbours of the atom / 12; 8 H_jj; 9..16
 * sign(m_k)|m_k|^(1/k), m_k = e_j^T (H_OO - H_jj)^k e_j, k = 2..9; 17
 * sum_{i!=j} S_ij^2 (0 if S = NULL); 18..21 mean, std, min, max of diag(H_OO);
 * 22 sum_{i!=j} H_ij^2 in row j of H_OO; 23 mean Frobenius norm of the atom's
 * in-subspace neighbour blocks; 24 rows / 1000; 25 fraction of atoms at the
 * largest hop distance; 26..31 zero.  Moments in FP64.  S (optional) must
 * have H's block pattern.  TB_ERR_SIZE when a subspace does not fit one CTA's
 * shared memory. */
int tb_descriptors(tb_ctx *ctx, const tb_bsr *H, const tb_bsr *S, const int64_t *rhs_rows, const int32_t *radii,
                   int64_t n_rhs, const int64_t *sub_ptr, const int32_t *sub_atoms, float *out, void *stream);

/* Iteration-count predictor: MLP 32 -> 64 -> 64 -> 1 with tanh hidden layers,
 * FP16 weights in the forward pass, FP32 accumulation and FP32 master weights.
 * params: mlp_param_count() floats, W1[64][32] | b1[64] | W2[64][64] | b2[64] |
 * w3[64] | b3.  Loss: mean squared error.  Arrays: X float[n][32], y float[n]. */
int mlp_param_count(void);
/* Gradient of the batch loss at params (FP16-rounded forward weights), and the
 * loss (optional). */
int mlp_grad(tb_ctx *ctx, const float *params, const float *X, const float *y, int64_t n, float *grad,
             double *loss, void *stream);
/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on minibatches of
 * `batch` consecutive samples, `epochs` passes in the given sample order.
 * params: initial weights in, trained FP32 master weights out.  loss_hist
 * (optional, double[epochs]): full-data loss after each epoch. */
int mlp_train(tb_ctx *ctx, const float *X, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
              float *params, double *loss_hist, void *stream);
/* pred[i] = MLP(X[i]). */
int mlp_predict(tb_ctx *ctx, const float *params, const float *X, int64_t n, float *pred, void *stream);

/* ----------------------------------------------- Green's function -> LDOS, DM */
/* From the output of shifted_cocg_solve (same rhs/out-row layout):
 *   ldos[c*n_z + m] = -(1/pi) Im sum_k G_{i_k j}(z_m) S_{i_k j}   (Mulliken form;
 *                     S = NULL: -(1/pi) Im G_jj(z_m), row j must be kept)
 *   dm[out_row_ptr[c] + k] = -(1/pi) Im sum_m w[m] f(Re z_m) G_{i_k j}(z_m)
 * with f the Fermi-Dirac occupation at (mu, kT), kT = 0 a step with
 * f(mu) = 1/2, and w the quadrature weights (double[n_z]).  Either of ldos and
 * dm may be NULL.  All reductions in FP64.  Sec. 2 (DOS and Green's-function
 * analysis); the formulas are the standard ones, the paper prints none.
 * Errors: TB_ERR_ARG when S = NULL and a column does not keep its own row. */
int gf_reduce_ldos_dm(tb_ctx *ctx, const double *G, int32_t n_z, const double *z,
                      const double *w, double mu, double kT, const int64_t *rhs_rows,
                      int64_t n_rhs, const int64_t *out_row_ptr, const int64_t *out_rows,
                      const tb_bsr *S, double *ldos, double *dm, void *stream);

/* ------------------------------------------------- no-allocation variant */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot let a library allocate device memory (a pre-reserved memory arena
 * owns every allocation, a latency-critical loop must not hit the device
 * synchronisation of cudaFree, an embedding host forbids allocation after
 * start-up).  Same result as gf_reduce_ldos_dm, but it calls no cudaMalloc,
 * cudaFree or allocating routine: its scratch (one weight per kept entry and
 * four check flags) is a static device array of TB_REDUCE_STATIC_MAX_ENTRIES
 * + 32 doubles that every GPU loading the library holds until exit.
 *  - n_out (the number of kept entries) must be <= TB_REDUCE_STATIC_MAX_ENTRIES
 *    (else TB_ERR_SIZE, nothing queued);
 *  - every array (G, z, w, rhs_rows, out_row_ptr, out_rows, S's arrays, ldos,
 *    dm) must be device (or managed) memory of the current device (else
 *    TB_ERR_ARG);
 *  - each call first checks its index arrays on the device and synchronises
 *    the stream once to read the result; nothing is written to ldos or dm
 *    unless out_row_ptr starts at 0, is monotone and ends at n_out (else
 *    TB_ERR_SIZE), every row and rhs row lies inside S (else TB_ERR_ARG), S's
 *    structure is well formed (else TB_ERR_STRUCTURE) and, with S = NULL and
 *    ldos requested, every column keeps its own row (else TB_ERR_ARG);
 *  - the first call on a device looks up the scratch address
 *    (cudaGetSymbolAddress) with that device current; make it before any
 *    stream capture;
 *  - all calls share the scratch: calls whose GPU work overlaps (other
 *    streams or host threads) race; calls on one stream are ordered. */
#define TB_REDUCE_STATIC_MAX_ENTRIES 524288
int gf_reduce_ldos_dm_static(tb_ctx *ctx, const double *G, int32_t n_z, const double *z, const double *w,
                             double mu, double kT, const int64_t *rhs_rows, int64_t n_rhs,
                             const int64_t *out_row_ptr, int64_t n_out, const int64_t *out_rows,
                             const tb_bsr *S, double *ldos, double *dm, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TBGF_H */
