/*
 * tssvd.h - C ABI of the GB300 (sm_103a) library for the Gram-based
 * tall-skinny SVD and the randomized low-rank SVD of
 *   H. Li, Y. Kluger, M. Tygert, "Randomized algorithms for distributed
 *   computation of principal component analysis and singular value
 *   decomposition", arXiv:1612.08709.
 *
 * Conventions (all entry points):
 *  - Every matrix pointer is a DEVICE pointer owned by the caller.  The
 *    library never frees or retains caller memory.
 *  - Row-major storage with an explicit leading dimension for the input A
 *    (lda >= n elements).  Outputs are dense row-major: U is m x n
 *    (leading dimension n), S has n entries, V is n x n with column j the
 *    j-th right singular vector.  Singular values are in decreasing order.
 *  - Signs: each right singular vector is flipped so that its entry of
 *    largest magnitude (lowest index on ties) is positive; the matching
 *    left singular vector is flipped with it.
 *  - Work is queued on opts->stream (a cudaStream_t; NULL = the legacy
 *    default stream).  Each call returns only after that stream has
 *    finished the call's work, because the status code is read back from
 *    the device; output buffers are then complete.
 *  - Scratch memory: opts->workspace of opts->workspace_bytes bytes (query
 *    the size with the *_workspace_size functions).  If workspace is NULL
 *    the library uses an internal per-device buffer that it grows on demand
 *    with cudaMalloc and keeps until process exit; calls that use the
 *    internal buffer are serialised by a lock.
 *  - Return value: TSSVD_OK (0); a positive status below (results are
 *    still written); or -i when argument i (1-based) is invalid, in which
 *    case nothing is written and nothing is queued.
 */
#ifndef TSSVD_H
#define TSSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSSVD_OK 0
#define TSSVD_ENOCONV 1  /* a Jacobi solve used max_sweeps sweeps without converging */
#define TSSVD_RANKDEF 2  /* numerical rank r < n: S[r..], U and V columns r.. are 0 */
#define TSSVD_ETIMEOUT 3 /* a bounded device-side wait expired; results undefined */
#define TSSVD_ECUDA 4    /* a CUDA runtime call failed; results undefined */
#define TSSVD_ENOMEM 5   /* workspace too small, or the internal one could not grow */
#define TSSVD_ECOMM 6    /* the caller's all-reduce (tssvd_comm) reported a failure */

/* Arithmetic of the tall products (the passes over the m rows). */
typedef enum {
    /* Plain FP64: every tall product in FP64 fused multiply-add. */
    TSSVD_FP64 = 0,
    /* Mixed: the first pass's products (Gram of A and A V~) run on the
     * tcgen05 tensor cores with BF16x3 split operands and FP32 accumulation
     * drained to FP64; the products of the later orthonormalisation
     * pass(es) and the final U are FP64-accurate (the digit products of
     * TSSVD_FP64_TC); eigensolves and all n x n work stay FP64.  Two bf16
     * terms per value (about 16 significant bits), three term products per
     * product.  n <= 256.  Singular values to about 1e-6 of the largest.
     * With passes = 2, U is orthonormal to 1e-12 for condition numbers up
     * to about 1e5 (measured 1.4e-12 at 1e6, 6.8e-12 at 1e8: the first
     * pass leaves Y too ill-conditioned for one more pass to repair);
     * passes = 3 adds a pass that brings it back under 1e-12. */
    TSSVD_BF16X3 = 1,
    /* As TSSVD_BF16X3 with three bf16 terms per value (about 24 significant
     * bits, the accuracy of FP32 inputs) and six term products. n <= 256.
     * With passes = 2, U orthonormal to 1e-12 for condition numbers up to
     * about 1e5 (1.9e-12 at 1e6, 2.7e-9 at 1e8); passes = 3 as above. */
    TSSVD_BF16X6 = 2,
    /* FP64-accurate products on the tensor cores: every tall product of
     * both passes is emulated with seven 7-bit integer digits per value
     * (exact in bf16), exact per-level FP32 accumulation in tensor memory
     * and double-FP32 accumulation of the level sums, so the results carry
     * about 48 significant bits; the n x n work stays FP64.  Any n. */
    TSSVD_FP64_TC = 3,
    /* Batched calls only: for every (m, n) size class the library times
     * TSSVD_FP64 and TSSVD_FP64_TC once (both FP64-accurate) and keeps the
     * faster for that class for the rest of the process. */
    TSSVD_AUTO = 4
} tssvd_mode;

typedef struct {
    /* 1 = single orthonormalisation (Algorithm 3); 2 = double (Algorithm 4);
     * 3 = Algorithm 4 with its second pass (Gram of Y, eigendecomposition,
     * Q = Y W T^-1, R <- T W^T R) run once more on Q, an opt-in repair for
     * first passes too rough for one repair (the BF16-split modes at high
     * condition numbers); it costs one more Gram, eigensolve and tall
     * product, and an m x n double buffer in TSSVD_FP64 mode.  The TSQR
     * methods (ts_svd_tsqr, lowrank_svd_tsqr) take 1 or 2. */
    int passes;
    /* MaxEntry column scaling (passes >= 2 only): column j of A is divided by
     * the smallest power of two >= max_i |A_ij| before the Gram matrix is
     * formed, and the scaling is folded back into the small SVD. */
    int scale;
    /* Discard threshold: a column whose explicit norm is below
     * drop_tol * (largest norm) is dropped (Algorithms 3 and 4, discard
     * steps).  Default sqrt(1e-11), the square root of the paper's example
     * working precision (Remark "working"). */
    double drop_tol;
    int mode;       /* tssvd_mode */
    int max_sweeps; /* Jacobi sweep cap per eigen/SVD solve (default 50) */
    void *stream;   /* cudaStream_t */
    void *workspace;
    size_t workspace_bytes;
    /* ---- written by the call ---- */
    int64_t out_rank; /* number of nonzero singular values returned */
    /* Jacobi sweeps: [0] the first eigensolve (of A^T A, D-scaled; with
     * passes = 2, n <= 2048 and an FP64-accurate mode, the one-sided sweeps
     * on its pivoted Cholesky factor), [1] eig of Y^T Y, [2] SVD of R;
     * for 128 < n <= 2048 the one-sided solves ([0] and [2]; [1] too for
     * n > 256) start with an FP32 phase, and [0..2] count their FP64 sweeps
     * while [3] holds the FP32 sweeps of all such solves, summed (0 when
     * none ran); with passes = 3, [1] is the third pass's eigensolve */
    int sweeps[4];
    int ranks[2];     /* ranks kept by the first and second discard steps */
} tssvd_opts;

/* Fills *opts with the defaults: passes 2, scale 1, drop_tol sqrt(1e-11),
 * mode TSSVD_FP64, max_sweeps 50, default stream, internal workspace. */
void tssvd_default_opts(tssvd_opts *opts);

/* Human-readable text for a status code (static storage). */
const char *tssvd_status_string(int status);

/* Bytes of workspace ts_svd / ts_svd_f32 need for an m x n problem with
 * these options (elem_bytes = 8 for ts_svd, 4 for ts_svd_f32). */
size_t ts_svd_workspace_size(int64_t m, int64_t n, int elem_bytes, const tssvd_opts *opts);

/*
 * Thin SVD A = U diag(S) V^T of a tall-skinny A (m x n, m >= n >= 1).
 * passes = 2: Algorithm 4 (Gram of A, eigendecomposition, Y~ = A V~,
 * explicit column norms (Remark "normalizing"), discard, second Gram pass
 * on Y, R = T W^T S~ V~^T, SVD of R, U = Q P).  passes = 1: Algorithm 3.
 * The eigendecompositions and the SVD of R are Jacobi methods; the first
 * eigensolve of Algorithm 4 is accurate to the rounding already in the
 * Gram matrix (the second pass repairs the rest): for n <= 2048 in the
 * FP64-accurate modes it is a pivoted Cholesky factorization followed by
 * one-sided Jacobi on the factor, otherwise Gram-form Jacobi with a
 * normwise floor.  For 128 < n <= 2048 the one-sided solves (the first
 * eigensolve and the SVD of R; for n > 256 the second eigensolve too, on
 * the pivoted Cholesky factor of Y^T Y) run an FP32 phase first to pick
 * the starting basis, then converge in FP64 (FP64 results either way).
 *   A   [in]  m x n, row-major, leading dimension lda >= n; not modified.
 *   U   [out] m x n, row-major (leading dimension n).
 *   S   [out] n.
 *   V   [out] n x n, row-major; column j = right singular vector j.
 *   opts[in/out] options; out_rank, sweeps and ranks are written.
 * Errors: -1 A NULL, -2 m < n or m < 1, -3 n < 1, -4 lda < n, -5 U NULL,
 * -6 S NULL, -7 V NULL, -8 opts NULL or invalid field.
 */
int ts_svd(const double *A, int64_t m, int64_t n, int64_t lda, double *U, double *S,
           double *V, tssvd_opts *opts);

/*
 * ts_svd on host buffers (Algorithm 4 or 3 as opts->passes says): A (m x n,
 * row-major, lda), U (m x n, leading dimension n), S (n), V (n x n) are in
 * host memory; the call copies A to the device, runs the TS-SVD there and
 * copies the results back, then returns (the copies are ordered after the
 * work already queued on opts->stream).  A is copied in row chunks (about
 * 256 MB, at most 64) on a copy stream of the library's; with
 * TSSVD_FP64_TC and passes >= 2 the first pass's column maxima and Gram
 * partials start on each chunk as it lands (Section 2's per-partition
 * Gram matrices, summed), and U goes back in the same chunks while the
 * next chunk's product runs.  Other modes copy, compute and copy in turn.
 * The overlap needs page-locked host buffers (cudaHostAlloc or
 * cudaHostRegister); pageable ones work, with the copies serialised.  The
 * workspace (opts->workspace, or the internal one) also holds device
 * copies of A and U: ts_svd_host_workspace_size.  Host-buffer calls on one
 * device share the copy streams and take turns.  Status and errors as
 * ts_svd.
 */
size_t ts_svd_host_workspace_size(int64_t m, int64_t n, const tssvd_opts *opts);
int ts_svd_host(const double *A, int64_t m, int64_t n, int64_t lda, double *U, double *S,
                double *V, tssvd_opts *opts);

/* As ts_svd for FP32 storage: A, U, S, V are float.  The n x n
 * eigensolves and small SVD run in FP64; tall products as opts->mode says
 * (FP64 arithmetic on the FP32 data, or BF16x3 on the tensor cores). */
int ts_svd_f32(const float *A, int64_t m, int64_t n, int64_t lda, float *U, float *S,
               float *V, tssvd_opts *opts);

/*
 * Row-sharded calls (several GPUs, one process each).  The rows of A are
 * split over the ranks; each rank holds its row block.  The exchange steps
 * of the method are all-reductions of small arrays, made through the
 * caller's collective:
 *   allreduce(buf, count, dtype, op, stream, ctx)
 * reduces `count` elements of the DEVICE array buf over all ranks in place
 * (dtype TSSVD_DT_F64: double, op TSSVD_OP_SUM; dtype TSSVD_DT_U64:
 * unsigned 64-bit, op TSSVD_OP_MAX), ordered on `stream` (a cudaStream_t)
 * like the library's own kernels, and returns 0 on success.  Every rank
 * must receive the same bits (the n x n solves are then repeated
 * identically on every rank, with no further exchange).  A NCCL all-reduce
 * on the stream meets this.  rank and size describe the caller's group
 * (rank in [0, size)).
 */
#define TSSVD_DT_F64 0
#define TSSVD_DT_U64 1
#define TSSVD_OP_SUM 0
#define TSSVD_OP_MAX 1
typedef int (*tssvd_allreduce_fn)(void *buf, int64_t count, int dtype, int op, void *stream,
                                  void *ctx);
typedef struct {
    tssvd_allreduce_fn allreduce;
    void *ctx;
    int rank;
    int size;
} tssvd_comm;

/*
 * ts_svd on a row-sharded A: Algorithm 4 (opts->passes = 2) or 3
 * (passes = 1) where each rank holds rows of A (A_local, m_local x n,
 * lda), in the form of the paper's Section 2 aggregation of per-partition
 * Gram matrices: each Gram matrix is formed from the local rows and summed
 * over the ranks (one all-reduce of n x n doubles per Gram matrix); the
 * MaxEntry column maxima (one all-reduce of n words, maximum) and every
 * explicit column norm (one all-reduce of n sums of squares per norm step)
 * likewise; the eigendecompositions, the discards and the small SVD then
 * run on every rank on identical data, and the tall products stay local.
 *   A       [in]  m_local x n, row-major, lda >= n (device).
 *   U       [out] the rank's m_local rows of U (m_local x n, leading
 *                 dimension n).
 *   S, V    [out] n and n x n, identical on every rank.
 *   comm    [in]  the collective (a NULL allreduce means a single rank).
 *   opts    as for ts_svd (workspace: ts_svd_workspace_size(m_local, ...)).
 * m_local >= n on every rank.  Returns as ts_svd, or TSSVD_ECOMM when the
 * all-reduce failed (results undefined).
 * Errors: -1 A, -2 m_local < n, -3 n, -4 lda, -5 U, -6 S, -7 V, -8 comm
 * (NULL, or rank / size out of range), -9 opts.
 */
int ts_svd_rowshard(const double *A, int64_t m_local, int64_t n, int64_t lda, double *U,
                    double *S, double *V, const tssvd_comm *comm, tssvd_opts *opts);

/* Bytes of workspace ts_svd_tsqr needs. */
size_t ts_svd_tsqr_workspace_size(int64_t m, int64_t n, const tssvd_opts *opts);

/*
 * Thin SVD by the randomized TSQR methods: Algorithm 1 (opts->passes = 1)
 * or Algorithm 2 (passes = 2).  Each row of A is mixed by the random
 * orthogonal Omega = D F S D~ F S~ of Remark "randomness" (pairs of reals
 * read as complex numbers; F the unitary DFT; n odd is padded with a zero
 * column to n' = n + 1, h = n'/2), the mixed matrix B* = A Omega* is
 * factored B* = Q R by Householder TSQR (row blocks of about 4n', a
 * reduction tree over the stacked R factors, Q formed explicitly from the
 * reflections), rows of R whose |R_jj| is below |R_00| times the working
 * precision wp = opts->drop_tol^2 are discarded with Q's columns; passes =
 * 2 then factors Q = Q2 R2 (same discard) and uses T = R2 R.  The SVD of
 * T (or R) = U~ Sigma V~^T is one-sided Jacobi; U = Q U~, V = Omega^-1 V~.
 * The leading n triplets are returned with the sign rule of ts_svd.  All
 * arithmetic is FP64; opts->mode selects the engine of the two tall
 * products (B* = A Omega* and U = Q U~): TSSVD_FP64 (FMA) or TSSVD_FP64_TC
 * (FP64-accurate digit products on the tensor cores).  opts->scale is not
 * used.
 *   A     [in]  m x n row-major, leading dimension lda >= n (device).
 *   theta [in]  2h phases (device, radians): the diagonal of D (h values)
 *               then of D~ (h values), drawn uniformly by the caller.
 *   perm  [in]  2h indices (device): the permutation of S, (S x)_a =
 *               x_perm[a], then that of S~; each a permutation of 0..h-1.
 *   U, S, V, opts as for ts_svd.  n <= 4096.
 * Errors: -1 A, -2 m < n, -3 n, -4 lda, -5 theta, -6 perm NULL or not in
 * range (detected on the device), -7 U, -8 S, -9 V, -10 opts (or a mode
 * other than TSSVD_FP64 / TSSVD_FP64_TC).
 */
int ts_svd_tsqr(const double *A, int64_t m, int64_t n, int64_t lda, const double *theta,
                const int64_t *perm, double *U, double *S, double *V, tssvd_opts *opts);

/*
 * Rank-k approximation by Algorithm 7: randomized subspace iteration
 * (Algorithm 5) with `iters` power steps orthonormalised by Algorithm 1,
 * the last by Algorithm 2, then Algorithm 6 with the SVD of B = Q^T A as
 * the Algorithm 2 TS-SVD of B^T = A^T Q.  Directions discarded by a TS-SVD
 * are removed (the next step works with the kept width, read back from the
 * device), as in Algorithms 1 and 2.  Every TS-SVD uses the caller's one
 * mixing draw for l columns, restricted to its width w (the first
 * ceil(w/2) phases of each set; each permutation's entries below ceil(w/2)
 * in their order).  The TS-SVDs are FP64; opts->mode selects the engine
 * of the tall products A Q~ and A^T Q: TSSVD_FP64 (FMA) or TSSVD_FP64_TC
 * (FP64-accurate digit products on the tensor cores; other modes are
 * rejected).  The discard compares R's diagonal with the working
 * precision opts->drop_tol^2.
 *   A, m, n, lda, k, l, iters, Omega, U, S, V as for lowrank_svd
 *   (l <= 4096).
 *   theta, perm: the draw of ts_svd_tsqr for l columns (2 ceil(l/2) each).
 * Errors: -1 A, -2 m, -3 n, -4 lda, -5 k, -6 l, -7 iters, -8 Omega,
 * -9 theta, -10 perm (NULL or not a permutation), -11 U, -12 S, -13 V,
 * -14 opts (or a mode other than TSSVD_FP64 / TSSVD_FP64_TC).
 */
int lowrank_svd_tsqr(const double *A, int64_t m, int64_t n, int64_t lda, int64_t k, int64_t l,
                     int iters, const double *Omega, const double *theta, const int64_t *perm,
                     double *U, double *S, double *V, tssvd_opts *opts);

/* Bytes of workspace ts_pca / ts_pca_f32 need: those of ts_svd plus the
 * centred copy (m x n elements) and the column-sum partials. */
size_t ts_pca_workspace_size(int64_t m, int64_t n, int elem_bytes, const tssvd_opts *opts);

/*
 * Principal component analysis of the m observations (rows) of A: the thin
 * SVD of the column-centred matrix A - 1 mu^T, mu_j the mean of column j
 * (the first problem of the paper's abstract, PCA of a highly rectangular
 * matrix, solved with Algorithm 4 or 3 as opts->passes says).  The means
 * are FP64 column sums divided by m and rounded once to the storage type;
 * the centred values A_ij - mu_j are formed explicitly (FP64 difference,
 * one rounding) in the workspace rather than as a rank-one correction of
 * the Gram matrix, which cancels catastrophically when |mu| dominates the
 * spread of the data.  The principal directions are the columns of V, the
 * scores U diag(S), and the variances S_j^2 / (m - 1).  The centred
 * matrix has rank at most m - 1, so for m = n the last singular value is 0
 * (TSSVD_RANKDEF); a matrix whose rows are all equal gives rank 0.
 *   A   [in]  m x n, row-major, leading dimension lda >= n; not modified.
 *   mu  [out] n column means.
 *   U, S, V, opts as for ts_svd, for the centred matrix.
 * Errors: -1 A NULL, -2 m < n or m < 1, -3 n < 1, -4 lda < n, -5 mu NULL,
 * -6 U NULL, -7 S NULL, -8 V NULL, -9 opts NULL or invalid field.
 */
int ts_pca(const double *A, int64_t m, int64_t n, int64_t lda, double *mu, double *U,
           double *S, double *V, tssvd_opts *opts);

/* As ts_pca for FP32 storage (means and centred values rounded to FP32;
 * the SVD as ts_svd_f32). */
int ts_pca_f32(const float *A, int64_t m, int64_t n, int64_t lda, float *mu, float *U,
               float *S, float *V, tssvd_opts *opts);

/* Bytes of workspace lowrank_svd needs. */
size_t lowrank_svd_workspace_size(int64_t m, int64_t n, int64_t l, const tssvd_opts *opts);

/*
 * Rank-k approximation A ~ U diag(S) V^T of a general A (m x n) by
 * Algorithm 8: randomized subspace iteration (Algorithm 5) with `iters`
 * power steps, each normalised by the single-pass Gram TS-SVD
 * (Algorithm 3), the last one by the two-pass TS-SVD (Algorithm 4),
 * followed by the direct SVD of Algorithm 6 (the SVD of B = Q^T A is the
 * two-pass TS-SVD of B^T = A^T Q, n x l).  The leading k of the l
 * triplets are returned.  MaxEntry scaling (opts->scale) is not used.
 * opts->mode: TSSVD_FP64 runs every product in FP64 FMA; TSSVD_FP64_TC
 * runs the products A X and A^T Q and the TS-SVDs with FP64-accurate
 * digit-sliced tensor-core products (the digit images of A, 14 bytes per
 * entry each for the row and the column image, are built once per call
 * and reused by every power step); TSSVD_BF16X3/X6 apply to the TS-SVDs'
 * first passes only (l <= 256), the products with A staying FP64.
 *   A     [in]  m x n row-major, leading dimension lda >= n.
 *   k, l  1 <= k <= l <= min(m, n).
 *   iters number of power steps i >= 0.
 *   Omega [in]  n x l row-major: the starting matrix (i.i.d. Gaussian,
 *               drawn by the caller).
 *   U [out] m x k, S [out] k, V [out] n x k (row-major, dense).
 * Errors: -1 A, -2 m, -3 n, -4 lda, -5 k, -6 l, -7 iters, -8 Omega,
 * -9 U, -10 S, -11 V, -12 opts.
 */
int lowrank_svd(const double *A, int64_t m, int64_t n, int64_t lda, int64_t k, int64_t l,
                int iters, const double *Omega, double *U, double *S, double *V,
                tssvd_opts *opts);

/*
 * Adjoint of the thin SVD computed by ts_svd (full column rank, distinct
 * singular values).  Given the forward inputs A, S, V and the gradients
 * dU (m x n), dS (n), dV (n x n) of a loss with respect to U, S, V (any of
 * the three may be NULL, meaning zero), writes dA (m x n, leading
 * dimension n).  U is recomputed as A V diag(S)^-1 instead of being stored.
 * With F_ij = 1/(s_j^2 - s_i^2) (0 on the diagonal), J = U^T dU, K = V^T dV:
 *   dA = U [ (F o (J - J^T)) S + diag(dS) + S (F o (K - K^T)) - J S^-1 ] V^T
 *        + dU S^-1 V^T.
 * This is the standard thin-SVD adjoint (it is not part of the paper).
 * opts->mode TSSVD_FP64_TC runs the three tall products (U, U^T dU and dA)
 * on the FP64-accurate digit-sliced tensor-core kernels; other modes use
 * FP64 FMA.  Returns 3 if a device wait expired.
 * Errors: -1 A, -2 m, -3 n, -4 lda, -5 S, -6 V, -10 dA, -11 opts.
 */
int ts_svd_backward(const double *A, int64_t m, int64_t n, int64_t lda, const double *S,
                    const double *V, const double *dU, const double *dS, const double *dV,
                    double *dA, tssvd_opts *opts);

/*
 * Adjoint of the rank-k SVD returned by lowrank_svd (Algorithm 8).  Given
 * the forward outputs U (m x k), S (k, distinct and positive), V (n x k)
 * and the gradients dU (m x k), dS (k), dV (n x k) of a loss (any of the
 * three may be NULL, meaning zero), writes dA (m x n, leading dimension n):
 *   dA = U [ (F o (J - J^T)) S + diag(dS) + S (F o (K - K^T)) ] V^T
 *        + (I - U U^T) dU S^-1 V^T + U S^-1 dV^T (I - V V^T),
 * F, J, K as for ts_svd_backward.  This is the derivative of the leading k
 * singular triplets when A has rank k; for other A it omits the coupling
 * with the discarded singular values, which the rank-k factors do not
 * carry.  A itself is not needed.  All arrays are row-major and dense,
 * device pointers owned by the caller; dA is fully overwritten.
 * opts->mode TSSVD_FP64_TC forms the one m x n product, [U | dU] times a
 * 2k x n factor, on the digit-sliced tensor-core kernels; other modes use
 * FP64 FMA.  Returns 3 if a device wait expired.
 * Errors: -1 m < 1, -2 n < 1, -3 k < 1 or k > min(m, n), -4 U, -5 S,
 * -6 V, -10 dA, -11 opts.
 */
int lowrank_svd_backward(int64_t m, int64_t n, int64_t k, const double *U, const double *S,
                         const double *V, const double *dU, const double *dS, const double *dV,
                         double *dA, tssvd_opts *opts);

/* As ts_svd_backward for FP32 storage (the FP32 forward of ts_svd_f32);
 * the adjoint is evaluated in FP64 and dA rounded to FP32. */
int ts_svd_backward_f32(const float *A, int64_t m, int64_t n, int64_t lda, const float *S,
                        const float *V, const float *dU, const float *dS, const float *dV,
                        float *dA, tssvd_opts *opts);

/* One member of a batch for ts_svd_batched. */
typedef struct {
    const void *A;   /* [in]  m x n, row-major, leading dimension lda (device) */
    int64_t m, n, lda;
    void *U;         /* [out] m x n (leading dimension n) */
    void *S;         /* [out] n */
    void *V;         /* [out] n x n */
    int64_t out_rank; /* [out] */
    int status;      /* [out] status of this member (as ts_svd returns) */
    int mode;        /* [out] arithmetic mode used (TSSVD_AUTO resolved) */
    int sweeps[3];   /* [out] Jacobi sweeps of its three solves, as tssvd_opts */
} tssvd_desc;

/*
 * Many independent tall-skinny SVDs (Algorithm 3 or 4 each, as opts->passes
 * says) of uneven sizes in one submission.  All members have the same
 * element type (elem_bytes 8 = double, 4 = float) and the same options.
 * The members are ordered largest first and spread over worker streams;
 * members on one worker stream run one after another and share one slice
 * of the workspace (ts_svd_batched_workspace_size).  When every member has
 * n <= 256, passes = 2 and the mode is TSSVD_FP64_TC or TSSVD_AUTO, the
 * batch runs in phases instead: the members' tall products and small steps
 * on the worker streams, and each of the three Jacobi solves of all members
 * as one launch with a cluster of two thread blocks per member (the eigensolves
 * one-sided on the pivoted Cholesky factor; for n >= 64 the first
 * eigensolve and the SVD of R start with an FP32 phase, as the single-call
 * solver does from n = 129); every member then runs
 * TSSVD_FP64_TC, its per-solve state is kept in the workspace between the
 * phases, and for double members U's storage holds Y~ until U is written.
 * Results match single calls to rounding (bit for bit on the per-member
 * path).  The whole batch is
 * captured once into a CUDA graph, which is cached by the batch's
 * descriptors and options and replayed on later calls with the same ones;
 * one graph launch on opts->stream runs the batch.  Returns after the
 * stream has finished; each member's status, rank and resolved mode are
 * written to its descriptor, and the call returns the first nonzero member
 * status (TSSVD_OK if none).  opts->mode may be TSSVD_AUTO.
 * Errors: -1 descs NULL, -2 count < 1, -3 elem_bytes, -4 opts; -(100 + i)
 * when member i has an invalid field.
 */
size_t ts_svd_batched_workspace_size(const tssvd_desc *descs, int count, int elem_bytes,
                                     const tssvd_opts *opts);
int ts_svd_batched(tssvd_desc *descs, int count, int elem_bytes, tssvd_opts *opts);

/*
 * Gram matrix B = A^T A of A (m x n, row-major, lda >= n): the first step of
 * Algorithms 3 and 4 (and the Z = Y^T Y step of Algorithm 4), in FP64 on
 * the CUDA cores.  Split-K over the rows: each CTA accumulates a partial
 * Gram of a row slab (the per-partition Gram matrices the paper aggregates,
 * Section 2) into workspace, and a second kernel sums the partials in a
 * fixed order, so the result is deterministic.  B is n x n row-major
 * (leading dimension n), written in full (both triangles).  Uses
 * opts->stream and opts->workspace (ts_gram_workspace_size bytes) like
 * ts_svd; returns after the stream has finished.  opts->mode selects FP64
 * DFMA, the BF16-split tensor-core product (n <= 256) or the FP64-accurate
 * digit-sliced tensor-core product (TSSVD_FP64_TC, any n).
 * Errors: -1 A, -2 m, -3 n, -4 lda, -5 B, -6 opts.
 */
size_t ts_gram_workspace_size(int64_t m, int64_t n);
int ts_gram(const double *A, int64_t m, int64_t n, int64_t lda, double *B, tssvd_opts *opts);

/*
 * Tall product C = A M: A is m x k (row-major, lda), M is k x n (ldm), C is
 * m x n (ldc), all FP64 device memory.  The product Y~ = A V~ of
 * Algorithms 3 and 4 (and U = Q P, Y = A Q~ of Algorithm 5) as a call of its
 * own.  opts->mode selects FP64 DFMA, the BF16-split tensor-core product
 * (n <= 256) or the FP64-accurate digit-sliced tensor-core product
 * (TSSVD_FP64_TC, any n).  Uses opts->stream and opts->workspace
 * (ts_matmul_workspace_size bytes); returns after the stream has finished.
 * Errors: -1 A, -2 m, -3 k, -4 lda, -5 M, -6 n, -7 ldm, -8 C, -9 ldc,
 * -10 opts.
 */
size_t ts_matmul_workspace_size(int64_t m, int64_t k, int64_t n);
int ts_matmul(const double *A, int64_t m, int64_t k, int64_t lda, const double *M, int64_t n,
              int64_t ldm, double *C, int64_t ldc, tssvd_opts *opts);

/*
 * ts_gram_noalloc: B = A^T A like ts_gram, for callers that must not have
 * the library allocate device memory (for example a host framework that
 * owns all device memory through its own pool, or code that cannot accept
 * the device-wide synchronisation cudaMalloc may cause).  The paper has no
 * counterpart; it is a deployment variant of the Gram step.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *    The split-K partial sums live in a fixed 4 MiB scratch array that is
 *    part of the library's device image; every GPU that loads the library
 *    holds it until the process exits.
 *  - Size limit: n <= 724 (n*n partial entries must fit the scratch); a
 *    larger n returns -3 and prints the reason.  m is unrestricted.
 *  - The first call on each device looks up the scratch's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one scratch array, which keeps the last call's
 *    contents (every entry a call reads is written by the same call first).
 *    Calls whose work overlaps on the GPU (for example on two streams at
 *    once) race on it: serialise them.
 *  - stream is a cudaStream_t (NULL = legacy default stream); the call
 *    returns after the stream has finished.  B is n x n row-major.
 * Errors: -1 A, -2 m, -3 n (or n > 724), -4 lda, -5 B; TSSVD_ECUDA.
 */
int ts_gram_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, double *B, void *stream);

/*
 * Instrumentation (not part of the paper's method).
 * tssvd_launch_count: number of kernels the library has launched in this
 * process.  tssvd_profile_enable(1) makes every later launch record a CUDA
 * event pair on its own stream; tssvd_profile_report synchronises the
 * device, writes one line per kernel name "name launches total_ms" into
 * buf (NUL-terminated, truncated to len) and clears the records; with
 * buf == NULL it only returns the bytes the full report needs and keeps the
 * records.  tssvd_profile_enable returns the previous setting.
 */
long long tssvd_launch_count(void);
int tssvd_profile_enable(int on);
size_t tssvd_profile_report(char *buf, size_t len);

/* tssvd_fp64_fma_rate: measures the FP64 fused multiply-add rate of the
 * current device (the ceiling of the FP64 kernels: the Jacobi solvers, the
 * Householder factorizations and the FP64 tall products), in TFLOP/s
 * (2 flops per FMA), by timing a kernel of independent FMA chains with CUDA
 * events on `stream` (a cudaStream_t; NULL = legacy default stream), best
 * of four runs after one warm-up (about 1.5 s in all).  Writes *tflops and
 * returns TSSVD_OK, or -1 (tflops NULL) / TSSVD_ECUDA.  Allocates nothing. */
int tssvd_fp64_fma_rate(double *tflops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TSSVD_H */
