// Internal declarations shared by the library's CUDA translation units.
// Target: GB300 (sm_103a) only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tssvd.h"

namespace tssvd {

typedef int64_t i64;

// Device-side status block, one per call.  `err` is set by kernels whose
// bounded waits expire (TSSVD_ETIMEOUT); the host reads the block once at
// the end of the call.
struct DevStatus {
    int err;
    int rank1;     // first discard step
    int rank2;     // second discard step
    int rank;      // nonzero singular values returned
    int sweeps[4]; // Jacobi sweeps per solve (-1 = cap reached)
    int bar[4];    // scratch for the Jacobi grid barrier (bar[0..1]: 64-bit count)
    int orient;    // 1: the small SVD ran on the columns of R (else of R^T)
    int pad[3];
};

// Number of SMs of the current device (cached per device).
int num_sms();

// Adds kernel launches made by a graph replay to the launch counter.
void add_launches(long long k);
// Whether launch profiling is on, and a kernel time measured by the caller
// (a launch inside a graph replay, timed by event nodes of the graph) added
// to the profile under `name`.
bool profiling();
void prof_add_ms(const char *name, double ms);

// Wraps one kernel launch: counts it, and when profiling is on records a
// CUDA event pair around it on its stream (see profiler.cu).
struct ProfScope {
    int idx;
    cudaStream_t s;
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
};

// ---------------------------------------------------------------- products
// All tall products accumulate in FP64 (DFMA on the CUDA cores).

// bits[j] = max_i |A_ij| as the bit pattern of a non-negative double
// (bits must be zeroed first).  The MaxEntry of every column.
template <typename T>
cudaError_t launch_colmax(const T *A, i64 m, i64 n, i64 lda, unsigned long long *bits,
                          cudaStream_t s);

// d[j] = smallest power of two >= max_i |A_ij| (1 for a zero column),
// dinv[j] = 1 / d[j].
cudaError_t launch_pow2_scale(const unsigned long long *bits, i64 n, double *d, double *dinv,
                              cudaStream_t s);

// Split-K partials of C = A^T B: A is K x M (lda), B is K x N (ldb), both
// row-major.  P holds `splits` slices of M x N.  With upper_only (A == B,
// M == N) only tiles on or above the diagonal are computed.
template <typename TA, typename TB>
cudaError_t launch_tn_partial(const TA *A, i64 lda, const TB *B, i64 ldb, i64 K, i64 M, i64 N,
                              int splits, bool upper_only, double *P, cudaStream_t s);
int tn_splits(i64 K, i64 M, i64 N, bool upper_only);

// C[i][j] = rs[i] * cs[j] * sum_s P[s][i][j] (rs, cs may be null); sym:
// only i <= j is summed and mirrored.  Deterministic (fixed order over s).
cudaError_t launch_tn_reduce(const double *P, int splits, i64 M, i64 N, const double *rs,
                             const double *cs, bool sym, double *C, i64 ldc, cudaStream_t s);

// C = A B with A m x K (lda, type TA), B K x N (ldb, FP64); C written as TC
// when non-null (ldc).  NP[g][j] receives per-CTA-row partial sums of
// squares of column j of the FP64 product (g < nn_grid_rows(m, N)).
template <typename TA, typename TC>
cudaError_t launch_nn(const TA *A, i64 lda, const double *B, i64 ldb, i64 m, i64 K, i64 N,
                      TC *C, i64 ldc, double *NP, cudaStream_t s);
int nn_grid_rows(i64 m, i64 N);

// Column sums of squares of X (m x n, FP64): partials NP[g][j],
// g < colsumsq_rows(m, n); sum them with launch_norms_reduce.
int colsumsq_rows(i64 m, i64 n);
cudaError_t launch_colsumsq(const double *X, i64 ldx, i64 m, i64 n, double *NP, cudaStream_t s);
// Algorithms 1 and 2 (tsqr.cu).  Mt = O^T (2h x 2h) of Remark
// "randomness"'s mixing from th (2h phases) and perm (2h indices); *bad is
// set if a permutation entry is out of range.
cudaError_t launch_mixing(int h, const double *th, const i64 *perm, double *Mt, int *bad,
                          cudaStream_t s);
// The draw for w columns (hw = ceil(w/2)) from one for h complex entries.
cudaError_t launch_restrict_mix(const double *th, const i64 *perm, int h, int hw, double *thw,
                                i64 *permw, int *bad, cudaStream_t s);
// Householder TSQR of X (m x n, dense, destroyed): R (n x n, upper) and
// Q (m x n) with X = Q R; work: tsqr_workspace_doubles(m, n) doubles.
size_t tsqr_workspace_doubles(i64 m, int n);
cudaError_t launch_tsqr(double *X, i64 m, int n, double *work, double *R, double *Q,
                        cudaStream_t s);
// Discard of R's small diagonal entries (rows of R, columns of Q zeroed).
cudaError_t launch_tsqr_discard(double *R, double *Q, i64 m, int n, double wp, int *keep,
                                cudaStream_t s);
// launch_colmax streams whole rows when n <= 32 * kColStatMaxCh, with
// colstat_blocks(m, n) blocks (0 when n is larger).
constexpr int kColStatMaxCh = 16;
int colstat_blocks(i64 m, i64 n);
// Column means mu = A^T 1 / m (FP64 sums of the deviations from the first
// row, rounded once to T): P holds colsum_rows(m, n) * n doubles of
// partials.
int colsum_rows(i64 m, i64 n);
template <typename T>
cudaError_t launch_col_means(const T *A, i64 lda, i64 m, i64 n, double *P, T *mu, cudaStream_t s);
// C = A - 1 mu^T, C dense (leading dimension n).
template <typename T>
cudaError_t launch_center(const T *A, i64 lda, i64 m, i64 n, const T *mu, T *C, cudaStream_t s);

// out[j] = sqrt(sum_g NP[g][j]) in fixed order.
cudaError_t launch_norms_reduce(const double *NP, int g, i64 N, double *out, cudaStream_t s);
// The same sums without the square root (row-sharded calls: the squares
// are summed over the ranks first), and x[j] = sqrt(x[j]).
cudaError_t launch_sumsq_reduce(const double *NP, int g, i64 N, double *out, cudaStream_t s);
cudaError_t launch_sqrt_inplace(double *x, i64 N, cudaStream_t s);

// ------------------------------------------------- tensor-core products
// BF16-split products on tcgen05 (gemm_tc.cu).  S = number of bf16 terms
// per value (2 or 3).  Both require n (resp. N) <= 256.
int tc_gram_splits(i64 m);
// Partials P[split][i][j] (splits x n x n) of A^T A, FP64.
template <typename T>
cudaError_t launch_tc_gram(const T *A, i64 lda, i64 m, int n, int S, int splits, double *P,
                           DevStatus *st, cudaStream_t s);
// Bytes of the split image of a K x N right-hand matrix.
size_t tc_split_b_bytes(int K, int N, int S);
cudaError_t launch_tc_split_b(const double *M, i64 ldm, int K, int N, int S, uint8_t *img,
                              cudaStream_t s);
// C (m x N, FP64, ldc) = A (m x K) * M, with M given as its split image.
template <typename T>
cudaError_t launch_tc_nn(const T *A, i64 lda, i64 m, int K, const uint8_t *img, int N, int S,
                         double *C, i64 ldc, DevStatus *st, cudaStream_t s);

// FP64-accurate digit-sliced products on tcgen05 (gemm_oz.cu).
int oz_gram_tiles(int n);
int oz_gram_splits(i64 m, int n);
size_t oz_image_bytes(int K, int N);
size_t oz_gram_image_bytes(i64 m, int n);
size_t oz_row_image_bytes(i64 m, int K);
// P[split][i][j] partial Grams of X (m x n); |X[k][j]| <= 2^ex[j].  gimg:
// scratch of oz_gram_image_bytes(m, n) for the digit image.
template <typename T>
cudaError_t launch_oz_gram(const T *X, i64 ldx, i64 m, int n, const int *ex, int splits,
                           uint8_t *gimg, double *P, DevStatus *st, cudaStream_t s);
// A^T B from column digit images (see launch_oz_col_image): partials
// P[split][i][j] (M x N) over the rows of A (m x M) and B (m x N).
int oz_tn_splits(i64 m, int M, int N);
cudaError_t launch_oz_col_image(const double *X, i64 ldx, i64 m, int n, const int *ex,
                                uint8_t *img, cudaStream_t s);
cudaError_t launch_oz_tn(const uint8_t *aimg, const int *exa, int M, const uint8_t *bimg,
                         const int *exb, int N, i64 m, int splits, double *P, DevStatus *st,
                         cudaStream_t s);
// Digit image of diag(2^-pk) M (K x N) and its column exponents em.
cudaError_t launch_oz_image(const double *M, i64 ldm, int K, int N, const int *pk, int *em,
                            uint8_t *img, cudaStream_t s);
// er[r] = exponent bounding row r of A diag(2^pk).  per_sm caps the grid
// at that many CTAs per SM (small when it runs beside a Jacobi solve).
template <typename T>
cudaError_t launch_oz_rowexp(const T *A, i64 lda, i64 m, int K, const int *pk, int *er,
                             cudaStream_t s, int per_sm = 16);
// C = A M with A prescaled by 2^pk (see launch_oz_image), row exponents er;
// aimg: scratch of oz_row_image_bytes(m, K) for A's digit image.
template <typename T, typename TC>
cudaError_t launch_oz_nn(const T *A, i64 lda, i64 m, int K, const int *pk, const int *er,
                         uint8_t *aimg, const uint8_t *bimg, const int *em, int N, TC *C, i64 ldc,
                         DevStatus *st, cudaStream_t s);
// The two halves of launch_oz_nn: A's row digit image, and the product
// from a prebuilt image (to reuse one image of A for several products).
template <typename T>
cudaError_t launch_oz_row_image(const T *A, i64 lda, i64 m, int K, const int *pk, const int *er,
                                uint8_t *aimg, cudaStream_t s, int per_sm = 16);
// Optionally (N <= 512, oz_nn_fuses) with the output's column statistics:
// colmax_out[j] = max(colmax_out[j], bits of max_i |C_ij|) (zeroed by the
// caller) and colsq_out[b * N + j] = the sum of C_ij^2 over the rows of
// CTA b (oz_nn_grid(m, N) rows of partials, reduced by the caller).
int oz_nn_grid(i64 m, int N);
bool oz_nn_fuses(int N);
template <typename TC>
cudaError_t launch_oz_nn_run(const uint8_t *aimg, i64 m, int K, const int *er, const uint8_t *bimg,
                             const int *em, int N, TC *C, i64 ldc, DevStatus *st, cudaStream_t s,
                             unsigned long long *colmax_out = nullptr, double *colsq_out = nullptr);
cudaError_t launch_oz_exp_from_bits(const unsigned long long *bits, int n, int *ex, cudaStream_t s);
// pk[j] = round(log2(sc[j])) (0 for sc[j] <= 0).
cudaError_t launch_oz_pow2_of(const double *sc, int n, int *pk, cudaStream_t s);
// out[j] = -in[j].
cudaError_t launch_neg_int(const int *in, int n, int *out, cudaStream_t s);
// dst[j] = max(dst[j], src[j]) for column maxima held as the bit patterns
// of non-negative doubles (launch_colmax), whose integer order is numeric.
cudaError_t launch_bits_max(unsigned long long *dst, const unsigned long long *src, i64 n,
                            cudaStream_t s);

// -------------------------------------------------------------- Jacobi
// One-sided (Hestenes) Jacobi with a parallel round-robin pair order, as
// one cooperative kernel with a bounded grid barrier.  X is nr x nc
// column-major (column j at X + j*ldx), J (nc x nc, column-major) receives
// the accumulated rotations: X_in J = X_out with orthogonal columns.
// ctr must point to at least max_sweeps + 4 zeroed ints of device memory;
// prm to jacobi_prm_doubles(nc) doubles of scratch.
inline size_t jacobi_prm_doubles(i64 nc) { return 8 * (size_t)((nc + 1) / 2) + (size_t)nc + 8; }
// tol: the rotation threshold |x_p . x_q| > tol |x_p| |x_q| (0: nr 2^-53).
// J == null: the rotations are not accumulated (only X_out is wanted).
cudaError_t launch_jacobi(double *X, i64 ldx, double *J, i64 ldj, int nr, int nc,
                          int max_sweeps, int *ctr, double *prm, DevStatus *st, int which,
                          cudaStream_t s, double tol = 0.0);

// Pivoted Cholesky of the symmetric W (n x n row-major, consumed) with a
// floor: P^T W P = R^T R, pivots the largest remaining diagonal entries;
// once all remaining ones are <= 2^-52 max_i W_ii the trailing block of R
// is that floor's square root times I (W = 0: R = I).  X = R^T
// column-major (ldx), piv[i] = the original index of pivoted index i.
// One CTA; used for n <= kPcholMaxN.
constexpr int kPcholMaxN = 256;
cudaError_t launch_pchol(double *W, int n, double *X, i64 ldx, int *piv, cudaStream_t s);
// The same for many independent problems in one launch, one CTA each
// (X with ldx = n; every n <= nmax <= 256; tasks a device array).
struct PcholTask {
    double *W;
    double *X;
    int *piv;
    int n;
};
cudaError_t launch_pchol_batch(const PcholTask *tasks, int ntasks, int nmax, cudaStream_t s);
// The same factorization over the whole grid (cooperative launch, one
// barrier per pivot step) with logical pivoting: W stays in the original
// order and X's column k is row k of R~ = R P^T (so W = R~^T R~, and X's
// rows are in the original order: nothing to un-pivot).  key: 3 unsigned
// 64-bit words of scratch.  n <= kPcholGridMaxN.
constexpr int kPcholGridMaxN = 2048;
cudaError_t launch_pchol_grid(double *W, int n, double *X, i64 ldx, unsigned long long *key,
                              DevStatus *st, cudaStream_t s);
// One-sided Jacobi in two precisions (jacobi_mixed.cu) for
// kJacobiMixedMinN <= n <= kJacobiMixedMaxN: an FP32 phase (at most
// kJacobiMixedF32Sweeps sweeps, its count added to st->sweeps[3]) picks an
// orthogonal basis K (made orthogonal in FP64 by two Newton-Schulz steps),
// X <- X K, then launch_jacobi in FP64 with threshold tol finishes (its
// sweeps in st->sweeps[which]).  X is n x n column-major (ldx = n);
// Jout (n x n column-major, or null) receives K times the FP64 phase's
// rotations.  Scratch: f32 (n*n doubles, holding two n x n FP32 arrays),
// K, T, H, X0 (n x n doubles each), P (tn_splits(n, n, n, false) * n * n
// doubles) and NP (nn_grid_rows(n, n) * n doubles); prm and ctr as for
// launch_jacobi.
// From n = 129 the FP32 phase pays for its conversions and Newton-Schulz
// products (2,000,000 x 200: 67.9 -> 63.4 ms; at n = 50..100 even).
constexpr int kJacobiMixedMinN = 129;
constexpr int kJacobiMixedMaxN = 2048;
constexpr int kJacobiMixedF32Sweeps = 40;
struct JacobiMixedScratch {
    double *f32, *K, *T, *H, *X0, *P, *NP;
};

// Batched one-sided Jacobi (jacobi_batch.cu): a cluster of two CTAs per task, each an
// independent n x n problem (n <= kJacobiBatchMaxN) with X column-major
// (ldx = n), J (n x n, column-major) set to the identity and receiving the
// rotations when non-null, threshold tol as launch_jacobi, and its sweep
// count in st->sweeps[which] (-1 when max_sweeps ran out).  tasks is a
// device array of ntasks entries, ordered largest first.
constexpr int kJacobiBatchMaxN = 256;
struct JacobiTask {
    double *X;
    double *J;
    int n;
    int which;
    double tol;
    DevStatus *st;
    // non-null: the solve starts with an FP32 phase (its sweeps added to
    // st->sweeps[3]); scratch of 2 n^2 floats and 2 n^2 doubles
    float *w32;
    double *wk;
};
cudaError_t launch_jacobi_batch(const JacobiTask *tasks, int ntasks, int max_sweeps,
                                cudaStream_t s);
bool jacobi_mixed_applies(i64 n);
cudaError_t launch_jacobi_mixed(double *X, i64 n, double *Jout, const JacobiMixedScratch &w,
                                int max_sweeps, int *ctr, double *prm, DevStatus *st, int which,
                                cudaStream_t s, double tol = 0.0);
// V[piv[i]][j] = Xn[i][j], n x n row-major.
cudaError_t launch_row_scatter(const double *Xn, const int *piv, int n, double *V, cudaStream_t s);

// Eigendecomposition of the symmetric B (n x n row-major) by Gram-form
// Jacobi, same pair schedule and barrier.  V (n x n, column-major)
// accumulates the rotations; on return lam holds the eigenvalues (diagonal
// of the rotated B) in decreasing order and Vout (row-major, ldvo) the
// matching eigenvectors as columns.  B2: a second n x n buffer (ldb) for
// the one-barrier-per-round form, or NULL for the two-barrier in-place
// form; either way B's contents are consumed.  prm: scratch of
// jacobi_prm_doubles(n) doubles; perm: n ints; ctr as for launch_jacobi.
// The eigenvectors are returned with unit norms (V's accumulated columns
// divided by their recomputed norms).
// normwise (one-barrier forms only): a pair rotates only when |b_PQ| also
// exceeds 2^-52 times the largest diagonal entry (refreshed each sweep),
// i.e. is above the rounding already in B; used for the first Gram
// eigensolve of the two-pass algorithm.
cudaError_t launch_jacobi_eig(double *B, double *B2, i64 ldb, double *V, i64 ldv, double *lam,
                              double *Vout, i64 ldvo, int n, int max_sweeps, int *ctr, double *prm,
                              int *perm, DevStatus *st, int which, cudaStream_t s,
                              bool normwise = false);

// Column norms of the column-major X, stable descending order, and the
// sorted outputs.  Eigen mode: Vout (nc x nc row-major, column r = J
// column perm[r]) and lam[r].  SVD mode additionally: Uout (nr x nc
// row-major, column r = X column perm[r] / sigma_r, 0 when sigma_r = 0).
// (orient non-null and *orient != 0, nr == nc: the J and X/s outputs trade
// places, for a Jacobi run on the columns of R instead of R^T.)
// jnorm (nc doubles of scratch, or null): J's columns are divided by their
// recomputed norms, removing the rounding drift of the accumulated
// rotations (needed wherever J is a result).
cudaError_t launch_jacobi_finalize(const double *X, i64 ldx, const double *J, i64 ldj, int nr,
                                   int nc, double *norms, int *perm, double *Jout, i64 ldjo,
                                   double *lam, double *Xout, i64 ldxo, cudaStream_t s,
                                   const int *orient = nullptr, double *jnorm = nullptr);

// ---------------------------------------------------------- small ops
// Discard rule: smax = max sig; r = 1 + last j with sig_j > 0 and not
// (sig_j < smax*tol); inv[j] = 1/sig_j for j < r (0 otherwise).  Writes r
// to *rank_out.
cudaError_t launch_discard(const double *sig, i64 n, double tol, double *inv, int *rank_out,
                           cudaStream_t s);
// out[i][j] = rs[i] * M[i][j] * cs[j] (rs/cs may be null), rows x cols.
cudaError_t launch_scale2(const double *M, i64 ldm, i64 rows, i64 cols, const double *rs,
                          const double *cs, double *out, i64 ldo, cudaStream_t s);
// G[b][c] = (keep[b] != 0 ? sig[b] : 0) * Vt[c][b] * d[c]  (n x n), keep = inv.
cudaError_t launch_build_g(const double *sig, const double *keep, const double *Vt, i64 ldv,
                           const double *d, i64 n, double *G, cudaStream_t s);
// Sign canonicalisation of the columns of V (rows x cols row-major):
// sgn[j] = +-1 so that the entry of largest magnitude (lowest index on
// ties) becomes positive; sgn[j] = 0 when sig[j] == 0.  V is flipped in place.
cudaError_t launch_signs(double *V, i64 ldv, i64 rows, i64 cols, const double *sig,
                         double *sgn, cudaStream_t s);
// rank = number of sig[j] > 0 -> *rank_out.
cudaError_t launch_count_positive(const double *sig, i64 n, int *rank_out, cudaStream_t s);
// out[j] = sqrt(max(G[j][j], 0)).
cudaError_t launch_diag_sqrt(const double *G, i64 ldg, i64 n, double *out, cudaStream_t s);
// out[j] = keep[j] != 0 ? val[j] : 0 (val null: 1).
cudaError_t launch_keepval(const double *val, const double *keep, i64 n, double *out,
                           cudaStream_t s);
// X = R or R^T (n x n, dense) for the one-sided Jacobi SVD of R; *orient
// receives 1 for R^T storage (Jacobi on the columns of R).  Columns of R are
// chosen when the MaxEntry scaling d (null: none) spans more than
// kOrientBits binary orders of magnitude and no row of R was discarded
// (*rank2 == n): R = B diag(d), and one-sided Jacobi converges in a few
// sweeps on column-graded matrices but slowly on their transposes.
constexpr int kOrientBits = 12;
cudaError_t launch_orient_copy(const double *d, const int *rank2, const double *R, i64 n,
                               double *X, int *orient, cudaStream_t s);
// dst[j][i] = src[i][j] * rs[j] (rs may be null); src rows x cols.
cudaError_t launch_transpose(const double *src, i64 lds, i64 rows, i64 cols, const double *rs,
                             double *dst, i64 ldd, cudaStream_t s);
// n x n core of the thin-SVD adjoint (J, K, dS may be null).
cudaError_t launch_adjoint_core(const double *J, const double *K, const double *sv,
                                const double *dS, i64 n, double *M, cudaStream_t s);
// M[a][b] -= K[b][a] * sinv[a] (k x k).
cudaError_t launch_core_fix(double *M, const double *K, const double *sinv, i64 k, cudaStream_t s);
// X[a][j] += sinv[a] * D[j][a] (X k x n, D n x k).
cudaError_t launch_add_scaled_t(const double *D, i64 ldd, i64 n, i64 k, const double *sinv,
                                double *X, i64 ldx, cudaStream_t s);
// Conversions to the output type.
template <typename T>
cudaError_t launch_convert(const double *src, i64 lds, i64 rows, i64 cols, T *dst, i64 ldd,
                           cudaStream_t s);
// U[i][j] *= cs[j] in place (rows x cols, row-major).
template <typename T>
cudaError_t launch_scale_cols_inplace(T *U, i64 ldu, i64 rows, i64 cols, const double *cs,
                                      cudaStream_t s);
// Copy a row-major matrix of type TS into a double matrix.
template <typename TS>
cudaError_t launch_to_double(const TS *src, i64 lds, i64 rows, i64 cols, double *dst, i64 ldd,
                             cudaStream_t s);

}  // namespace tssvd
