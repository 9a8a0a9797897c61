/*
 * Plain FP64 CPU oracle for the Gram-based tall-skinny SVD and the
 * randomized low-rank SVD of Li, Kluger & Tygert, "Randomized algorithms
 * for distributed computation of PCA and SVD" (arXiv:1612.08709).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library, and it imports nothing from it.
 *
 * Everything is written as the paper states it, step by step, in double
 * precision, with plain loops (no BLAS).  OpenMP is used only to split
 * independent rows or columns of a product across threads; it does not
 * change what is summed, only the order in which per-thread partial sums of
 * a Gram matrix are added.
 *
 * Matrices are row-major with an explicit leading dimension ("ld", in
 * elements).  Singular vectors are stored as columns: V[i*ldv + j] is entry
 * i of right singular vector j.
 *
 * Readings of the paper this file takes (each also listed in the design
 * notes of the repository):
 *  - The small eigenproblems and the small SVD use one-sided (Hestenes)
 *    cyclic Jacobi with row-cyclic pair order.  A pair (p,q) is rotated when
 *    |x_p . x_q| > tol * sqrt(|x_p|^2 |x_q|^2), tol = nrows * 2^-53; the
 *    iteration stops after a sweep with no rotation, or after max_sweeps.
 *    For the two Gram eigenproblems the method runs in Gram form (the
 *    inner products are the entries of the Gram matrix itself, see
 *    or_jacobi_eig); the SVD of R runs on the columns of R^T.  Results are
 *    sorted in decreasing order, ties by original index.
 *  - MaxEntry column scaling (an addition to the paper's method): column j
 *    of A is divided by d_j, the smallest power of two >= max_i |A_ij|
 *    (d_j = 1 for a zero column).  It applies to the two-pass algorithm
 *    only, where the diagonal D is absorbed into R = T W^T S~ V~^T D
 *    before the final small SVD; the one-pass algorithm ignores it.
 *  - The discard rule drops every column whose explicit norm is strictly
 *    less than (largest norm) * drop_tol; the paper's value for drop_tol is
 *    the square root of the working precision (Remark "working").
 *  - Sign convention: each right singular vector is flipped so that its
 *    entry of largest magnitude (lowest index on ties) is positive; the
 *    matching left singular vector is flipped with it.
 *  - PCA (the first problem of the abstract; the paper does not spell out
 *    the centering): the principal components of the rows of A are the
 *    singular triplets of C = A - 1 mu^T with mu the column means, and C is
 *    formed explicitly before the TS-SVD.
 *  - The low-rank SVD returns the leading k of the l triplets that the
 *    direct SVD produces; the SVD of B = Q^T A is taken as the two-pass
 *    tall-skinny SVD of B^T = A^T Q (n x l).
 *
 * Pins: see tests/test_oracle_pins.py (brute-force SVD on tiny inputs,
 * known spectra, the paper's low-rank error values on its DCT test matrix,
 * orthonormality invariants, closed forms for n = 1, finite differences
 * for the gradient).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

#define OR_OK 0
#define OR_ENOCONV 1
#define OR_RANKDEF 2
#define OR_ENOMEM (-100)

/* ------------------------------------------------------------------ */
/* Small helpers (plain loops).                                        */
/* ------------------------------------------------------------------ */

static double *dalloc(i64 n)
{
    if (n <= 0) n = 1;
    return (double *)calloc((size_t)n, sizeof(double));
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* B (n x n, ldb) = A^T A for A (m x n, lda).  Definition of the Gram matrix
 * (Algorithm 3, first step; Algorithm 4, first and Z = Y^T Y steps). */
void or_gram(const double *A, i64 m, i64 n, i64 lda, double *B, i64 ldb)
{
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) B[i * ldb + j] = 0.0;
    int nt = or_num_threads();
    /* One partial Gram per thread over a static row partition, summed in
     * thread order afterwards, so the result is the same on every run with
     * the same thread count. */
    double **parts = (double **)calloc((size_t)nt, sizeof(double *));
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *P = dalloc(n * n);
        parts[t] = P;
#pragma omp for schedule(static)
        for (i64 k = 0; k < m; k++) {
            const double *a = A + k * lda;
            for (i64 i = 0; i < n; i++) {
                double ai = a[i];
                double *p = P + i * n;
                for (i64 j = i; j < n; j++) p[j] += ai * a[j];
            }
        }
    }
    for (int t = 0; t < nt; t++) {
        if (!parts[t]) continue;
        for (i64 i = 0; i < n; i++)
            for (i64 j = i; j < n; j++) B[i * ldb + j] += parts[t][i * n + j];
        free(parts[t]);
    }
    free(parts);
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < i; j++) B[i * ldb + j] = B[j * ldb + i];
}

/* C (m x p, ldc) = A (m x n, lda) * X (n x p, ldx). */
void or_matmul(const double *A, i64 m, i64 n, i64 lda, const double *X,
               i64 p, i64 ldx, double *C, i64 ldc)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < m; i++) {
        double *c = C + i * ldc;
        for (i64 j = 0; j < p; j++) c[j] = 0.0;
        for (i64 k = 0; k < n; k++) {
            double a = A[i * lda + k];
            const double *x = X + k * ldx;
            for (i64 j = 0; j < p; j++) c[j] += a * x[j];
        }
    }
}

/* C (n x p, ldc) = A^T (A is m x n, lda) * X (m x p, ldx). */
void or_matmul_tn(const double *A, i64 m, i64 n, i64 lda, const double *X,
                  i64 p, i64 ldx, double *C, i64 ldc)
{
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < n; i++) {
        double *c = C + i * ldc;
        for (i64 j = 0; j < p; j++) c[j] = 0.0;
        for (i64 k = 0; k < m; k++) {
            double a = A[k * lda + i];
            const double *x = X + k * ldx;
            for (i64 j = 0; j < p; j++) c[j] += a * x[j];
        }
    }
}

/* Euclidean norm of every column (Remark "normalizing"). */
void or_col_norms(const double *Y, i64 m, i64 n, i64 ldy, double *s)
{
    for (i64 j = 0; j < n; j++) {
        double acc = 0.0;
        for (i64 i = 0; i < m; i++) acc += Y[i * ldy + j] * Y[i * ldy + j];
        s[j] = sqrt(acc);
    }
}

/* d_j = smallest power of two >= max_i |A_ij|; 1 for a zero column. */
void or_maxentry_scale(const double *A, i64 m, i64 n, i64 lda, double *d)
{
    for (i64 j = 0; j < n; j++) {
        double mx = 0.0;
        for (i64 i = 0; i < m; i++) {
            double v = fabs(A[i * lda + j]);
            if (v > mx) mx = v;
        }
        if (mx == 0.0 || !isfinite(mx)) {
            d[j] = 1.0;
        } else {
            int e;
            double f = frexp(mx, &e); /* mx = f * 2^e, f in [0.5, 1) */
            d[j] = (f == 0.5) ? mx : ldexp(1.0, e);
        }
    }
}

/* ------------------------------------------------------------------ */
/* One-sided (Hestenes) cyclic Jacobi.                                  */
/* ------------------------------------------------------------------ */

/*
 * Orthogonalises the columns of X (nr x nc, ldx) in place by plane
 * rotations, accumulating the rotations in J (nc x nc, ldj, set to I here):
 * on return X_in * J = X_out with mutually orthogonal columns.  J's
 * columns are then scaled to unit norm (unit_columns), and the
 * columns of X_out and J are permuted into order of decreasing norm
 * (stable), and s[j] = |X_out column j|.  Returns the number of sweeps
 * taken, or -1 if max_sweeps sweeps all rotated something.
 *
 * For a symmetric positive semi-definite X this is an eigendecomposition:
 * X J = J diag(lambda), so J holds eigenvectors and s the eigenvalues
 * (Algorithm 3 and 4, eigendecomposition steps).  For a general X it is a
 * singular value decomposition X = (X_out diag(1/s)) diag(s) J^T
 * (Algorithm 4, SVD of R).
 */
/* sqrt(|a b|), as sqrt|a| sqrt|b| so that it neither overflows nor
 * underflows for squared norms near the ends of the exponent range. */
static double jac_geo(double a, double b)
{
    return sqrt(fabs(a)) * sqrt(fabs(b));
}

/* Rotation angle that annihilates the (p,q) inner product g of two columns
 * with squared norms a, b: t = tan(theta) is the smaller root of
 * t^2 + 2 zeta t - 1 = 0, zeta = (b - a) / (2 g), that is
 * t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)).  For |zeta| > 1 the same
 * value is r / (1 + sqrt(1 + r^2)) with r = 1 / |zeta| = |2 g| / |b - a|,
 * which neither overflows nor loses the angle when a and b differ by
 * hundreds of orders of magnitude (zeta itself would overflow there).
 * The result is 0 only when the angle underflows; the caller then treats
 * the pair as converged, since the rotation would be the identity. */
static double jac_tan(double a, double b, double g)
{
    const double d = b - a, ad = fabs(d), ag2 = fabs(2.0 * g);
    double t;
    if (ad > ag2) {
        const double r = ag2 / ad;
        t = r / (1.0 + sqrt(1.0 + r * r));
    } else {
        const double z = ad / ag2;
        t = 1.0 / (z + sqrt(1.0 + z * z));
    }
    const int pos = (d == 0.0) || ((d > 0.0) == (g > 0.0));
    return pos ? t : -t;
}

/* Divides each column of the n x n matrix J (ldj) by its Euclidean norm.
 * The accumulated rotations are the eigenvectors (or singular vectors) of
 * the Jacobi methods, which are unit vectors by definition; each FP64
 * rotation with c = 1/sqrt(1 + t^2), s = c t has c^2 + s^2 = 1 + O(eps),
 * biased upward once t^2 is below the rounding unit, so over many
 * rotations the columns' norms drift above 1 (about 1e-13 at n = 300,
 * which is what limited the orthonormality of U = Q P in Algorithm 4). */
static void unit_columns(double *J, i64 n, i64 ldj)
{
    for (i64 j = 0; j < n; j++) {
        double ss = 0.0;
        for (i64 i = 0; i < n; i++) ss += J[i * ldj + j] * J[i * ldj + j];
        const double nr = sqrt(ss);
        if (nr > 0.0)
            for (i64 i = 0; i < n; i++) J[i * ldj + j] /= nr;
    }
}

int or_jacobi(double *X, i64 nr, i64 nc, i64 ldx, double *J, i64 ldj,
              double *s, int max_sweeps)
{
    const double tol = (double)nr * ldexp(1.0, -53);
    for (i64 i = 0; i < nc; i++)
        for (i64 j = 0; j < nc; j++) J[i * ldj + j] = (i == j) ? 1.0 : 0.0;

    int sweeps_done = -1;
    for (int sweep = 1; sweep <= max_sweeps; sweep++) {
        i64 rotations = 0;
        for (i64 p = 0; p < nc - 1; p++) {
            for (i64 q = p + 1; q < nc; q++) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (i64 i = 0; i < nr; i++) {
                    double xp = X[i * ldx + p], xq = X[i * ldx + q];
                    alpha += xp * xp;
                    beta += xq * xq;
                    gamma += xp * xq;
                }
                if (gamma == 0.0 || !(fabs(gamma) > tol * jac_geo(alpha, beta)))
                    continue;
                double t = jac_tan(alpha, beta, gamma);
                if (t == 0.0) continue;
                rotations++;
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (i64 i = 0; i < nr; i++) {
                    double xp = X[i * ldx + p], xq = X[i * ldx + q];
                    X[i * ldx + p] = c * xp - sn * xq;
                    X[i * ldx + q] = sn * xp + c * xq;
                }
                for (i64 i = 0; i < nc; i++) {
                    double jp = J[i * ldj + p], jq = J[i * ldj + q];
                    J[i * ldj + p] = c * jp - sn * jq;
                    J[i * ldj + q] = sn * jp + c * jq;
                }
            }
        }
        if (rotations == 0) {
            sweeps_done = sweep;
            break;
        }
    }
    unit_columns(J, nc, ldj);

    /* Norms and a stable sort by decreasing norm (insertion sort on an
     * index array keeps equal norms in original order). */
    i64 *idx = (i64 *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(i64));
    double *nrm = dalloc(nc);
    or_col_norms(X, nr, nc, ldx, nrm);
    for (i64 j = 0; j < nc; j++) idx[j] = j;
    for (i64 a = 1; a < nc; a++) {
        i64 key = idx[a];
        i64 b = a - 1;
        while (b >= 0 && nrm[idx[b]] < nrm[key]) {
            idx[b + 1] = idx[b];
            b--;
        }
        idx[b + 1] = key;
    }
    double *tx = dalloc(nr * nc), *tj = dalloc(nc * nc);
    for (i64 i = 0; i < nr; i++)
        for (i64 j = 0; j < nc; j++) tx[i * nc + j] = X[i * ldx + idx[j]];
    for (i64 i = 0; i < nc; i++)
        for (i64 j = 0; j < nc; j++) tj[i * nc + j] = J[i * ldj + idx[j]];
    for (i64 i = 0; i < nr; i++)
        for (i64 j = 0; j < nc; j++) X[i * ldx + j] = tx[i * nc + j];
    for (i64 i = 0; i < nc; i++)
        for (i64 j = 0; j < nc; j++) J[i * ldj + j] = tj[i * nc + j];
    for (i64 j = 0; j < nc; j++) s[j] = nrm[idx[j]];
    free(idx);
    free(nrm);
    free(tx);
    free(tj);
    return sweeps_done;
}

/*
 * Eigendecomposition of a symmetric positive semi-definite B (n x n, ldb)
 * by one-sided Jacobi in Gram form: B is taken as the Gram matrix of an
 * implicit matrix X (B = X^T X), and the rotation of pair (p,q) is the one
 * that orthogonalises columns p and q of X, computed from b_pp, b_qq, b_pq
 * and applied as B <- J^T B J (so b_pq becomes 0, b_pp <- b_pp - t b_pq,
 * b_qq <- b_qq + t b_pq).  Rotations accumulate in V (n x n, ldv, set to I
 * here) and are scaled to unit columns at the end (unit_columns).  Same
 * rotation test and stopping rule as or_jacobi with
 * tol = n * 2^-53 (relative to sqrt(|b_pp b_qq|)).  On return lam holds the
 * diagonal of the rotated B sorted in decreasing order (stable), V's
 * columns are permuted to match, and B holds the rotated matrix (unsorted).
 * Returns the number of sweeps, or -1 if the cap was reached.
 */
int or_jacobi_eig(double *B, i64 n, i64 ldb, double *V, i64 ldv, double *lam,
                  int max_sweeps)
{
    const double tol = (double)n * ldexp(1.0, -53);
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) V[i * ldv + j] = (i == j) ? 1.0 : 0.0;
    int sweeps_done = -1;
    for (int sweep = 1; sweep <= max_sweeps; sweep++) {
        i64 rotations = 0;
        for (i64 p = 0; p < n - 1; p++) {
            for (i64 q = p + 1; q < n; q++) {
                double a = B[p * ldb + p], b = B[q * ldb + q], g = B[p * ldb + q];
                if (g == 0.0 || !(fabs(g) > tol * jac_geo(a, b))) continue;
                double t = jac_tan(a, b, g);
                if (t == 0.0) continue;
                rotations++;
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                /* B <- B J (columns p, q), then B <- J^T B (rows p, q). */
                for (i64 k = 0; k < n; k++) {
                    double bp = B[k * ldb + p], bq = B[k * ldb + q];
                    B[k * ldb + p] = c * bp - sn * bq;
                    B[k * ldb + q] = sn * bp + c * bq;
                }
                for (i64 k = 0; k < n; k++) {
                    double bp = B[p * ldb + k], bq = B[q * ldb + k];
                    B[p * ldb + k] = c * bp - sn * bq;
                    B[q * ldb + k] = sn * bp + c * bq;
                }
                /* the 2 x 2 block in closed form */
                B[p * ldb + p] = a - t * g;
                B[q * ldb + q] = b + t * g;
                B[p * ldb + q] = 0.0;
                B[q * ldb + p] = 0.0;
                for (i64 k = 0; k < n; k++) {
                    double vp = V[k * ldv + p], vq = V[k * ldv + q];
                    V[k * ldv + p] = c * vp - sn * vq;
                    V[k * ldv + q] = sn * vp + c * vq;
                }
            }
        }
        if (rotations == 0) {
            sweeps_done = sweep;
            break;
        }
    }
    unit_columns(V, n, ldv);
    /* stable sort by decreasing diagonal */
    i64 *idx = (i64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(i64));
    double *dg = dalloc(n), *tv = dalloc(n * n);
    for (i64 j = 0; j < n; j++) {
        idx[j] = j;
        dg[j] = B[j * ldb + j];
    }
    for (i64 a = 1; a < n; a++) {
        i64 key = idx[a];
        i64 b = a - 1;
        while (b >= 0 && dg[idx[b]] < dg[key]) {
            idx[b + 1] = idx[b];
            b--;
        }
        idx[b + 1] = key;
    }
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) tv[i * n + j] = V[i * ldv + idx[j]];
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) V[i * ldv + j] = tv[i * n + j];
    for (i64 j = 0; j < n; j++) lam[j] = dg[idx[j]];
    free(idx);
    free(dg);
    free(tv);
    return sweeps_done;
}

/* Flip V column j (n rows) and U column j (m rows) so that V's entry of
 * largest magnitude (lowest index on ties) is positive. */
static void canonical_signs(double *U, i64 m, i64 ldu, double *V, i64 n,
                            i64 ldv, i64 r)
{
    for (i64 j = 0; j < r; j++) {
        i64 best = 0;
        double bv = -1.0;
        for (i64 i = 0; i < n; i++) {
            double a = fabs(V[i * ldv + j]);
            if (a > bv) {
                bv = a;
                best = i;
            }
        }
        if (V[best * ldv + j] < 0.0) {
            for (i64 i = 0; i < n; i++) V[i * ldv + j] = -V[i * ldv + j];
            if (U)
                for (i64 i = 0; i < m; i++) U[i * ldu + j] = -U[i * ldu + j];
        }
    }
}

/* Number of leading entries of the decreasing sequence s kept by the
 * discard rule: s_j is dropped when s_j < s_0 * drop_tol (or s_j == 0). */
static i64 keep_count(const double *s, i64 n, double drop_tol)
{
    if (n == 0) return 0;
    double thr = s[0] * drop_tol;
    i64 r = 0;
    for (i64 j = 0; j < n; j++)
        if (s[j] > 0.0 && !(s[j] < thr)) r = j + 1;
    return r;
}

/* ------------------------------------------------------------------ */
/* Algorithm 3: Gram-based TS-SVD, single orthonormalisation.           */
/* ------------------------------------------------------------------ */

/*
 * A (m x n, lda) -> U (m x n, ldu), S (n), V (n x n, ldv), *rank.
 * Columns r..n-1 of U and V and entries r..n-1 of S are set to zero.
 * Returns OR_OK, OR_RANKDEF (r < n), or OR_ENOCONV (Jacobi cap hit).
 */
int or_ts_svd1(const double *A, i64 m, i64 n, i64 lda, double drop_tol,
               int max_sweeps, double *U, i64 ldu, double *S, double *V,
               i64 ldv, i64 *rank)
{
    int status = OR_OK;
    double *B = dalloc(n * n), *Vt = dalloc(n * n), *lam = dalloc(n);
    double *Ut = dalloc(m * n), *sig = dalloc(n);
    /* Form the Gram matrix B = A^T A. */
    or_gram(A, m, n, lda, B, n);
    /* Eigendecomposition B = V D V^T. */
    if (or_jacobi_eig(B, n, n, Vt, n, lam, max_sweeps) < 0) status = OR_ENOCONV;
    /* U~ = A V. */
    or_matmul(A, m, n, lda, Vt, n, n, Ut, n);
    /* Sigma = Euclidean norms of the columns of U~. */
    or_col_norms(Ut, m, n, n, sig);
    /* The eigenvalue order fixes the column order; the explicit norms can
     * deviate from it only at rounding level, so the kept set is the
     * leading columns whose norms pass the rule against the largest norm. */
    double smax = 0.0;
    for (i64 j = 0; j < n; j++)
        if (sig[j] > smax) smax = sig[j];
    i64 r = 0;
    for (i64 j = 0; j < n; j++)
        if (sig[j] > 0.0 && !(sig[j] < smax * drop_tol)) r = j + 1;
    /* U = U~ Sigma^{-1}; discarded columns are zeroed. */
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++)
            U[i * ldu + j] = (j < r) ? Ut[i * n + j] / sig[j] : 0.0;
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) V[i * ldv + j] = (j < r) ? Vt[i * n + j] : 0.0;
    for (i64 j = 0; j < n; j++) S[j] = (j < r) ? sig[j] : 0.0;
    canonical_signs(U, m, ldu, V, n, ldv, r);
    *rank = r;
    if (status == OR_OK && r < n) status = OR_RANKDEF;
    free(B);
    free(Vt);
    free(lam);
    free(Ut);
    free(sig);
    return status;
}

/* ------------------------------------------------------------------ */
/* Algorithm 4: Gram-based TS-SVD, double orthonormalisation.           */
/* ------------------------------------------------------------------ */

/*
 * Same interface as or_ts_svd1, plus `scale` (MaxEntry column scaling).
 * Also returns, when `diag` is non-NULL, diag[0] = first-pass rank r,
 * diag[1] = second-pass rank r', diag[2..] unused.
 */
int or_ts_svd2(const double *A, i64 m, i64 n, i64 lda, int scale,
               double drop_tol, int max_sweeps, double *U, i64 ldu, double *S,
               double *V, i64 ldv, i64 *rank, i64 *diag)
{
    int status = OR_OK;
    double *d = dalloc(n);
    double *As = dalloc(m * n);
    double *B = dalloc(n * n), *Vt = dalloc(n * n), *lam = dalloc(n);
    double *Yt = dalloc(m * n), *sigt = dalloc(n);

    /* Optional MaxEntry scaling: work on A D^{-1}. */
    if (scale)
        or_maxentry_scale(A, m, n, lda, d);
    else
        for (i64 j = 0; j < n; j++) d[j] = 1.0;
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) As[i * n + j] = A[i * lda + j] / d[j];

    /* B = A^T A. */
    or_gram(As, m, n, n, B, n);
    /* B = V~ D~ V~^T. */
    if (or_jacobi_eig(B, n, n, Vt, n, lam, max_sweeps) < 0) status = OR_ENOCONV;
    /* Y~ = A V~. */
    or_matmul(As, m, n, n, Vt, n, n, Yt, n);
    /* Sigma~ = column norms of Y~. */
    or_col_norms(Yt, m, n, n, sigt);
    double smax = 0.0;
    for (i64 j = 0; j < n; j++)
        if (sigt[j] > smax) smax = sigt[j];
    /* Discard: columns whose norm is below max * drop_tol. */
    i64 r = 0;
    for (i64 j = 0; j < n; j++)
        if (sigt[j] > 0.0 && !(sigt[j] < smax * drop_tol)) r = j + 1;

    /* Y = Y~ Sigma~^{-1} (m x r). */
    double *Y = dalloc(m * r);
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < r; j++) Y[i * r + j] = Yt[i * n + j] / sigt[j];

    /* Z = Y^T Y; Z = W D W^T. */
    double *Z = dalloc(r * r), *W = dalloc(r * r), *mu = dalloc(r);
    or_gram(Y, m, r, r, Z, r);
    if (or_jacobi_eig(Z, r, r, W, r, mu, max_sweeps) < 0) status = OR_ENOCONV;
    /* Q~ = Y W; T = column norms of Q~. */
    double *Qt = dalloc(m * r), *T = dalloc(r);
    or_matmul(Y, m, r, r, W, r, r, Qt, r);
    or_col_norms(Qt, m, r, r, T);
    double tmax = 0.0;
    for (i64 j = 0; j < r; j++)
        if (T[j] > tmax) tmax = T[j];
    i64 r2 = 0;
    for (i64 j = 0; j < r; j++)
        if (T[j] > 0.0 && !(T[j] < tmax * drop_tol)) r2 = j + 1;

    /* Q = Q~ T^{-1} (m x r2). */
    double *Q = dalloc(m * r2);
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < r2; j++) Q[i * r2 + j] = Qt[i * r + j] / T[j];

    /* R = T W^T Sigma~ V~^T (r2 x n), with D folded in: R = ... V~^T D. */
    double *R = dalloc(r2 * n);
    for (i64 a = 0; a < r2; a++)
        for (i64 c = 0; c < n; c++) {
            double acc = 0.0;
            for (i64 b = 0; b < r; b++)
                acc += W[b * r + a] * sigt[b] * Vt[c * n + b];
            R[a * n + c] = T[a] * acc * d[c];
        }

    /* SVD R = P Sigma V^T via one-sided Jacobi on R^T (n x r2):
     * R^T P = X with orthogonal columns, Sigma = column norms, V = X/Sigma. */
    double *Rt = dalloc(n * r2), *P = dalloc(r2 * r2), *sg = dalloc(r2);
    for (i64 a = 0; a < r2; a++)
        for (i64 c = 0; c < n; c++) Rt[c * r2 + a] = R[a * n + c];
    if (or_jacobi(Rt, n, r2, r2, P, r2, sg, max_sweeps) < 0) status = OR_ENOCONV;

    /* U = Q P (m x r2). */
    double *Uq = dalloc(m * r2);
    or_matmul(Q, m, r2, r2, P, r2, r2, Uq, r2);

    i64 rk = 0;
    for (i64 j = 0; j < r2; j++)
        if (sg[j] > 0.0) rk = j + 1;
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) U[i * ldu + j] = (j < rk) ? Uq[i * r2 + j] : 0.0;
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++)
            V[i * ldv + j] = (j < rk) ? Rt[i * r2 + j] / sg[j] : 0.0;
    for (i64 j = 0; j < n; j++) S[j] = (j < rk) ? sg[j] : 0.0;
    canonical_signs(U, m, ldu, V, n, ldv, rk);
    *rank = rk;
    if (diag) {
        diag[0] = r;
        diag[1] = r2;
    }
    if (status == OR_OK && rk < n) status = OR_RANKDEF;

    free(d); free(As); free(B); free(Vt); free(lam); free(Yt); free(sigt);
    free(Y); free(Z); free(W); free(mu); free(Qt); free(T); free(Q); free(R);
    free(Rt); free(P); free(sg); free(Uq);
    return status;
}

/* ------------------------------------------------------------------ */
/* Algorithms 1 and 2: randomized TS-SVD via TSQR (Remark "randomness") */
/* ------------------------------------------------------------------ */

/*
 * The random orthogonal mixing of Remark "randomness",
 * Omega = D F S D~ F S~ on C^h: D = diag(exp(i th1)), D~ = diag(exp(i th2)),
 * F the unitary DFT ((F x)_a = sum_b x_b exp(-2 pi i a b / h) / sqrt(h)),
 * (S x)_a = x_{p1[a]}, (S~ x)_a = x_{p2[a]}.  A real vector of length 2h
 * is read as h complex numbers (x_{2k} + i x_{2k+1}); O (2h x 2h, row
 * major) is the real matrix of Omega in that reading:
 *   O[2j][2k] = Re w, O[2j][2k+1] = -Im w, O[2j+1][2k] = Im w,
 *   O[2j+1][2k+1] = Re w, with w = Omega_jk.
 * Column k of Omega is Omega applied to e_k, step by step.
 */
static void or_dft(const double *xr, const double *xi, i64 h, double *yr, double *yi)
{
    const double pi = 3.14159265358979323846, sc = 1.0 / sqrt((double)h);
    for (i64 a = 0; a < h; a++) {
        double sr = 0.0, si = 0.0;
        for (i64 b = 0; b < h; b++) {
            const double ang = -2.0 * pi * (double)((a * b) % h) / (double)h;
            const double c = cos(ang), sn = sin(ang);
            sr += xr[b] * c - xi[b] * sn;
            si += xr[b] * sn + xi[b] * c;
        }
        yr[a] = sr * sc;
        yi[a] = si * sc;
    }
}

void or_mixing(i64 h, const double *th1, const double *th2, const i64 *p1, const i64 *p2,
               double *O)
{
    double *xr = dalloc(h), *xi = dalloc(h), *yr = dalloc(h), *yi = dalloc(h);
    const i64 n2 = 2 * h;
    for (i64 k = 0; k < h; k++) {
        /* S~ e_k */
        for (i64 a = 0; a < h; a++) {
            xr[a] = (p2[a] == k) ? 1.0 : 0.0;
            xi[a] = 0.0;
        }
        or_dft(xr, xi, h, yr, yi); /* F */
        for (i64 a = 0; a < h; a++) { /* D~ */
            const double c = cos(th2[a]), sn = sin(th2[a]);
            const double r = yr[a] * c - yi[a] * sn, im = yr[a] * sn + yi[a] * c;
            yr[a] = r;
            yi[a] = im;
        }
        for (i64 a = 0; a < h; a++) { /* S */
            xr[a] = yr[p1[a]];
            xi[a] = yi[p1[a]];
        }
        or_dft(xr, xi, h, yr, yi); /* F */
        for (i64 j = 0; j < h; j++) { /* D, then the real 2 x 2 blocks */
            const double c = cos(th1[j]), sn = sin(th1[j]);
            const double wr = yr[j] * c - yi[j] * sn, wi = yr[j] * sn + yi[j] * c;
            O[(2 * j) * n2 + 2 * k] = wr;
            O[(2 * j) * n2 + 2 * k + 1] = -wi;
            O[(2 * j + 1) * n2 + 2 * k] = wi;
            O[(2 * j + 1) * n2 + 2 * k + 1] = wr;
        }
    }
    free(xr);
    free(xi);
    free(yr);
    free(yi);
}

/* sqrt(sum x_i^2) with scaling, so that neither overflows nor underflows. */
static double scaled_norm(const double *x, i64 cnt, i64 stride)
{
    double mx = 0.0;
    for (i64 i = 0; i < cnt; i++)
        if (fabs(x[i * stride]) > mx) mx = fabs(x[i * stride]);
    if (mx == 0.0) return 0.0;
    double ss = 0.0;
    for (i64 i = 0; i < cnt; i++) {
        const double t = x[i * stride] / mx;
        ss += t * t;
    }
    return mx * sqrt(ss);
}

/*
 * Householder QR of X (m x n, ldx, m >= n): X = Q R with Q (m x n, ldq)
 * orthonormal and R (n x n, ldr) upper triangular.  Reflection j is
 * H_j = I - tau_j v v^T with v_j = 1, chosen so that H_j maps column j
 * (rows j..m-1) onto beta e_j, beta = -sign(x_jj) |x|; a column that is
 * already zero below and on the diagonal takes H_j = I.  Q is formed by
 * applying the reflections to [I; 0] in reverse order.
 */
void or_householder_qr(const double *X, i64 m, i64 n, i64 ldx, double *Q, i64 ldq, double *R,
                       i64 ldr)
{
    double *W = dalloc(m * n), *tau = dalloc(n);
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) W[i * n + j] = X[i * ldx + j];
    for (i64 j = 0; j < n; j++) {
        const double alpha = W[j * n + j];
        const double xn = (j + 1 < m) ? scaled_norm(W + (j + 1) * n + j, m - j - 1, n) : 0.0;
        if (xn == 0.0) {
            tau[j] = 0.0;
            continue;
        }
        const double beta = -copysign(hypot(alpha, xn), alpha);
        tau[j] = (beta - alpha) / beta;
        const double sc = 1.0 / (alpha - beta);
        for (i64 i = j + 1; i < m; i++) W[i * n + j] *= sc;
        W[j * n + j] = beta;
        for (i64 c = j + 1; c < n; c++) {
            double w = W[j * n + c];
            for (i64 i = j + 1; i < m; i++) w += W[i * n + j] * W[i * n + c];
            W[j * n + c] -= tau[j] * w;
            for (i64 i = j + 1; i < m; i++) W[i * n + c] -= tau[j] * W[i * n + j] * w;
        }
    }
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) R[i * ldr + j] = (j >= i) ? W[i * n + j] : 0.0;
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) Q[i * ldq + j] = (i == j) ? 1.0 : 0.0;
    for (i64 j = n - 1; j >= 0; j--) {
        if (tau[j] == 0.0) continue;
        for (i64 c = j; c < n; c++) {
            double w = Q[j * ldq + c];
            for (i64 i = j + 1; i < m; i++) w += W[i * n + j] * Q[i * ldq + c];
            Q[j * ldq + c] -= tau[j] * w;
            for (i64 i = j + 1; i < m; i++) Q[i * ldq + c] -= tau[j] * W[i * n + j] * w;
        }
    }
    free(W);
    free(tau);
}

/* The discard step of Algorithms 1 and 2: row j of R (n x n) is dropped,
 * with column j of Q (m x n), when |R_jj| is below |R_00| times the working
 * precision wp (or is zero); dropped rows and columns become zero. */
static void tsqr_discard(double *Q, i64 m, double *R, i64 n, double wp)
{
    const double thr = fabs(R[0]) * wp;
    for (i64 j = 0; j < n; j++) {
        const double d = fabs(R[j * n + j]);
        if (d > 0.0 && !(d < thr)) continue;
        for (i64 c = 0; c < n; c++) R[j * n + c] = 0.0;
        for (i64 i = 0; i < m; i++) Q[i * n + j] = 0.0;
    }
}

/*
 * Algorithm 1 (passes = 1) or Algorithm 2 (passes = 2) on A (m x n, lda):
 * B* = A Omega* (each row of A mixed by O; n odd is padded with a zero
 * column to n' = n + 1), B* = Q R by Householder QR (TSQR computes the
 * same factorization up to the signs of R's rows), discard, [Q = Q2 R2,
 * discard, T = R2 R], SVD of T (or R) = U~ Sigma V~^T by one-sided Jacobi
 * on its transpose's columns, U = Q U~, V = O^T V~ (first n rows).
 * Returns the leading n triplets; status as or_ts_svd2.
 */
int or_ts_svd_tsqr(const double *A, i64 m, i64 n, i64 lda, int passes, double wp,
                   const double *th1, const double *th2, const i64 *p1, const i64 *p2,
                   int max_sweeps, double *U, i64 ldu, double *S, double *V, i64 ldv,
                   i64 *rank)
{
    const i64 np = n + (n & 1), h = np / 2;
    int status = OR_OK;
    double *O = dalloc(np * np), *Bs = dalloc(m * np), *Q1 = dalloc(m * np);
    double *R1 = dalloc(np * np), *T = dalloc(np * np), *Tt = dalloc(np * np);
    double *J = dalloc(np * np), *sg = dalloc(np), *Uf = dalloc(m * np);
    or_mixing(h, th1, th2, p1, p2, O);
    /* B* = A_pad O^T: row i of B* is O applied to row i of A */
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < np; j++) {
            double acc = 0.0;
            for (i64 k = 0; k < n; k++) acc += A[i * lda + k] * O[j * np + k];
            Bs[i * np + j] = acc;
        }
    or_householder_qr(Bs, m, np, np, Q1, np, R1, np);
    tsqr_discard(Q1, m, R1, np, wp);
    double *Qf = Q1;
    double *Q2 = NULL, *R2 = NULL;
    if (passes == 2) {
        Q2 = dalloc(m * np);
        R2 = dalloc(np * np);
        or_householder_qr(Q1, m, np, np, Q2, np, R2, np);
        tsqr_discard(Q2, m, R2, np, wp);
        for (i64 i = 0; i < np; i++)
            for (i64 j = 0; j < np; j++) {
                double acc = 0.0;
                for (i64 k = 0; k < np; k++) acc += R2[i * np + k] * R1[k * np + j];
                T[i * np + j] = acc;
            }
        Qf = Q2;
    } else {
        memcpy(T, R1, sizeof(double) * np * np);
    }
    /* T = J Sigma (X / Sigma)^T from one-sided Jacobi on the columns of T^T */
    for (i64 i = 0; i < np; i++)
        for (i64 j = 0; j < np; j++) Tt[j * np + i] = T[i * np + j];
    if (or_jacobi(Tt, np, np, np, J, np, sg, max_sweeps) < 0) status = OR_ENOCONV;
    /* U = Qf J, V = O^T (X / Sigma) */
    or_matmul(Qf, m, np, np, J, np, np, Uf, np);
    i64 r = 0;
    for (i64 j = 0; j < n; j++)
        if (sg[j] > 0.0) r = j + 1;
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) U[i * ldu + j] = (j < r) ? Uf[i * np + j] : 0.0;
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) {
            double acc = 0.0;
            if (j < r)
                for (i64 k = 0; k < np; k++) acc += O[k * np + i] * Tt[k * np + j] / sg[j];
            V[i * ldv + j] = acc;
        }
    for (i64 j = 0; j < n; j++) S[j] = (j < r) ? sg[j] : 0.0;
    canonical_signs(U, m, ldu, V, n, ldv, r);
    *rank = r;
    if (status == OR_OK && r < n) status = OR_RANKDEF;
    free(O); free(Bs); free(Q1); free(R1); free(T); free(Tt); free(J); free(sg); free(Uf);
    free(Q2); free(R2);
    return status;
}

/* ------------------------------------------------------------------ */
/* PCA (abstract, problem 1): SVD of the column-centred matrix.         */
/* ------------------------------------------------------------------ */

/* mu_j = (sum_i A_ij) / m.  The sum is taken in row order with Neumaier's
 * compensated summation (a running sum plus a running correction for the
 * rounding error of each addition), so it is accurate to about one
 * rounding whatever m and the offset of the column; this accuracy matters
 * because an error in mu_j perturbs every centred entry of column j. */
void or_col_means(const double *A, i64 m, i64 n, i64 lda, double *mu)
{
    for (i64 j = 0; j < n; j++) {
        double t = 0.0, corr = 0.0;
        for (i64 i = 0; i < m; i++) {
            const double a = A[i * lda + j];
            const double u = t + a;
            if (fabs(t) >= fabs(a))
                corr += (t - u) + a;
            else
                corr += (a - u) + t;
            t = u;
        }
        mu[j] = (t + corr) / (double)m;
    }
}

/*
 * Principal components of the rows of A: mu = column means, then the
 * TS-SVD (Algorithm 4 when passes = 2, else Algorithm 3) of the centred
 * matrix C = A - 1 mu^T, formed explicitly.  Outputs and status as
 * or_ts_svd1 / or_ts_svd2, plus mu (n).
 */
int or_pca(const double *A, i64 m, i64 n, i64 lda, int passes, int scale,
           double drop_tol, int max_sweeps, double *mu, double *U, i64 ldu,
           double *S, double *V, i64 ldv, i64 *rank)
{
    double *C = dalloc(m * n);
    or_col_means(A, m, n, lda, mu);
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) C[i * n + j] = A[i * lda + j] - mu[j];
    int st;
    if (passes == 1)
        st = or_ts_svd1(C, m, n, n, drop_tol, max_sweeps, U, ldu, S, V, ldv,
                        rank);
    else
        st = or_ts_svd2(C, m, n, n, scale, drop_tol, max_sweeps, U, ldu, S, V,
                        ldv, rank, NULL);
    free(C);
    return st;
}

/* ------------------------------------------------------------------ */
/* Algorithms 5, 6 and 8: randomized low-rank SVD (Gram flavour).       */
/* ------------------------------------------------------------------ */

/* Orthonormal basis of the range of Y (rows x cols) by the one- or
 * two-pass TS-SVD; returns the basis width and writes it to Qout
 * (rows x cols, leading width columns). */
static i64 ts_basis(const double *Y, i64 rows, i64 cols, int passes,
                    double drop_tol, int max_sweeps, double *Qout, int *st)
{
    double *S = dalloc(cols), *V = dalloc(cols * cols);
    i64 r = 0;
    int s;
    if (passes == 1)
        s = or_ts_svd1(Y, rows, cols, cols, drop_tol, max_sweeps, Qout, cols,
                       S, V, cols, &r);
    else
        s = or_ts_svd2(Y, rows, cols, cols, 0, drop_tol, max_sweeps, Qout,
                       cols, S, V, cols, &r, NULL);
    if (s == OR_ENOCONV) *st = OR_ENOCONV;
    free(S);
    free(V);
    return r;
}

/*
 * Algorithm 8 = Algorithm 6 fed by Algorithm 5, with Algorithm 3 for the
 * power steps and Algorithm 4 for the last step and for the SVD of B.
 * A (m x n, lda); Omega (n x l, row-major, ld = l) is the starting matrix
 * Q~_0 (i.i.d. Gaussian, supplied by the caller).  Outputs: U (m x k, ldu),
 * S (k), V (n x k, ldv), *rank = number of nonzero triplets returned.
 * If `ranks` is non-NULL it receives the basis widths of every step in
 * order: [Q_1, Q~_1, ..., Q_i, Q~_i, Q, direct-SVD rank] (2*iters + 2).
 */
int or_lowrank_svd(const double *A, i64 m, i64 n, i64 lda, i64 k, i64 l,
                   int iters, const double *Omega, double drop_tol,
                   int max_sweeps, double *U, i64 ldu, double *S, double *V,
                   i64 ldv, i64 *rank, i64 *ranks)
{
    int st = OR_OK;
    i64 w = l; /* current basis width */
    double *Qtil = dalloc(n * l), *Q = dalloc(m * l);
    double *Y = dalloc(m * l), *Yt = dalloc(n * l), *tmp;
    i64 ri = 0;
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < l; j++) Qtil[i * l + j] = Omega[i * l + j];

    for (int it = 0; it < iters; it++) {
        /* Y_j = A Q~_{j-1}. */
        or_matmul(A, m, n, lda, Qtil, w, w, Y, w);
        /* Y_j = Q_j R_j by Algorithm 3. */
        tmp = dalloc(m * w);
        i64 w1 = ts_basis(Y, m, w, 1, drop_tol, max_sweeps, tmp, &st);
        for (i64 i = 0; i < m; i++)
            for (i64 j = 0; j < w1; j++) Q[i * w1 + j] = tmp[i * w + j];
        free(tmp);
        if (ranks) ranks[ri++] = w1;
        /* Y~_j = A^T Q_j. */
        or_matmul_tn(A, m, n, lda, Q, w1, w1, Yt, w1);
        /* Y~_j = Q~_j R~_j by Algorithm 3. */
        tmp = dalloc(n * w1);
        i64 w2 = ts_basis(Yt, n, w1, 1, drop_tol, max_sweeps, tmp, &st);
        for (i64 i = 0; i < n; i++)
            for (i64 j = 0; j < w2; j++) Qtil[i * w2 + j] = tmp[i * w1 + j];
        free(tmp);
        if (ranks) ranks[ri++] = w2;
        w = w2;
    }
    /* Y = A Q~_i; Y = Q R by Algorithm 4. */
    or_matmul(A, m, n, lda, Qtil, w, w, Y, w);
    tmp = dalloc(m * w);
    i64 wq = ts_basis(Y, m, w, 2, drop_tol, max_sweeps, tmp, &st);
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < wq; j++) Q[i * wq + j] = tmp[i * w + j];
    free(tmp);
    if (ranks) ranks[ri++] = wq;

    /* Algorithm 6: B = Q^T A, taken as B^T = A^T Q (n x wq); its two-pass
     * TS-SVD B^T = U1 S V1^T gives B = V1 S U1^T, so U~ = V1, V = U1. */
    double *Bt = dalloc(n * wq), *U1 = dalloc(n * wq), *S1 = dalloc(wq),
           *V1 = dalloc(wq * wq);
    or_matmul_tn(A, m, n, lda, Q, wq, wq, Bt, wq);
    i64 rb = 0;
    int s2 = or_ts_svd2(Bt, n, wq, wq, 0, drop_tol, max_sweeps, U1, wq, S1, V1,
                        wq, &rb, NULL);
    if (s2 == OR_ENOCONV) st = OR_ENOCONV;
    if (ranks) ranks[ri++] = rb;
    /* U = Q U~ = Q V1 (m x wq). */
    double *Uf = dalloc(m * wq);
    or_matmul(Q, m, wq, wq, V1, wq, wq, Uf, wq);

    i64 kk = k < rb ? k : rb;
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < k; j++) U[i * ldu + j] = (j < kk) ? Uf[i * wq + j] : 0.0;
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < k; j++) V[i * ldv + j] = (j < kk) ? U1[i * wq + j] : 0.0;
    for (i64 j = 0; j < k; j++) S[j] = (j < kk) ? S1[j] : 0.0;
    canonical_signs(U, m, ldu, V, n, ldv, kk);
    *rank = kk;
    if (st == OR_OK && kk < k) st = OR_RANKDEF;

    free(Qtil); free(Q); free(Y); free(Yt); free(Bt); free(U1); free(S1);
    free(V1); free(Uf);
    return st;
}

/*
 * The mixing draw for w columns derived from the draw for l >= w columns
 * (h = ceil(l/2) complex entries, h' = ceil(w/2)): the first h' phases of
 * each set, and each permutation restricted to 0..h'-1 (its entries below
 * h' in their order: the restriction of a uniform random permutation is a
 * uniform random permutation of the subset).
 */
static void restrict_mix(const double *th1, const double *th2, const i64 *p1, const i64 *p2,
                         i64 h, i64 hw, double *t1w, double *t2w, i64 *p1w, i64 *p2w)
{
    for (i64 a = 0; a < hw; a++) {
        t1w[a] = th1[a];
        t2w[a] = th2[a];
    }
    i64 c1 = 0, c2 = 0;
    for (i64 a = 0; a < h; a++) {
        if (p1[a] < hw) p1w[c1++] = p1[a];
        if (p2[a] < hw) p2w[c2++] = p2[a];
    }
}

/* Algorithm 1 or 2 on X (rows x w, ldx) with the draw restricted to w
 * columns; U (rows x w, ldu), S, V (w x w, ldv); returns the rank. */
static i64 tsqr_restricted(const double *X, i64 rows, i64 w, i64 ldx, int passes, double wp,
                           const double *th1, const double *th2, const i64 *p1, const i64 *p2,
                           i64 h, int max_sweeps, double *U, i64 ldu, double *S, double *V,
                           i64 ldv, int *st)
{
    const i64 hw = (w + 1) / 2;
    double *t1w = dalloc(hw), *t2w = dalloc(hw), *Xc = dalloc(rows * w);
    i64 *p1w = (i64 *)malloc(sizeof(i64) * (size_t)hw), *p2w = (i64 *)malloc(sizeof(i64) * (size_t)hw);
    restrict_mix(th1, th2, p1, p2, h, hw, t1w, t2w, p1w, p2w);
    for (i64 i = 0; i < rows; i++)
        for (i64 j = 0; j < w; j++) Xc[i * w + j] = X[i * ldx + j];
    double *Uc = dalloc(rows * w), *Vc = dalloc(w * w);
    i64 r = 0;
    if (or_ts_svd_tsqr(Xc, rows, w, w, passes, wp, t1w, t2w, p1w, p2w, max_sweeps, Uc, w, S, Vc,
                       w, &r) == OR_ENOCONV)
        *st = OR_ENOCONV;
    for (i64 i = 0; i < rows; i++)
        for (i64 j = 0; j < w; j++) U[i * ldu + j] = Uc[i * w + j];
    for (i64 i = 0; i < w; i++)
        for (i64 j = 0; j < w; j++) V[i * ldv + j] = Vc[i * w + j];
    free(t1w); free(t2w); free(Xc); free(p1w); free(p2w); free(Uc); free(Vc);
    return r;
}

/*
 * Algorithm 7 = Algorithm 6 fed by Algorithm 5, with Algorithm 1 for the
 * power steps and Algorithm 2 for the last step and for the SVD of B (the
 * TS-SVD of B^T = A^T Q).  As in Algorithms 1 and 2, discarded directions
 * are removed: each step continues with the basis width the previous
 * TS-SVD kept.  The mixing of every TS-SVD comes from the one draw for l
 * columns (theta1, theta2, perm1, perm2, length ceil(l/2)), restricted to
 * the current width.  Outputs as or_lowrank_svd.
 */
int or_lowrank_svd_tsqr(const double *A, i64 m, i64 n, i64 lda, i64 k, i64 l, int iters,
                        const double *Omega, const double *th1, const double *th2,
                        const i64 *p1, const i64 *p2, double wp, int max_sweeps, double *U,
                        i64 ldu, double *S, double *V, i64 ldv, i64 *rank)
{
    int st = OR_OK;
    const i64 h = (l + 1) / 2;
    double *Qt = dalloc(n * l), *Q = dalloc(m * l), *Y = dalloc(m * l), *Yt = dalloc(n * l);
    double *tS = dalloc(l), *tV = dalloc(l * l);
    i64 w = l;
    for (i64 i = 0; i < n * l; i++) Qt[i] = Omega[i];
    for (int it = 0; it < iters && w > 0; it++) {
        or_matmul(A, m, n, lda, Qt, w, w, Y, w);
        w = tsqr_restricted(Y, m, w, w, 1, wp, th1, th2, p1, p2, h, max_sweeps, Q, l, tS, tV, l,
                            &st);
        if (w == 0) break;
        /* Q (m x w) compacted to leading dimension w */
        for (i64 i = 0; i < m; i++)
            for (i64 j = 0; j < w; j++) Y[i * w + j] = Q[i * l + j];
        or_matmul_tn(A, m, n, lda, Y, w, w, Yt, w);
        const i64 w2 = tsqr_restricted(Yt, n, w, w, 1, wp, th1, th2, p1, p2, h, max_sweeps, Qt,
                                       l, tS, tV, l, &st);
        for (i64 i = 0; i < n; i++)
            for (i64 j = 0; j < w2; j++) Yt[i * w2 + j] = Qt[i * l + j];
        memcpy(Qt, Yt, sizeof(double) * (size_t)(n * w2));
        w = w2;
    }
    i64 rb = 0;
    double *Bt = dalloc(n * l), *U1 = dalloc(n * l), *S1 = dalloc(l), *V1 = dalloc(l * l);
    double *Uf = dalloc(m * l);
    if (w > 0) {
        or_matmul(A, m, n, lda, Qt, w, w, Y, w);
        const i64 wq = tsqr_restricted(Y, m, w, w, 2, wp, th1, th2, p1, p2, h, max_sweeps, Q, l,
                                       tS, tV, l, &st);
        if (wq > 0) {
            for (i64 i = 0; i < m; i++)
                for (i64 j = 0; j < wq; j++) Y[i * wq + j] = Q[i * l + j];
            /* Algorithm 6: B^T = A^T Q = U1 S1 V1^T, U~ = V1, V = U1 */
            or_matmul_tn(A, m, n, lda, Y, wq, wq, Bt, wq);
            rb = tsqr_restricted(Bt, n, wq, wq, 2, wp, th1, th2, p1, p2, h, max_sweeps, U1, l,
                                 S1, V1, l, &st);
            for (i64 i = 0; i < m; i++)
                for (i64 j = 0; j < wq; j++) {
                    double acc = 0.0;
                    for (i64 c = 0; c < wq; c++) acc += Y[i * wq + c] * V1[c * l + j];
                    Uf[i * l + j] = acc;
                }
        }
    }
    const i64 kk = k < rb ? k : rb;
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < k; j++) U[i * ldu + j] = (j < kk) ? Uf[i * l + j] : 0.0;
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < k; j++) V[i * ldv + j] = (j < kk) ? U1[i * l + j] : 0.0;
    for (i64 j = 0; j < k; j++) S[j] = (j < kk) ? S1[j] : 0.0;
    canonical_signs(U, m, ldu, V, n, ldv, kk);
    *rank = kk;
    if (st == OR_OK && kk < k) st = OR_RANKDEF;
    free(Qt); free(Q); free(Y); free(Yt); free(tS); free(tV); free(Bt); free(U1); free(S1);
    free(V1); free(Uf);
    return st;
}

/* ------------------------------------------------------------------ */
/* Thin-SVD adjoint.                                                    */
/* ------------------------------------------------------------------ */

/*
 * Gradient of a loss L(U, S, V) through the thin SVD A = U diag(S) V^T of a
 * full-column-rank A (m x n, m >= n, distinct singular values), given
 * dU = dL/dU (m x n), dS = dL/dS (n), dV = dL/dV (n x n).  This is the
 * standard adjoint of the thin SVD (Townsend 2016; Giles 2008), written
 * out term by term:
 *   F_ij = 1/(s_j^2 - s_i^2) for i != j, 0 on the diagonal,
 *   J = U^T dU, K = V^T dV,
 *   dA = U [ (F o (J - J^T)) S + diag(dS) + S (F o (K - K^T)) ] V^T
 *        + (I - U U^T) dU S^{-1} V^T
 * (the term U S^{-1} dV^T (I - V V^T) vanishes because V is square).
 * U is recomputed as A V S^{-1}, as the forward pass would return it.
 */
void or_ts_svd_backward(const double *A, i64 m, i64 n, i64 lda,
                        const double *S, const double *V, i64 ldv,
                        const double *dU, i64 lddu, const double *dS,
                        const double *dV, i64 lddv, double *dA, i64 ldda)
{
    double *U = dalloc(m * n), *J = dalloc(n * n), *K = dalloc(n * n);
    double *M = dalloc(n * n), *Vc = dalloc(n * n), *dVc = dalloc(n * n);
    double *dUc = dalloc(m * n);
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) {
            Vc[i * n + j] = V[i * ldv + j];
            dVc[i * n + j] = dV ? dV[i * lddv + j] : 0.0;
        }
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) dUc[i * n + j] = dU ? dU[i * lddu + j] : 0.0;
    /* U = A V S^{-1}. */
    or_matmul(A, m, n, lda, Vc, n, n, U, n);
    for (i64 i = 0; i < m; i++)
        for (i64 j = 0; j < n; j++) U[i * n + j] /= S[j];
    /* J = U^T dU, K = V^T dV. */
    or_matmul_tn(U, m, n, n, dUc, n, n, J, n);
    or_matmul_tn(Vc, n, n, n, dVc, n, n, K, n);
    /* Inner n x n matrix M (before the -J S^{-1} projection term). */
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) {
            double v = 0.0;
            if (i != j) {
                double F = 1.0 / (S[j] * S[j] - S[i] * S[i]);
                v += F * (J[i * n + j] - J[j * n + i]) * S[j];
                v += S[i] * F * (K[i * n + j] - K[j * n + i]);
            } else {
                v += dS ? dS[i] : 0.0;
            }
            /* (I - U U^T) dU S^{-1} V^T = dU S^{-1} V^T - U (J S^{-1}) V^T */
            v -= J[i * n + j] / S[j];
            M[i * n + j] = v;
        }
    /* dA = U (M V^T) + dU (S^{-1} V^T). */
    double *MVt = dalloc(n * n), *SVt = dalloc(n * n);
    for (i64 i = 0; i < n; i++)
        for (i64 j = 0; j < n; j++) {
            double acc = 0.0;
            for (i64 b = 0; b < n; b++) acc += M[i * n + b] * Vc[j * n + b];
            MVt[i * n + j] = acc;
            SVt[i * n + j] = Vc[j * n + i] / S[i];
        }
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < m; i++) {
        for (i64 j = 0; j < n; j++) {
            double acc = 0.0;
            for (i64 b = 0; b < n; b++)
                acc += U[i * n + b] * MVt[b * n + j] + dUc[i * n + b] * SVt[b * n + j];
            dA[i * ldda + j] = acc;
        }
    }
    free(U); free(J); free(K); free(M); free(Vc); free(dVc); free(dUc);
    free(MVt); free(SVt);
}

/*
 * Adjoint of a rank-k SVD A ~ U diag(S) V^T (the output of Algorithm 8):
 * U (m x k, ldu), S (k, distinct and positive), V (n x k, ldv), cotangents
 * dU (m x k), dS (k), dV (n x k) (NULL = zero) -> dA (m x n, ldda).  With
 * J = U^T dU, K = V^T dV and F_ab = 1/(S_b^2 - S_a^2) (a != b, F_aa = 0):
 *   dA = U [ (F o (J - J^T)) S + diag(dS) + S (F o (K - K^T)) ] V^T
 *        + (I - U U^T) dU S^{-1} V^T + U S^{-1} dV^T (I - V V^T).
 * This is the derivative of the leading k singular triplets when A has
 * rank k (the singular values past k are 0); for other A it leaves out
 * the coupling with the discarded part of the spectrum.
 */
void or_lowrank_svd_backward(const double *U, i64 m, i64 k, i64 ldu,
                             const double *S, const double *V, i64 n, i64 ldv,
                             const double *dU, i64 lddu, const double *dS,
                             const double *dV, i64 lddv, double *dA, i64 ldda)
{
    double *J = dalloc(k * k), *K = dalloc(k * k), *C = dalloc(k * k);
    double *PdU = dalloc(m * k), *PdV = dalloc(n * k);
    /* J = U^T dU, K = V^T dV */
    for (i64 a = 0; a < k; a++)
        for (i64 b = 0; b < k; b++) {
            double ja = 0.0, ka = 0.0;
            if (dU)
                for (i64 i = 0; i < m; i++) ja += U[i * ldu + a] * dU[i * lddu + b];
            if (dV)
                for (i64 i = 0; i < n; i++) ka += V[i * ldv + a] * dV[i * lddv + b];
            J[a * k + b] = ja;
            K[a * k + b] = ka;
        }
    /* the k x k core */
    for (i64 a = 0; a < k; a++)
        for (i64 b = 0; b < k; b++) {
            double v = 0.0;
            if (a != b) {
                const double F = 1.0 / (S[b] * S[b] - S[a] * S[a]);
                v += F * (J[a * k + b] - J[b * k + a]) * S[b];
                v += S[a] * F * (K[a * k + b] - K[b * k + a]);
            } else if (dS) {
                v += dS[a];
            }
            C[a * k + b] = v;
        }
    /* (I - U U^T) dU = dU - U J and (I - V V^T) dV = dV - V K */
    for (i64 i = 0; i < m; i++)
        for (i64 b = 0; b < k; b++) {
            double v = dU ? dU[i * lddu + b] : 0.0;
            for (i64 a = 0; a < k; a++) v -= U[i * ldu + a] * J[a * k + b];
            PdU[i * k + b] = v;
        }
    for (i64 i = 0; i < n; i++)
        for (i64 b = 0; b < k; b++) {
            double v = dV ? dV[i * lddv + b] : 0.0;
            for (i64 a = 0; a < k; a++) v -= V[i * ldv + a] * K[a * k + b];
            PdV[i * k + b] = v;
        }
#pragma omp parallel for schedule(static)
    for (i64 i = 0; i < m; i++) {
        double *UC = dalloc(k);
        for (i64 b = 0; b < k; b++) {
            double v = 0.0;
            for (i64 a = 0; a < k; a++) v += U[i * ldu + a] * C[a * k + b];
            UC[b] = v;
        }
        for (i64 j = 0; j < n; j++) {
            double acc = 0.0;
            for (i64 b = 0; b < k; b++)
                acc += UC[b] * V[j * ldv + b] + PdU[i * k + b] * V[j * ldv + b] / S[b] +
                       U[i * ldu + b] * PdV[j * k + b] / S[b];
            dA[i * ldda + j] = acc;
        }
        free(UC);
    }
    free(J); free(K); free(C); free(PdU); free(PdV);
}

/* ------------------------------------------------------------------ */
/* Error metrics (Table "heads").                                       */
/* ------------------------------------------------------------------ */

/* MaxEntry(|U^T U - I|) over the first r columns of U (m x r, ldu). */
double or_orth_error(const double *U, i64 m, i64 r, i64 ldu)
{
    double *G = dalloc(r * r);
    or_gram(U, m, r, ldu, G, r);
    double e = 0.0;
    for (i64 i = 0; i < r; i++)
        for (i64 j = 0; j < r; j++) {
            double v = fabs(G[i * r + j] - (i == j ? 1.0 : 0.0));
            if (v > e) e = v;
        }
    free(G);
    return e;
}

/* Simple splitmix64 stream for the power method's starting vector. */
static uint64_t sm64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/*
 * Spectral norm of E = A - U diag(S) V^T (A m x n; U m x r; V n x r) by
 * `iters` steps of the power method on E^T E, from a seeded start, without
 * forming E (the paper uses 20 steps for its tables).
 */
double or_spectral_error(const double *A, i64 m, i64 n, i64 lda,
                         const double *U, i64 ldu, const double *S,
                         const double *V, i64 ldv, i64 r, int iters,
                         uint64_t seed)
{
    double *x = dalloc(n), *y = dalloc(m), *t = dalloc(r);
    uint64_t st = seed;
    for (i64 i = 0; i < n; i++)
        x[i] = (double)(sm64(&st) >> 11) * ldexp(1.0, -53) - 0.5;
    double est = 0.0;
    for (int it = 0; it < iters; it++) {
        double nx = 0.0;
        for (i64 i = 0; i < n; i++) nx += x[i] * x[i];
        nx = sqrt(nx);
        if (nx == 0.0) return 0.0;
        for (i64 i = 0; i < n; i++) x[i] /= nx;
        /* y = E x = A x - U (S (V^T x)) */
        for (i64 j = 0; j < r; j++) {
            double acc = 0.0;
            for (i64 i = 0; i < n; i++) acc += V[i * ldv + j] * x[i];
            t[j] = S[j] * acc;
        }
#pragma omp parallel for schedule(static)
        for (i64 i = 0; i < m; i++) {
            double acc = 0.0;
            for (i64 j = 0; j < n; j++) acc += A[i * lda + j] * x[j];
            for (i64 j = 0; j < r; j++) acc -= U[i * ldu + j] * t[j];
            y[i] = acc;
        }
        double ny = 0.0;
        for (i64 i = 0; i < m; i++) ny += y[i] * y[i];
        est = sqrt(ny);
        /* x = E^T y = A^T y - V (S (U^T y)) */
        for (i64 j = 0; j < r; j++) {
            double acc = 0.0;
            for (i64 i = 0; i < m; i++) acc += U[i * ldu + j] * y[i];
            t[j] = S[j] * acc;
        }
#pragma omp parallel for schedule(static)
        for (i64 i = 0; i < n; i++) {
            double acc = 0.0;
            for (i64 k = 0; k < m; k++) acc += A[k * lda + i] * y[k];
            for (i64 j = 0; j < r; j++) acc -= V[i * ldv + j] * t[j];
            x[i] = acc;
        }
    }
    free(x);
    free(y);
    free(t);
    return est;
}
