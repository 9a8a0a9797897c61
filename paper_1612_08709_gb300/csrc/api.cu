// C ABI entry points and the host-side orchestration of each call.
//
// Every step of a call is a kernel queued on the caller's stream; the host
// only validates arguments, carves the workspace and, at the end, reads the
// device status block back (one small device-to-host copy and a stream
// synchronisation).  Column discards never change array shapes: a dropped
// column is carried as a zero column with a zero inverse norm, which the
// Jacobi solves leave untouched (its inner products are exactly zero) and
// which sorts last, so no host round trip is needed between passes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace tssvd {

int num_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

namespace {

// ---------------------------------------------------------------- workspace

// Bump allocator over a device buffer.  In sizing mode (base == nullptr)
// it only accumulates the bytes a call would take.
struct Bump {
    char *base;
    size_t off;
    size_t cap;
    bool overflow;
    explicit Bump(void *b, size_t c) : base((char *)b), off(0), cap(c), overflow(false) {}
    template <typename T>
    T *take(size_t count)
    {
        // 256-byte aligned absolute addresses, whatever the base
        const size_t addr = ((size_t)base + off + 255) & ~(size_t)255;
        off = addr - (size_t)base;
        T *p = nullptr;
        if (base) {
            if (off + count * sizeof(T) > cap)
                overflow = true;
            else
                p = (T *)(base + off);
        }
        off += count * sizeof(T);
        return p;
    }
    bool sizing() const { return base == nullptr; }
};

// The internal workspace: one growable buffer per device, used when the
// caller passes none.  Calls that use it hold the lock for their duration.
struct InternalWs {
    std::mutex mu;
    void *ptr = nullptr;
    size_t bytes = 0;
};
InternalWs g_ws[64];

#define CK(...)                                \
    do {                                       \
        cudaError_t e_ = (__VA_ARGS__);        \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)

// ------------------------------------------------------ row-sharded calls

// Set when the caller's all-reduce fails inside a row-sharded call (the
// entry point turns it into TSSVD_ECOMM).
thread_local int t_comm_failed = 0;

// The caller's all-reduce of a device array (a no-op without a collective).
cudaError_t comm_allreduce(const tssvd_comm *c, void *buf, i64 count, int dtype, int op,
                           cudaStream_t s)
{
    if (!c || !c->allreduce) return cudaSuccess;
    if (c->allreduce(buf, (int64_t)count, dtype, op, (void *)s, c->ctx) != 0) {
        t_comm_failed = 1;
        return cudaErrorUnknown;
    }
    return cudaSuccess;
}

// Explicit column norms from per-block sums of squares NP (g x N): local
// sums, summed over the ranks, then the square roots.  Without a collective
// it is launch_norms_reduce (same arithmetic, one kernel).
cudaError_t shard_norms(const tssvd_comm *c, const double *NP, int g, i64 N, double *out,
                        cudaStream_t s)
{
    if (!c || !c->allreduce) return launch_norms_reduce(NP, g, N, out, s);
    CK(launch_sumsq_reduce(NP, g, N, out, s));
    CK(comm_allreduce(c, out, N, TSSVD_DT_F64, TSSVD_OP_SUM, s));
    return launch_sqrt_inplace(out, N, s);
}

// ------------------------------------------------------------ TS-SVD core

// Enqueues Algorithm 3 (passes == 1) or Algorithm 4 (passes == 2; passes ==
// 3 runs its second pass twice) on A
// (m x n, lda, type T).  Writes U (m x n, ldu, type T), S (n) and V (n x n,
// row-major, ldv) as doubles or T per the template parameters; all outputs
// carry zeros past the numerical rank.  In sizing mode only the workspace
// is counted.
inline int mode_terms(int mode) { return mode == TSSVD_BF16X6 ? 3 : (mode == TSSVD_BF16X3 ? 2 : 0); }


// The first Gram eigensolve of Algorithm 4, B = V~ D~ V~^T (B consumed),
// accurate to the FP64 rounding already in B (the second pass repairs the
// rest), for a B formed with FP64-accurate products.
// For n <= kPcholGridMaxN: pivoted Cholesky P^T B P = R^T R over the whole
// grid with logical pivoting (launch_pchol_grid: X = (R P^T)^T, nothing to
// un-pivot), one-sided Jacobi on the columns of X without accumulating
// the rotations (threshold 2^-51: the columns come out orthogonal to
// rounding), whose normalised columns, sorted by norm, are the
// eigenvectors: B = X X^T = (X K)(X K)^T with X K = W Sigma gives
// B = W Sigma^2 W^T.  On a graded B this converges in a third of the
// sweeps of the Gram-form solver (13 sweeps instead of 37 on 1,000,000 x
// 1,000 with sigma 1 .. 1e-8).  The grid factorization replaced the
// single-CTA one here (2.9 -> 1.1 ms at n = 200); the single-CTA one
// serves the batched solves.  For n >= kJacobiMixedMinN the Jacobi solve
// starts with the FP32 phase.  Larger n: Gram-form Jacobi with the
// normwise floor.  Scratch: Xw, Jw, B2, Xn (n x n), norms, lam (n), perm,
// piv (n ints).
static cudaError_t first_eig(double *B, double *B2, i64 n, double *Xw, double *Jw, double *Xn,
                             double *lam, double *norms, double *Vt, int max_sweeps, int *ctr,
                             double *prm, int *perm, int *piv, DevStatus *st, cudaStream_t s,
                             const JacobiMixedScratch &mw)
{
    if (n <= kPcholGridMaxN) {
        CK(launch_pchol_grid(B, (int)n, Xw, n, (unsigned long long *)prm, st, s));
        if (jacobi_mixed_applies(n))
            CK(launch_jacobi_mixed(Xw, n, nullptr, mw, max_sweeps, ctr, prm, st, 0, s, 0x1p-51));
        else
            CK(launch_jacobi(Xw, n, nullptr, n, (int)n, (int)n, max_sweeps, ctr, prm, st, 0, s,
                             0x1p-51));
        return launch_jacobi_finalize(Xw, n, nullptr, n, (int)n, (int)n, norms, perm, nullptr, n,
                                      lam, Vt, n, s);
    }
    return launch_jacobi_eig(B, B2, n, Jw, n, lam, Vt, n, (int)n, max_sweeps, ctr, prm, perm, st, 0,
                             s, true);
}

// The second eigensolve of Algorithm 4, Z = W D W^T (Z consumed), with
// the relative rotation test (W must diagonalise Z to working precision:
// it sets the orthonormality of Q).  For kPcholMaxN < n <=
// kPcholGridMaxN: Z = R~^T R~ by the grid pivoted Cholesky (Z is well
// conditioned: the first pass leaves Y with a condition number near 10),
// then the two-precision one-sided Jacobi on R~^T without accumulation;
// the orthogonalised columns, normalised, are the eigenvectors.  Its FP64
// sweeps cost 3.5 n^2 operations a round against the Gram-form solver's
// 6 n^2, and the FP32 phase takes the first few orders of magnitude.
// Otherwise the Gram-form solver (at n <= 256 its two rounds a barrier
// keep it the faster one).
static cudaError_t second_eig(double *Z, double *Z2, i64 n, double *Xw, double *Jw, double *lam,
                              double *norms, double *W, int max_sweeps, int *ctr, double *prm,
                              int *perm, int *piv, DevStatus *st, cudaStream_t s,
                              const JacobiMixedScratch &mw)
{
    if (n > kPcholMaxN && jacobi_mixed_applies(n) && n <= kPcholGridMaxN) {
        CK(launch_pchol_grid(Z, (int)n, Xw, n, (unsigned long long *)prm, st, s));
        CK(launch_jacobi_mixed(Xw, n, nullptr, mw, max_sweeps, ctr, prm, st, 1, s));
        return launch_jacobi_finalize(Xw, n, nullptr, n, (int)n, (int)n, norms, perm, nullptr, n,
                                      lam, W, n, s);
    }
    return launch_jacobi_eig(Z, Z2, n, Jw, n, lam, W, n, (int)n, max_sweeps, ctr, prm, perm, st, 1,
                             s);
}

// The small SVD of Algorithm 4, R = P Sigma V^T (R n x n row-major), by
// one-sided Jacobi on the columns of R^T, or of R when the MaxEntry scaling
// D is strongly graded (the device flag st->orient set by
// launch_orient_copy: column grading is what the one-sided method handles
// accurately).  Outputs Pm (P), sigma, Vo (V), sorted.
static cudaError_t final_svd(double *R, i64 n, const double *d, double *Xw, double *Jw,
                             double *norms, double *Pm, double *sigma, double *Vo, int max_sweeps,
                             int *ctr, double *prm, int *perm, DevStatus *st, cudaStream_t s,
                             const JacobiMixedScratch &mw)
{
    CK(launch_orient_copy(d, &st->rank2, R, n, Xw, &st->orient, s));
    if (jacobi_mixed_applies(n))
        CK(launch_jacobi_mixed(Xw, n, Jw, mw, max_sweeps, ctr, prm, st, 2, s));
    else
        CK(launch_jacobi(Xw, n, Jw, n, (int)n, (int)n, max_sweeps, ctr, prm, st, 2, s));
    return launch_jacobi_finalize(Xw, n, Jw, n, (int)n, (int)n, norms, perm, Pm, n, sigma, Vo, n,
                                  s, &st->orient, prm);
}

template <typename T, typename TO>
cudaError_t ts_core(const T *A, i64 m, i64 n, i64 lda, TO *U, i64 ldu, TO *S, TO *V, i64 ldv,
                    int passes, int scale, double tol, int max_sweeps, Bump &ws, DevStatus *st,
                    cudaStream_t s, const tssvd_comm *comm = nullptr)
{
    const bool sizing = ws.sizing();
    const i64 nn = n * n;
    int *ctr = ws.take<int>((size_t)max_sweeps + 4);
    unsigned long long *bits = ws.take<unsigned long long>(n);
    double *d = ws.take<double>(n), *dinv = ws.take<double>(n);
    const int sp1 = tn_splits(m, n, n, true);
    const int sp2 = tn_splits(n, n, n, false);
    const int sp = sp1 > sp2 ? sp1 : sp2;
    double *P = ws.take<double>((size_t)sp * nn);
    const int gy = nn_grid_rows(m, n);
    double *NP = ws.take<double>((size_t)gy * n);
    double *B = ws.take<double>(nn), *Xw = ws.take<double>(nn), *Jw = ws.take<double>(nn);
    double *Vt = ws.take<double>(nn), *W = ws.take<double>(nn), *M = ws.take<double>(nn);
    double *G = ws.take<double>(nn), *R = ws.take<double>(nn), *Pm = ws.take<double>(nn);
    double *Vo = ws.take<double>(nn), *Pp = ws.take<double>(nn), *M3 = ws.take<double>(nn);
    double *lam = ws.take<double>(n), *sig = ws.take<double>(n), *sinv = ws.take<double>(n);
    double *Tn = ws.take<double>(n), *tinv = ws.take<double>(n), *Tk = ws.take<double>(n);
    double *sgn = ws.take<double>(n), *norms = ws.take<double>(n), *sigma = ws.take<double>(n);
    double *cs = ws.take<double>(n);
    int *perm = ws.take<int>(n), *piv = ws.take<int>(n);
    double *prm = ws.take<double>(jacobi_prm_doubles(n));
    double *B2 = ws.take<double>(nn);
    double *Yt = (passes >= 2) ? ws.take<double>((size_t)m * n) : nullptr;
    // Q~ of the second pass, the third pass's input
    double *Q2 = (passes == 3) ? ws.take<double>((size_t)m * n) : nullptr;
    if (sizing) return cudaSuccess;
    if (ws.overflow) return cudaErrorMemoryAllocation;

    if (passes == 1) {
        // ---- Algorithm 3 ----
        // B = A^T A.
        CK(launch_tn_partial<T, T>(A, lda, A, lda, m, n, n, sp1, true, P, s));
        CK(launch_tn_reduce(P, sp1, n, n, nullptr, nullptr, true, B, n, s));
        CK(comm_allreduce(comm, B, nn, TSSVD_DT_F64, TSSVD_OP_SUM, s));
        // B = V D V^T (Gram-form Jacobi; B is rotated in place).
        CK(launch_jacobi_eig(B, B2, n, Jw, n, lam, Vt, n, (int)n, max_sweeps, ctr, prm, perm, st, 0,
                             s));
        // U~ = A V, Sigma = explicit column norms of U~ (Remark "normalizing").
        CK(launch_nn<T, TO>(A, lda, Vt, n, m, n, n, U, ldu, NP, s));
        CK(shard_norms(comm, NP, gy, n, sig, s));
        // Discard, U = U~ Sigma^{-1}, sign convention.
        CK(launch_discard(sig, n, tol, sinv, &st->rank1, s));
        CK(launch_scale2(Vt, n, n, n, nullptr, nullptr, Vo, n, s));
        CK(launch_signs(Vo, n, n, n, sinv, sgn, s));
        CK(launch_scale2(sinv, n, 1, n, nullptr, sgn, cs, n, s));
        CK(launch_scale_cols_inplace<TO>(U, ldu, m, n, cs, s));
        CK(launch_keepval(sig, sinv, n, sigma, s));
        CK(launch_count_positive(sigma, n, &st->rank, s));
        CK(launch_convert<TO>(sigma, n, 1, n, S, n, s));
        CK(launch_convert<TO>(Vo, n, n, n, V, ldv, s));
        return cudaSuccess;
    }

    // ---- Algorithm 4 ----
    const double *rs1 = nullptr;
    const double *M1 = Vt;
    if (scale) {
        // MaxEntry column scaling D (powers of two, so exact).
        CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s));
        CK(launch_colmax<T>(A, m, n, lda, bits, s));
        CK(comm_allreduce(comm, bits, n, TSSVD_DT_U64, TSSVD_OP_MAX, s));
        CK(launch_pow2_scale(bits, n, d, dinv, s));
        rs1 = dinv;
    }
    // B = (A D^-1)^T (A D^-1).
    CK(launch_tn_partial<T, T>(A, lda, A, lda, m, n, n, sp1, true, P, s));
    CK(launch_tn_reduce(P, sp1, n, n, rs1, rs1, true, B, n, s));
    CK(comm_allreduce(comm, B, nn, TSSVD_DT_F64, TSSVD_OP_SUM, s));
    // B = V~ D~ V~^T (B consumed).
    CK(first_eig(B, B2, n, Xw, Jw, Pm, lam, norms, Vt, max_sweeps, ctr, prm, perm, piv, st, s,
                 JacobiMixedScratch{B2, Jw, W, G, R, P, NP}));
    // Y~ = (A D^-1) V~ = A (D^-1 V~); Sigma~ = explicit column norms.
    if (scale) {
        CK(launch_scale2(Vt, n, n, n, dinv, nullptr, M, n, s));
        M1 = M;
    }
    CK(launch_nn<T, double>(A, lda, M1, n, m, n, n, Yt, n, NP, s));
    CK(shard_norms(comm, NP, gy, n, sig, s));
    // Discard; Y = Y~ Sigma~^{-1} is kept implicit: sinv scales the next
    // products instead of a separate pass over Y.
    CK(launch_discard(sig, n, tol, sinv, &st->rank1, s));
    // R = T W^T Sigma~ V~^T D is built from G = Sigma~ V~^T D.
    CK(launch_build_g(sig, sinv, Vt, n, scale ? d : nullptr, n, G, s));

    // The second orthonormalisation pass on Y = Yin diag(cin); with
    // passes = 3 once more on the second pass's Q = Q~ T^-1 (Q~ written
    // out, T its explicit column norms): Yin = Q~, cin = T^-1 (zero for
    // the columns the second pass dropped), and R <- T3 W3^T R, since
    // Q = Q3 T3 W3^T.
    const double *Yin = Yt;
    const double *cin = sinv;
    for (int pass = 2; pass <= passes; ++pass) {
        const bool last = pass == passes;
        // Z = Y^T Y = diag(cin) (Yin^T Yin) diag(cin).
        CK(launch_tn_partial<double, double>(Yin, n, Yin, n, m, n, n, sp1, true, P, s));
        CK(launch_tn_reduce(P, sp1, n, n, cin, cin, true, B, n, s));
        CK(comm_allreduce(comm, B, nn, TSSVD_DT_F64, TSSVD_OP_SUM, s));
        // Z = W D W^T.
        CK(second_eig(B, B2, n, Xw, Jw, lam, norms, W, max_sweeps, ctr, prm, perm, piv, st, s,
                      JacobiMixedScratch{B2, Jw, M3, Pm, Vo, P, NP}));
        // Q~ = Y W = Yin (diag(cin) W); T = explicit column norms of Q~
        // (Q~ itself is written out only when another pass reads it).
        CK(launch_scale2(W, n, n, n, cin, nullptr, M, n, s));
        CK(launch_nn<double, double>(Yin, n, M, n, m, n, n, last ? (double *)nullptr : Q2,
                                     last ? 0 : n, NP, s));
        CK(shard_norms(comm, NP, gy, n, Tn, s));
        CK(launch_discard(Tn, n, tol, tinv, &st->rank2, s));
        CK(launch_keepval(Tn, tinv, n, Tk, s));
        // R = T W^T G (G = Sigma~ V~^T D in the second pass, the previous
        // R in the third)
        CK(launch_tn_partial<double, double>(W, n, pass == 2 ? G : R, n, n, n, n, sp2, false, P,
                                             s));
        CK(launch_tn_reduce(P, sp2, n, n, Tk, nullptr, false, R, n, s));
        if (!last) {
            Yin = Q2;
            cin = tinv;
        }
    }
    // R = P Sigma V^T by one-sided Jacobi (final_svd): on the columns of
    // R^T (R row-major = R^T column-major: R^T P = X, Sigma = column norms,
    // V = X Sigma^-1), or of R when the MaxEntry scaling is strongly graded
    // (the device-side flag st->orient routes the outputs).
    CK(final_svd(R, n, scale ? d : nullptr, Xw, Jw, norms, Pm, sigma, Vo, max_sweeps, ctr, prm,
                 perm, st, s, JacobiMixedScratch{B, B2, M3, G, W, P, NP}));
    CK(launch_signs(Vo, n, n, n, sigma, sgn, s));
    CK(launch_count_positive(sigma, n, &st->rank, s));
    // U = Q P = Yin (diag(cin) W T^-1 P diag(sgn)) with the last pass's
    // input, M = diag(cin) W and T.
    CK(launch_scale2(Pm, n, n, n, tinv, sgn, Pp, n, s));
    CK(launch_nn<double, double>(M, n, Pp, n, n, n, n, M3, n, NP, s));
    CK(launch_nn<double, TO>(Yin, n, M3, n, m, n, n, U, ldu, NP, s));
    CK(launch_convert<TO>(sigma, n, 1, n, S, n, s));
    CK(launch_convert<TO>(Vo, n, n, n, V, ldv, s));
    return cudaSuccess;
}

// Host-buffer form (ts_svd_host): A's rows arrive in chunks of `rows` rows
// (a multiple of 128; the last chunk may be shorter) on a copy stream, chunk
// k signalled by arrived[k]; U leaves in the same chunks on the stream
// `out` (ready[k] recorded on the compute stream after chunk k's product).
struct HostIO {
    int chunks;
    i64 rows;
    cudaEvent_t *arrived, *ready;
    double *U_host;
    i64 ldu_host;
    cudaStream_t out;
};

inline i64 io_rows(const HostIO *io, i64 m, int k)
{
    const i64 r0 = (i64)k * io->rows;
    return std::min(io->rows, m - r0);
}

// The FP64-accurate tensor-core form: the same steps as ts_core, with every
// tall product on the digit-sliced tensor-core kernels.
template <typename T, typename TO>
cudaError_t ts_core_oz(const T *A, i64 m, i64 n, i64 lda, TO *U, i64 ldu, TO *S, TO *V, i64 ldv,
                       int passes, int scale, double tol, int max_sweeps, Bump &ws, DevStatus *st,
                       cudaStream_t s, const tssvd_comm *comm = nullptr, int terms = 0,
                       const HostIO *io = nullptr)
{
    // terms > 0 (the BF16-split modes, two or three passes, n <= 256): the
    // first pass's two products (Gram of A, A V~) are BF16-split
    // tensor-core products with that many bf16 terms a value; the later
    // passes and the final U stay FP64-accurate (digit products).
    if (passes < 2) terms = 0;
    const bool sizing = ws.sizing();
    const i64 nn = n * n;
    int *ctr = ws.take<int>((size_t)max_sweeps + 4);
    unsigned long long *bits = ws.take<unsigned long long>(n);
    double *d = ws.take<double>(n), *dinv = ws.take<double>(n);
    int *exA = ws.take<int>(n), *pk1 = ws.take<int>(n), *exY = ws.take<int>(n);
    int *pk2 = ws.take<int>(n), *em = ws.take<int>(n);
    int *er = ws.take<int>(m);
    // (host-buffer form: two passes, digit products only)
    if (passes < 2 || terms || comm) io = nullptr;
    const int osp = oz_gram_splits(m, (int)n);
    const int sp2 = tn_splits(n, n, n, false);
    int osp_io = 0;  // the chunks' Gram partials, side by side
    if (io)
        for (int k = 0; k < io->chunks; k++) osp_io += oz_gram_splits(io_rows(io, m, k), (int)n);
    double *P = ws.take<double>((size_t)std::max(std::max(osp, sp2), osp_io) * nn);
    unsigned long long *bitsk = io ? ws.take<unsigned long long>(n) : nullptr;
    const int gcs = colsumsq_rows(m, n);
    const int gys = nn_grid_rows(n, n);
    // column maxima of Y~ from the digit product's epilogue
    const bool fuse = !terms && oz_nn_fuses((int)n);
    double *NP = ws.take<double>((size_t)(gcs > gys ? gcs : gys) * n);
    uint8_t *img = ws.take<uint8_t>(oz_image_bytes((int)n, (int)n));
    double *B = ws.take<double>(nn), *G2 = ws.take<double>(nn), *Jw = ws.take<double>(nn);
    double *Vt = ws.take<double>(nn), *W = ws.take<double>(nn), *M = ws.take<double>(nn);
    double *G = ws.take<double>(nn), *R = ws.take<double>(nn), *Pm = ws.take<double>(nn);
    double *Vo = ws.take<double>(nn), *Pp = ws.take<double>(nn), *M3 = ws.take<double>(nn);
    double *Xw = ws.take<double>(nn);
    double *lam = ws.take<double>(n), *sig = ws.take<double>(n), *sinv = ws.take<double>(n);
    double *Tn = ws.take<double>(n), *tinv = ws.take<double>(n), *Tk = ws.take<double>(n);
    double *sgn = ws.take<double>(n), *norms = ws.take<double>(n), *sigma = ws.take<double>(n);
    double *cs = ws.take<double>(n);
    int *perm = ws.take<int>(n), *piv = ws.take<int>(n);
    double *prm = ws.take<double>(jacobi_prm_doubles(n));
    double *B2 = ws.take<double>(nn);
    double *Yt = ws.take<double>((size_t)m * n);
    const size_t gib = oz_gram_image_bytes(m, (int)n), rib = oz_row_image_bytes(m, (int)n);
    uint8_t *big = ws.take<uint8_t>(gib > rib ? gib : rib);  // digit images of the tall operand
    const bool u_is_double = sizeof(TO) == sizeof(double);
    double *Qt = (passes >= 2 && !u_is_double) ? ws.take<double>((size_t)m * n) : nullptr;
    const int tsp = terms ? tc_gram_splits(m) : 0;
    double *Ptc = terms ? ws.take<double>((size_t)tsp * nn) : nullptr;
    uint8_t *Bimg = terms ? ws.take<uint8_t>(tc_split_b_bytes((int)n, (int)n, terms)) : nullptr;
    if (sizing) return cudaSuccess;
    if (ws.overflow) return cudaErrorMemoryAllocation;

    // MaxEntry of every column: the Gram's digit scales (and D when scaling)
    CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s));
    int osp_used = osp;
    if (io) {
        // A's chunks as they arrive: each chunk's column maxima (the running
        // maxima for D, the chunk's own for its digit scales: any bound at
        // or above the chunk's values serves) and its Gram partials
        osp_used = 0;
        for (int k = 0; k < io->chunks; k++) {
            const i64 r0 = (i64)k * io->rows, rk = io_rows(io, m, k);
            CK(cudaStreamWaitEvent(s, io->arrived[k], 0));
            CK(cudaMemsetAsync(bitsk, 0, sizeof(unsigned long long) * n, s));
            CK(launch_colmax<T>(A + r0 * lda, rk, n, lda, bitsk, s));
            CK(launch_bits_max(bits, bitsk, n, s));
            CK(launch_oz_exp_from_bits(bitsk, (int)n, exY, s));
            const int ok = oz_gram_splits(rk, (int)n);
            CK(launch_oz_gram<T>(A + r0 * lda, lda, rk, (int)n, exY, ok, big,
                                 P + (size_t)osp_used * nn, st, s));
            osp_used += ok;
        }
    } else {
        CK(launch_colmax<T>(A, m, n, lda, bits, s));
    }
    CK(comm_allreduce(comm, bits, n, TSSVD_DT_U64, TSSVD_OP_MAX, s));
    CK(launch_oz_exp_from_bits(bits, (int)n, exA, s));
    const bool sc = (passes >= 2) && scale;
    const double *rs1 = nullptr;
    const int *pkA = nullptr;
    if (sc) {
        CK(launch_pow2_scale(bits, n, d, dinv, s));
        CK(launch_neg_int(exA, (int)n, pk1, s));
        rs1 = dinv;
        pkA = pk1;
    }
    // B = (A D^-1)^T (A D^-1)
    if (terms) {
        CK(launch_tc_gram<T>(A, lda, m, (int)n, terms, tsp, Ptc, st, s));
        CK(launch_tn_reduce(Ptc, tsp, n, n, rs1, rs1, true, B, n, s));
    } else {
        if (!io) CK(launch_oz_gram<T>(A, lda, m, (int)n, exA, osp, big, P, st, s));
        // A's row image for Y~ = A (D^-1 V~) (A's columns prescaled by D^-1
        // for the digit scales; the product is unchanged).  Building the
        // row images beside the Jacobi kernels on a second stream was tried
        // and slowed the latency-bound solves 2.5x (L2 and issue contention).
        CK(launch_oz_rowexp<T>(A, lda, m, (int)n, pkA, er, s));
        CK(launch_oz_row_image<T>(A, lda, m, (int)n, pkA, er, big, s));
        CK(launch_tn_reduce(P, osp_used, n, n, rs1, rs1, true, B, n, s));
    }
    CK(comm_allreduce(comm, B, nn, TSSVD_DT_F64, TSSVD_OP_SUM, s));
    // B = V~ D~ V~^T (to B's rounding for Algorithm 4, relative for Algorithm
    // 3).  A B from split products carries errors far above its FP64
    // rounding, the floor the Cholesky form assumes: it takes the Gram-form
    // solver with the normwise floor.
    if (terms)
        CK(launch_jacobi_eig(B, B2, n, Jw, n, lam, Vt, n, (int)n, max_sweeps, ctr, prm, perm, st, 0,
                             s, true));
    else if (passes >= 2)
        CK(first_eig(B, B2, n, Xw, Jw, Pm, lam, norms, Vt, max_sweeps, ctr, prm, perm, piv, st, s,
                     JacobiMixedScratch{B2, Jw, W, G, R, P, NP}));
    else
        CK(launch_jacobi_eig(B, B2, n, Jw, n, lam, Vt, n, (int)n, max_sweeps, ctr, prm, perm, st, 0,
                             s));
    const double *M1 = Vt;
    if (sc) {
        CK(launch_scale2(Vt, n, n, n, dinv, nullptr, M, n, s));
        M1 = M;
    }
    if (terms) {
        // Y~ = A (D^-1 V~) by the split product (A itself, unscaled)
        CK(launch_tc_split_b(M1, n, (int)n, (int)n, terms, Bimg, s));
        CK(launch_tc_nn<T>(A, lda, m, (int)n, Bimg, (int)n, terms, Yt, n, st, s));
    } else {
        CK(launch_oz_image(M1, n, (int)n, (int)n, pkA, em, img, s));
        // Y~, with its column maxima (the next Gram's digit scales) taken in
        // the product's epilogue
        if (fuse) CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s));
        CK(launch_oz_nn_run<double>(big, m, (int)n, er, img, em, (int)n, Yt, n, st, s,
                                    fuse ? bits : nullptr, nullptr));
    }

    if (passes == 1) {
        // Sigma = explicit column norms; U = U~ Sigma^-1 with the sign convention
        CK(launch_colsumsq(Yt, n, m, n, NP, s));
        CK(shard_norms(comm, NP, gcs, n, sig, s));
        CK(launch_discard(sig, n, tol, sinv, &st->rank1, s));
        CK(launch_scale2(Vt, n, n, n, nullptr, nullptr, Vo, n, s));
        CK(launch_signs(Vo, n, n, n, sinv, sgn, s));
        CK(launch_scale2(sinv, n, 1, n, nullptr, sgn, cs, n, s));
        CK(launch_convert<TO>(Yt, n, m, n, U, ldu, s));
        CK(launch_scale_cols_inplace<TO>(U, ldu, m, n, cs, s));
        CK(launch_keepval(sig, sinv, n, sigma, s));
        CK(launch_count_positive(sigma, n, &st->rank, s));
        CK(launch_convert<TO>(sigma, n, 1, n, S, n, s));
        CK(launch_convert<TO>(Vo, n, n, n, V, ldv, s));
        return cudaSuccess;
    }

    // The second orthonormalisation pass on Y = Yin diag(cin); with
    // passes = 3 once more on the second pass's Q = Q~ T^-1: Yin = Q~
    // (written out), cin = T^-1 (zero for the columns the second pass
    // dropped) and R <- T3 W3^T R, since Q = Q3 T3 W3^T.  In the second
    // pass cin = Sigma~^-1 from the diagonal of Y~'s Gram matrix.
    double *Qb = u_is_double ? (double *)U : Qt;
    const i64 ldq = u_is_double ? ldu : n;
    const double *Yin = Yt;
    i64 ldy = n;
    const double *cin = sinv;
    bool have_bits = fuse;  // column maxima of Yin from the producing product
    for (int pass = 2; pass <= passes; ++pass) {
        const bool last = pass == passes;
        // Gram of Yin on the digit kernels (the local column maxima of Yin
        // set the digit scales: any bound on the local values serves)
        if (!have_bits) {
            CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s));
            CK(launch_colmax<double>(Yin, m, n, ldy, bits, s));
        }
        CK(launch_oz_exp_from_bits(bits, (int)n, exY, s));
        CK(launch_oz_gram<double>(Yin, ldy, m, (int)n, exY, osp, big, P, st, s));
        CK(launch_tn_reduce(P, osp, n, n, nullptr, nullptr, true, G2, n, s));
        CK(comm_allreduce(comm, G2, nn, TSSVD_DT_F64, TSSVD_OP_SUM, s));
        if (pass == 2) {
            CK(launch_diag_sqrt(G2, n, n, sig, s));
            CK(launch_discard(sig, n, tol, sinv, &st->rank1, s));
        }
        // Yin's row image for Q~ = Y W = (Yin 2^pk2) (2^-pk2 diag(cin) W)
        // and, in the last pass, for the final U (both prescaled by pk2 =
        // round(log2 cin))
        CK(launch_oz_pow2_of(cin, (int)n, pk2, s));
        CK(launch_oz_rowexp<double>(Yin, ldy, m, (int)n, pk2, er, s));
        CK(launch_oz_row_image<double>(Yin, ldy, m, (int)n, pk2, er, big, s));
        CK(launch_scale2(G2, n, n, n, cin, cin, B, n, s));
        // Z = W D W^T
        CK(second_eig(B, B2, n, Xw, Jw, lam, norms, W, max_sweeps, ctr, prm, perm, piv, st, s,
                      JacobiMixedScratch{B2, Jw, M3, Pm, Vo, P, NP}));
        // Q~; T = explicit column norms (the column sums of squares are a
        // separate pass: in the product's epilogue their FP64 FMAs cost
        // more than the pass they save).  Q~ goes to U's storage (or Qt);
        // a third pass reads it, and its own Q~ (norms only) goes to Yt.
        CK(launch_scale2(W, n, n, n, cin, nullptr, M, n, s));
        CK(launch_oz_image(M, n, (int)n, (int)n, pk2, em, img, s));
        double *Qo = (Yin == Yt) ? Qb : Yt;
        const i64 ldo = (Yin == Yt) ? ldq : n;
        have_bits = fuse && !last;
        if (have_bits) CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s));
        CK(launch_oz_nn_run<double>(big, m, (int)n, er, img, em, (int)n, Qo, ldo, st, s,
                                    have_bits ? bits : nullptr, nullptr));
        CK(launch_colsumsq(Qo, ldo, m, n, NP, s));
        CK(shard_norms(comm, NP, gcs, n, Tn, s));
        CK(launch_discard(Tn, n, tol, tinv, &st->rank2, s));
        CK(launch_keepval(Tn, tinv, n, Tk, s));
        // R = T W^T Sigma~ V~^T D (second pass), R <- T W^T R (third)
        if (pass == 2) CK(launch_build_g(sig, sinv, Vt, n, sc ? d : nullptr, n, G, s));
        CK(launch_tn_partial<double, double>(W, n, pass == 2 ? G : R, n, n, n, n, sp2, false, P,
                                             s));
        CK(launch_tn_reduce(P, sp2, n, n, Tk, nullptr, false, R, n, s));
        if (!last) {
            Yin = Qo;
            ldy = ldo;
            cin = tinv;
        }
    }
    CK(final_svd(R, n, sc ? d : nullptr, Xw, Jw, norms, Pm, sigma, Vo, max_sweeps, ctr, prm, perm,
                 st, s, JacobiMixedScratch{B, B2, M3, G, W, P, NP}));
    CK(launch_signs(Vo, n, n, n, sigma, sgn, s));
    CK(launch_count_positive(sigma, n, &st->rank, s));
    // U = Yin (diag(cin) W T^-1 P diag(sgn)) with the last pass's input,
    // prescaled like that pass's Q~ (Yin's row image is still in place)
    CK(launch_scale2(Pm, n, n, n, tinv, sgn, Pp, n, s));
    CK(launch_nn<double, double>(M, n, Pp, n, n, n, n, M3, n, NP, s));
    CK(launch_oz_image(M3, n, (int)n, (int)n, pk2, em, img, s));
    if (io) {
        // U by row chunks, each copied out while the next is computed (the
        // row image is stored by 128-row tiles)
        const size_t tile_bytes = oz_row_image_bytes(128, (int)n);
        for (int k = 0; k < io->chunks; k++) {
            const i64 r0 = (i64)k * io->rows, rk = io_rows(io, m, k);
            CK(launch_oz_nn_run<TO>(big + (size_t)(r0 / 128) * tile_bytes, rk, (int)n, er + r0,
                                    img, em, (int)n, U + r0 * ldu, ldu, st, s));
            CK(cudaEventRecord(io->ready[k], s));
            CK(cudaStreamWaitEvent(io->out, io->ready[k], 0));
            CK(cudaMemcpy2DAsync(io->U_host + r0 * io->ldu_host, sizeof(double) * io->ldu_host,
                                 U + r0 * ldu, sizeof(TO) * ldu, sizeof(double) * n, rk,
                                 cudaMemcpyDeviceToHost, io->out));
        }
    } else {
        CK(launch_oz_nn_run<TO>(big, m, (int)n, er, img, em, (int)n, U, ldu, st, s));
    }
    CK(launch_convert<TO>(sigma, n, 1, n, S, n, s));
    CK(launch_convert<TO>(Vo, n, n, n, V, ldv, s));
    return cudaSuccess;
}

// Dispatch on the arithmetic mode.
template <typename T, typename TO>
cudaError_t ts_any(const T *A, i64 m, i64 n, i64 lda, TO *U, i64 ldu, TO *S, TO *V, i64 ldv,
                   int passes, int scale, double tol, int max_sweeps, Bump &ws, DevStatus *st,
                   cudaStream_t s, int mode, const tssvd_comm *comm = nullptr)
{
    if (mode == TSSVD_FP64_TC)
        return ts_core_oz<T, TO>(A, m, n, lda, U, ldu, S, V, ldv, passes, scale, tol, max_sweeps,
                                 ws, st, s, comm);
    // The BF16-split modes: split products in the first pass, digit
    // products (FP64-accurate) in the second (and third)
    if ((mode == TSSVD_BF16X3 || mode == TSSVD_BF16X6) && passes >= 2)
        return ts_core_oz<T, TO>(A, m, n, lda, U, ldu, S, V, ldv, passes, scale, tol, max_sweeps,
                                 ws, st, s, comm, mode_terms(mode));
    return ts_core<T, TO>(A, m, n, lda, U, ldu, S, V, ldv, passes, scale, tol, max_sweeps, ws, st,
                          s, comm);
}

// Status words are summarised into the ABI's status code.
int summarise(const std::vector<DevStatus> &sts, int nsolves_per, int *rank_out)
{
    int code = TSSVD_OK;
    for (const DevStatus &h : sts)
        if (h.err) return TSSVD_ETIMEOUT;
    for (const DevStatus &h : sts)
        for (int i = 0; i < nsolves_per; i++)
            if (h.sweeps[i] < 0) code = TSSVD_ENOCONV;
    (void)rank_out;
    return code;
}

// Resolves the workspace for a call: the caller's, or the internal one
// (grown if needed; the returned lock is held for the call).
int acquire_ws(tssvd_opts *o, size_t need, void **base, std::unique_lock<std::mutex> &lk)
{
    if (o->workspace) {
        // the carve-up aligns every piece to 256 bytes from the base, so an
        // unaligned base costs up to 255 bytes (the queried sizes include them)
        const size_t pad = (256 - ((size_t)o->workspace & 255)) & 255;
        if (o->workspace_bytes < need + pad) return TSSVD_ENOMEM;
        *base = o->workspace;
        return TSSVD_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSSVD_ECUDA;
    InternalWs &w = g_ws[dev];
    lk = std::unique_lock<std::mutex>(w.mu);
    need += 256;  // room to align a base that is not 256-byte aligned
    if (w.bytes < need) {
        if (w.ptr) {
            cudaDeviceSynchronize();
            cudaFree(w.ptr);
            w.ptr = nullptr;
            w.bytes = 0;
        }
        if (cudaMalloc(&w.ptr, need) != cudaSuccess) {
            cudaGetLastError();
            w.ptr = nullptr;
            return TSSVD_ENOMEM;
        }
        w.bytes = need;
    }
    *base = w.ptr;
    return TSSVD_OK;
}

// ------------------------------------------------------------- batched

constexpr int kWorkers = 32;  // worker streams of a batch

struct WorkerStreams {
    bool ready = false;
    cudaStream_t w[kWorkers];
    cudaEvent_t fork, join[kWorkers];
    cudaStream_t own;  // blocking stream used when the caller passes NULL
};
WorkerStreams g_workers[64];

struct BatchGraph {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;  // kernel launches per replay
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_graphs;  // small most-recent-first cache
std::map<std::pair<int, int>, int> g_tuned;  // (log2 m, n/32) -> mode

int log2_ceil(i64 v)
{
    int e = 0;
    while (((i64)1 << e) < v) e++;
    return e;
}

int ensure_workers(int dev)
{
    WorkerStreams &W = g_workers[dev];
    if (W.ready) return 0;
    for (int i = 0; i < kWorkers; i++) {
        if (cudaStreamCreateWithFlags(&W.w[i], cudaStreamNonBlocking) != cudaSuccess) return -1;
        if (cudaEventCreateWithFlags(&W.join[i], cudaEventDisableTiming) != cudaSuccess) return -1;
    }
    if (cudaEventCreateWithFlags(&W.fork, cudaEventDisableTiming) != cudaSuccess) return -1;
    if (cudaStreamCreate(&W.own) != cudaSuccess) return -1;
    W.ready = true;
    return 0;
}

template <typename T>
size_t member_ws(const tssvd_desc &d, const tssvd_opts *o, int mode)
{
    Bump sz(nullptr, 0);
    ts_any<T, T>(nullptr, d.m, d.n, d.n, (T *)nullptr, d.n, (T *)nullptr, (T *)nullptr, d.n,
                 o->passes, o->scale, o->drop_tol, o->max_sweeps, sz, nullptr, nullptr, mode);
    return sz.off + 256;
}

// Plan of a batch: members ordered largest first, each assigned to the
// worker with the least work so far (longest-processing-time rule).
struct Plan {
    std::vector<int> order, worker, modes;
    std::vector<size_t> slice;  // bytes per worker
    size_t status_bytes = 0, total = 0;
};

template <typename T>
Plan make_plan(const tssvd_desc *d, int count, const tssvd_opts *o, const std::vector<int> &modes)
{
    Plan p;
    p.order.resize(count);
    for (int i = 0; i < count; i++) p.order[i] = i;
    auto work = [&](int i) { return (double)d[i].m * (double)d[i].n * (double)d[i].n; };
    std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) { return work(a) > work(b); });
    p.worker.assign(count, 0);
    p.modes = modes;
    std::vector<double> load(kWorkers, 0.0);
    p.slice.assign(kWorkers, 0);
    for (int i : p.order) {
        int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        p.worker[i] = w;
        load[w] += work(i);
        const size_t need = (member_ws<T>(d[i], o, modes[i]) + 255) & ~(size_t)255;
        p.slice[w] = std::max(p.slice[w], need);
    }
    p.status_bytes = ((sizeof(DevStatus) * (size_t)count + 255) / 256) * 256;
    p.total = p.status_bytes;
    for (size_t b : p.slice) p.total += b;
    return p;
}

int check_member(const tssvd_desc &d, int mode)
{
    if (!d.A || !d.U || !d.S || !d.V) return 1;
    if (d.n < 1 || d.n > 16384 || d.m < d.n || d.lda < d.n) return 1;
    if ((mode == TSSVD_BF16X3 || mode == TSSVD_BF16X6) && d.n > 256) return 1;
    return 0;
}

// Replays a batch graph on s and turns the members' status blocks into
// their status codes (the first failure is returned).
int finish_batch(BatchGraph *g, tssvd_desc *d, int count, const tssvd_opts *o, DevStatus *sts,
                 const std::vector<int> &modes, cudaStream_t s)
{
    std::vector<DevStatus> h(count);
    if (cudaGraphLaunch(g->exec, s) != cudaSuccess ||
        cudaMemcpyAsync(h.data(), sts, sizeof(DevStatus) * count, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    int first = TSSVD_OK;
    for (int i = 0; i < count; i++) {
        int code = TSSVD_OK;
        if (h[i].err)
            code = TSSVD_ETIMEOUT;
        else {
            const int solves = o->passes >= 2 ? 3 : 1;
            for (int j = 0; j < solves; j++)
                if (h[i].sweeps[j] < 0) code = TSSVD_ENOCONV;
            if (code == TSSVD_OK && h[i].rank < d[i].n) code = TSSVD_RANKDEF;
        }
        d[i].status = code;
        d[i].out_rank = h[i].rank;
        d[i].mode = modes[i];
        for (int j = 0; j < 3; j++) d[i].sweeps[j] = h[i].sweeps[j];
        if (first == TSSVD_OK && code != TSSVD_OK) first = code;
    }
    return first;
}

// Pinned host copies of the three task arrays of a cached phased graph
// (the graph copies them to the device at the start of every replay), and
// the event pairs the graph records around its three batched solves.
struct PinnedTasks {
    JacobiTask *h = nullptr;
    PcholTask *hp = nullptr;
    cudaEvent_t ev[6] = {};
    ~PinnedTasks()
    {
        if (h) cudaFreeHost(h);
        if (hp) cudaFreeHost(hp);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};
std::vector<std::pair<std::vector<unsigned long long>, std::shared_ptr<PinnedTasks>>> g_phased_tasks;

void evict_tasks(const std::vector<unsigned long long> &key)
{
    for (size_t k = 0; k < g_phased_tasks.size(); k++)
        if (g_phased_tasks[k].first == key) {
            g_phased_tasks.erase(g_phased_tasks.begin() + (long)k);
            return;
        }
}

// ------------------------------------------------ phased batch (FP64_TC)
//
// The batch of members with n <= kJacobiBatchMaxN in the FP64-accurate
// tensor-core form (Algorithm 4 per member) runs in phases: the members'
// tall products and small steps go to the worker streams, and each of the
// three Jacobi solves of every member runs in one launch of the batched
// solver (one CTA per member, jacobi_batch.cu) between them:
//   A: column maxima, Gram of A, pivoted Cholesky of B    | solve 1 (eig 1)
//   B: eigenvectors, Y~ = A (D^-1 V~), Gram of Y~, pivoted Cholesky of Z
//                                                          | solve 2 (eig 2)
//   C: W, Q~ and T, R = T W^T Sigma~ V~^T D                | solve 3 (SVD of R)
//   D: P, Sigma, V, U = Y~ (Sigma~^-1 W T^-1 P)
// Both eigensolves are one-sided on the pivoted Cholesky factor without
// accumulation (the factor's orthogonalised columns are the eigenvectors),
// the SVD of R one-sided with accumulation, as in the single-call path.
// State that lives across a solve (the n x n factors, V~, W, the scales,
// Y~) is kept per member; digit images, partial sums and the other n x n
// temporaries are per worker, sized for the worker's largest member.  For
// double outputs Y~ lives in U's storage (U's row image is built from it
// before the final product overwrites it).

struct PhasedMember {
    double *B;                             // n x n: the Gram matrix to factor
    double *X, *J, *Vt, *W;                // n x n
    double *d, *dinv, *sig, *sinv, *tinv;  // n
    int *pk1, *piv, *pk2;                  // n
    double *Y;                             // m x n: Y~
    float *w32;                            // 2 n^2: FP32 phase (n >= kBatchMixedMinN)
    double *wk;                            // 2 n^2: Newton-Schulz
};

// From this n the batched first eigensolve and SVD of R start with an FP32
// phase (the batch is bound by FP64 work: the phase leaves about 4 FP64
// sweeps of 10-14, for about two sweeps' worth of Newton-Schulz products).
constexpr i64 kBatchMixedMinN = 64;

struct PhasedScratch {
    unsigned long long *bits;
    int *exA, *exY, *em, *er, *perm;
    double *P, *NP, *Qw;
    uint8_t *img, *big;
    double *G2, *G, *R, *M, *M3, *Pm, *Vo, *Pp, *Xn;
    double *lam, *norms, *Tn, *Tk, *sgn, *sigma, *jn;
};

void take_member(Bump &b, i64 m, i64 n, bool own_y, PhasedMember &p)
{
    const i64 nn = n * n;
    p.B = b.take<double>(nn);
    p.X = b.take<double>(nn);
    p.J = b.take<double>(nn);
    p.Vt = b.take<double>(nn);
    p.W = b.take<double>(nn);
    p.d = b.take<double>(n);
    p.dinv = b.take<double>(n);
    p.sig = b.take<double>(n);
    p.sinv = b.take<double>(n);
    p.tinv = b.take<double>(n);
    p.pk1 = b.take<int>(n);
    p.piv = b.take<int>(n);
    p.pk2 = b.take<int>(n);
    p.Y = own_y ? b.take<double>((size_t)m * n) : nullptr;
    const bool mixed = n >= kBatchMixedMinN;
    p.w32 = mixed ? b.take<float>(2 * (size_t)nn) : nullptr;
    p.wk = mixed ? b.take<double>(2 * (size_t)nn) : nullptr;
}

void take_scratch(Bump &b, i64 m, i64 n, PhasedScratch &c)
{
    const i64 nn = n * n;
    c.bits = b.take<unsigned long long>(n);
    c.exA = b.take<int>(n);
    c.exY = b.take<int>(n);
    c.em = b.take<int>(n);
    c.perm = b.take<int>(n);
    c.er = b.take<int>(m);
    const int osp = oz_gram_splits(m, (int)n), sp2 = tn_splits(n, n, n, false);
    c.P = b.take<double>((size_t)(osp > sp2 ? osp : sp2) * nn);
    const int gcs = colsumsq_rows(m, n), gys = nn_grid_rows(n, n);
    c.NP = b.take<double>((size_t)(gcs > gys ? gcs : gys) * n);
    c.Qw = b.take<double>((size_t)m * n);
    c.img = b.take<uint8_t>(oz_image_bytes((int)n, (int)n));
    const size_t gib = oz_gram_image_bytes(m, (int)n), rib = oz_row_image_bytes(m, (int)n);
    c.big = b.take<uint8_t>(gib > rib ? gib : rib);
    double **nxn[] = {&c.G2, &c.G, &c.R, &c.M, &c.M3, &c.Pm, &c.Vo, &c.Pp, &c.Xn};
    for (double **q : nxn) *q = b.take<double>(nn);
    double **vec[] = {&c.lam, &c.norms, &c.Tn, &c.Tk, &c.sgn, &c.sigma, &c.jn};
    for (double **q : vec) *q = b.take<double>(n);
}

bool phased_applies(const tssvd_desc *d, int count, const tssvd_opts *o)
{
    if (o->passes != 2 || (o->mode != TSSVD_FP64_TC && o->mode != TSSVD_AUTO)) return false;
    for (int i = 0; i < count; i++)
        if (d[i].n < 1 || d[i].n > kJacobiBatchMaxN) return false;
    return true;
}

struct PhasedPlan {
    std::vector<int> order, worker;  // members by decreasing work; their workers
    std::vector<size_t> member_off;  // byte offsets of the members' state
    std::vector<size_t> slice_off, slice;  // workers' scratch
    size_t status_bytes = 0, tasks_off = 0, ptasks_off = 0, total = 0;
};

template <typename T>
PhasedPlan make_phased_plan(const tssvd_desc *d, int count)
{
    PhasedPlan p;
    p.order.resize(count);
    for (int i = 0; i < count; i++) p.order[i] = i;
    auto work = [&](int i) { return (double)d[i].m * (double)d[i].n * (double)d[i].n; };
    std::stable_sort(p.order.begin(), p.order.end(), [&](int a, int b) { return work(a) > work(b); });
    p.worker.assign(count, 0);
    std::vector<double> load(kWorkers, 0.0);
    p.slice.assign(kWorkers, 0);
    for (int i : p.order) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        p.worker[i] = w;
        load[w] += work(i);
        Bump sz(nullptr, 0);
        PhasedScratch c;
        take_scratch(sz, d[i].m, d[i].n, c);
        p.slice[w] = std::max(p.slice[w], (sz.off + 255) & ~(size_t)255);
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = up(sizeof(DevStatus) * (size_t)count);
    p.status_bytes = off;
    p.tasks_off = off;
    off += up(sizeof(JacobiTask) * 3 * (size_t)count);
    p.ptasks_off = off;
    off += up(sizeof(PcholTask) * (size_t)count);
    p.member_off.resize(count);
    const bool own_y = sizeof(T) != sizeof(double);
    for (int i = 0; i < count; i++) {
        p.member_off[i] = off;
        Bump sz(nullptr, 0);
        PhasedMember pm;
        take_member(sz, d[i].m, d[i].n, own_y, pm);
        off += up(sz.off);
    }
    p.slice_off.resize(kWorkers);
    for (int w = 0; w < kWorkers; w++) {
        p.slice_off[w] = off;
        off += p.slice[w];
    }
    p.total = off;
    return p;
}

// Segment A of member i: column maxima and the Gram matrix B of A (its
// pivoted Cholesky runs batched after the segment).
template <typename T>
cudaError_t phase_a(const tssvd_desc &dd, const tssvd_opts *o, PhasedMember &p,
                    PhasedScratch &c, DevStatus *st, cudaStream_t s)
{
    const T *A = (const T *)dd.A;
    const i64 m = dd.m, n = dd.n, lda = dd.lda;
    CK(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    CK(cudaMemsetAsync(c.bits, 0, sizeof(unsigned long long) * n, s));
    CK(launch_colmax<T>(A, m, n, lda, c.bits, s));
    CK(launch_oz_exp_from_bits(c.bits, (int)n, c.exA, s));
    if (o->scale) {
        CK(launch_pow2_scale(c.bits, n, p.d, p.dinv, s));
        CK(launch_neg_int(c.exA, (int)n, p.pk1, s));
    }
    const int osp = oz_gram_splits(m, (int)n);
    CK(launch_oz_gram<T>(A, lda, m, (int)n, c.exA, osp, c.big, c.P, st, s));
    const double *rs = o->scale ? p.dinv : nullptr;
    return launch_tn_reduce(c.P, osp, n, n, rs, rs, true, p.B, n, s);
}

// Segment B: V~ from the solved factor, Y~ = A (D^-1 V~), its Gram Z,
// Sigma~ and the discard (Z's pivoted Cholesky runs batched after it).
template <typename T>
cudaError_t phase_b(const tssvd_desc &dd, const tssvd_opts *o, PhasedMember &p,
                    PhasedScratch &c, DevStatus *st, cudaStream_t s)
{
    const T *A = (const T *)dd.A;
    const i64 m = dd.m, n = dd.n, lda = dd.lda;
    CK(launch_jacobi_finalize(p.X, n, nullptr, n, (int)n, (int)n, c.norms, c.perm, nullptr, n,
                              c.lam, c.Xn, n, s));
    CK(launch_row_scatter(c.Xn, p.piv, (int)n, p.Vt, s));
    const double *M1 = p.Vt;
    const int *pkA = o->scale ? p.pk1 : nullptr;
    if (o->scale) {
        CK(launch_scale2(p.Vt, n, n, n, p.dinv, nullptr, c.M, n, s));
        M1 = c.M;
    }
    CK(launch_oz_image(M1, n, (int)n, (int)n, pkA, c.em, c.img, s));
    CK(launch_oz_rowexp<T>(A, lda, m, (int)n, pkA, c.er, s));
    CK(launch_oz_row_image<T>(A, lda, m, (int)n, pkA, c.er, c.big, s));
    const bool fuse = oz_nn_fuses((int)n);
    CK(cudaMemsetAsync(c.bits, 0, sizeof(unsigned long long) * n, s));
    CK(launch_oz_nn_run<double>(c.big, m, (int)n, c.er, c.img, c.em, (int)n, p.Y, n, st, s,
                                fuse ? c.bits : nullptr, nullptr));
    if (!fuse) CK(launch_colmax<double>(p.Y, m, n, n, c.bits, s));
    CK(launch_oz_exp_from_bits(c.bits, (int)n, c.exY, s));
    const int osp = oz_gram_splits(m, (int)n);
    CK(launch_oz_gram<double>(p.Y, n, m, (int)n, c.exY, osp, c.big, c.P, st, s));
    CK(launch_tn_reduce(c.P, osp, n, n, nullptr, nullptr, true, c.G2, n, s));
    CK(launch_diag_sqrt(c.G2, n, n, p.sig, s));
    CK(launch_discard(p.sig, n, o->drop_tol, p.sinv, &st->rank1, s));
    return launch_scale2(c.G2, n, n, n, p.sinv, p.sinv, p.B, n, s);
}

// Segment C: W from the solved factor, Q~ = Y W and its explicit norms T,
// the discard, R = T W^T Sigma~ V~^T D, oriented for the one-sided SVD.
cudaError_t phase_c(const tssvd_desc &dd, const tssvd_opts *o, PhasedMember &p,
                    PhasedScratch &c, DevStatus *st, cudaStream_t s)
{
    const i64 m = dd.m, n = dd.n;
    CK(launch_jacobi_finalize(p.X, n, nullptr, n, (int)n, (int)n, c.norms, c.perm, nullptr, n,
                              c.lam, c.Xn, n, s));
    CK(launch_row_scatter(c.Xn, p.piv, (int)n, p.W, s));
    CK(launch_oz_pow2_of(p.sinv, (int)n, p.pk2, s));
    CK(launch_oz_rowexp<double>(p.Y, n, m, (int)n, p.pk2, c.er, s));
    CK(launch_oz_row_image<double>(p.Y, n, m, (int)n, p.pk2, c.er, c.big, s));
    CK(launch_scale2(p.W, n, n, n, p.sinv, nullptr, c.M, n, s));
    CK(launch_oz_image(c.M, n, (int)n, (int)n, p.pk2, c.em, c.img, s));
    CK(launch_oz_nn_run<double>(c.big, m, (int)n, c.er, c.img, c.em, (int)n, c.Qw, n, st, s));
    CK(launch_colsumsq(c.Qw, n, m, n, c.NP, s));
    CK(launch_norms_reduce(c.NP, colsumsq_rows(m, n), n, c.Tn, s));
    CK(launch_discard(c.Tn, n, o->drop_tol, p.tinv, &st->rank2, s));
    CK(launch_keepval(c.Tn, p.tinv, n, c.Tk, s));
    const double *dsc = o->scale ? p.d : nullptr;
    CK(launch_build_g(p.sig, p.sinv, p.Vt, n, dsc, n, c.G, s));
    const int sp2 = tn_splits(n, n, n, false);
    CK(launch_tn_partial<double, double>(p.W, n, c.G, n, n, n, n, sp2, false, c.P, s));
    CK(launch_tn_reduce(c.P, sp2, n, n, c.Tk, nullptr, false, c.R, n, s));
    return launch_orient_copy(dsc, &st->rank2, c.R, n, p.X, &st->orient, s);
}

// Segment D: P, Sigma, V from the solved R, signs, rank, and
// U = Y~ (Sigma~^-1 W T^-1 P diag(sgn)).
template <typename T>
cudaError_t phase_d(const tssvd_desc &dd, PhasedMember &p, PhasedScratch &c, DevStatus *st,
                    cudaStream_t s)
{
    const i64 m = dd.m, n = dd.n;
    CK(launch_jacobi_finalize(p.X, n, p.J, n, (int)n, (int)n, c.norms, c.perm, c.Pm, n, c.sigma,
                              c.Vo, n, s, &st->orient, c.jn));
    CK(launch_signs(c.Vo, n, n, n, c.sigma, c.sgn, s));
    CK(launch_count_positive(c.sigma, n, &st->rank, s));
    CK(launch_scale2(c.Pm, n, n, n, p.tinv, c.sgn, c.Pp, n, s));
    CK(launch_scale2(p.W, n, n, n, p.sinv, nullptr, c.M, n, s));
    CK(launch_nn<double, double>(c.M, n, c.Pp, n, n, n, n, c.M3, n, c.NP, s));
    CK(launch_oz_rowexp<double>(p.Y, n, m, (int)n, p.pk2, c.er, s));
    CK(launch_oz_row_image<double>(p.Y, n, m, (int)n, p.pk2, c.er, c.big, s));
    CK(launch_oz_image(c.M3, n, (int)n, (int)n, p.pk2, c.em, c.img, s));
    CK(launch_oz_nn_run<T>(c.big, m, (int)n, c.er, c.img, c.em, (int)n, (T *)dd.U, n, st, s));
    CK(launch_convert<T>(c.sigma, n, 1, n, (T *)dd.S, n, s));
    return launch_convert<T>(c.Vo, n, n, n, (T *)dd.V, n, s);
}

template <typename T>
int batched_phased(tssvd_desc *d, int count, tssvd_opts *o)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSSVD_ECUDA;
    std::lock_guard<std::mutex> glk(g_batch_mu);
    if (ensure_workers(dev)) return TSSVD_ECUDA;
    WorkerStreams &W = g_workers[dev];
    cudaStream_t s = o->stream ? (cudaStream_t)o->stream : W.own;
    for (int i = 0; i < count; i++)
        if (check_member(d[i], TSSVD_FP64_TC)) return -(100 + i);
    PhasedPlan plan = make_phased_plan<T>(d, count);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(o, plan.total + 256, &base, lk);
    if (rc) return rc;
    base = (void *)(((size_t)base + 255) & ~(size_t)255);
    char *cb = (char *)base;
    DevStatus *sts = (DevStatus *)base;
    JacobiTask *dtasks = (JacobiTask *)(cb + plan.tasks_off);
    PcholTask *dptasks = (PcholTask *)(cb + plan.ptasks_off);
    const bool own_y = sizeof(T) != sizeof(double);
    std::vector<PhasedMember> pm(count);
    for (int i = 0; i < count; i++) {
        Bump b(cb + plan.member_off[i], (size_t)1 << 62);
        take_member(b, d[i].m, d[i].n, own_y, pm[i]);
        if (!own_y) pm[i].Y = (double *)d[i].U;
    }

    std::vector<unsigned long long> key;
    key.push_back(0x9a5edULL);  // phased graphs apart from the per-member ones
    key.push_back((unsigned long long)count);
    key.push_back((unsigned long long)sizeof(T));
    key.push_back((unsigned long long)(uintptr_t)base);
    key.push_back((unsigned long long)(uintptr_t)s);
    unsigned long long tolbits;
    std::memcpy(&tolbits, &o->drop_tol, 8);
    key.push_back(tolbits);
    key.push_back(((unsigned long long)o->scale << 16) | (unsigned long long)o->max_sweeps);
    for (int i = 0; i < count; i++) {
        key.push_back((unsigned long long)(uintptr_t)d[i].A);
        key.push_back((unsigned long long)(uintptr_t)d[i].U);
        key.push_back((unsigned long long)(uintptr_t)d[i].S);
        key.push_back((unsigned long long)(uintptr_t)d[i].V);
        key.push_back((unsigned long long)d[i].m);
        key.push_back((unsigned long long)d[i].n);
        key.push_back((unsigned long long)d[i].lda);
    }
    BatchGraph *g = nullptr;
    for (auto &bg : g_graphs)
        if (bg.key == key) g = &bg;
    if (!g) {
        // the solve tasks, members by decreasing n (the long solves first)
        auto pin = std::make_shared<PinnedTasks>();
        if (cudaMallocHost(&pin->h, sizeof(JacobiTask) * 3 * (size_t)count) != cudaSuccess ||
            cudaMallocHost(&pin->hp, sizeof(PcholTask) * (size_t)count) != cudaSuccess) {
            cudaGetLastError();
            return TSSVD_ENOMEM;
        }
        for (cudaEvent_t &ev : pin->ev)
            if (cudaEventCreate(&ev) != cudaSuccess) {
                cudaGetLastError();
                return TSSVD_ECUDA;
            }
        std::vector<int> by_n(count);
        for (int i = 0; i < count; i++) by_n[i] = i;
        std::stable_sort(by_n.begin(), by_n.end(), [&](int a, int b) { return d[a].n > d[b].n; });
        for (int k = 0; k < count; k++) {
            const int i = by_n[k];
            const int n = (int)d[i].n;
            pin->h[k] = JacobiTask{pm[i].X, nullptr, n, 0, 0x1p-51, &sts[i], pm[i].w32, pm[i].wk};
            pin->h[count + k] = JacobiTask{pm[i].X, nullptr, n, 1, (double)n * 0x1p-53, &sts[i],
                                           nullptr, nullptr};
            pin->h[2 * count + k] = JacobiTask{pm[i].X, pm[i].J, n, 2, (double)n * 0x1p-53,
                                               &sts[i], pm[i].w32, pm[i].wk};
            pin->hp[k] = PcholTask{pm[i].B, pm[i].X, pm[i].piv, n};
        }
        const int nmax = (int)d[by_n[0]].n;
        const long long n0 = tssvd_launch_count();
        const int prof = tssvd_profile_enable(0);  // no event records inside the graph
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dtasks, pin->h, sizeof(JacobiTask) * 3 * (size_t)count,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dptasks, pin->hp, sizeof(PcholTask) * (size_t)count,
                                cudaMemcpyHostToDevice, s);
        for (int phase = 0; phase < 4 && e == cudaSuccess; phase++) {
            e = cudaEventRecord(W.fork, s);
            for (int w = 0; w < kWorkers && e == cudaSuccess; w++)
                e = cudaStreamWaitEvent(W.w[w], W.fork, 0);
            for (int i : plan.order) {
                if (e != cudaSuccess) break;
                const int w = plan.worker[i];
                Bump b(cb + plan.slice_off[w], plan.slice[w]);
                PhasedScratch c;
                take_scratch(b, d[i].m, d[i].n, c);
                cudaStream_t ws_ = W.w[w];
                if (phase == 0) e = phase_a<T>(d[i], o, pm[i], c, &sts[i], ws_);
                else if (phase == 1) e = phase_b<T>(d[i], o, pm[i], c, &sts[i], ws_);
                else if (phase == 2) e = phase_c(d[i], o, pm[i], c, &sts[i], ws_);
                else e = phase_d<T>(d[i], pm[i], c, &sts[i], ws_);
            }
            for (int w = 0; w < kWorkers; w++) {
                cudaError_t e2 = cudaEventRecord(W.join[w], W.w[w]);
                if (e == cudaSuccess) e = e2;
                e2 = cudaStreamWaitEvent(s, W.join[w], 0);
                if (e == cudaSuccess) e = e2;
            }
            // the pivoted Cholesky factorizations of segments A and B, batched
            if (phase < 2 && e == cudaSuccess) e = launch_pchol_batch(dptasks, count, nmax, s);
            // (external records: event nodes of the graph, readable after a replay)
            if (phase < 3 && e == cudaSuccess)
                e = cudaEventRecordWithFlags(pin->ev[2 * phase], s, cudaEventRecordExternal);
            if (phase < 3 && e == cudaSuccess)
                e = launch_jacobi_batch(dtasks + (size_t)phase * count, count, o->max_sweeps, s);
            if (phase < 3 && e == cudaSuccess)
                e = cudaEventRecordWithFlags(pin->ev[2 * phase + 1], s, cudaEventRecordExternal);
        }
        cudaError_t ec = cudaStreamEndCapture(s, &graph);
        tssvd_profile_enable(prof);
        if (e == cudaSuccess) e = ec;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            fprintf(stderr, "tssvd: batch capture failed: %s\n", cudaGetErrorString(e));
            cudaGetLastError();
            return TSSVD_ECUDA;
        }
        BatchGraph nb;
        nb.key = key;
        nb.exec = exec;
        nb.kernels = tssvd_launch_count() - n0;
        if (g_graphs.size() >= 8) {
            evict_tasks(g_graphs.back().key);
            cudaGraphExecDestroy(g_graphs.back().exec);
            g_graphs.pop_back();
        }
        g_graphs.insert(g_graphs.begin(), nb);
        g_phased_tasks.emplace_back(key, pin);
        g = &g_graphs.front();
    } else {
        add_launches(g->kernels);
    }
    std::vector<int> modes(count, TSSVD_FP64_TC);
    const int code = finish_batch(g, d, count, o, sts, modes, s);
    if (profiling())
        for (auto &pt : g_phased_tasks)
            if (pt.first == key)
                for (int p = 0; p < 3; p++) {
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, pt.second->ev[2 * p], pt.second->ev[2 * p + 1]) ==
                        cudaSuccess)
                        prof_add_ms("jacobi_batch", ms);
                    else
                        cudaGetLastError();
                }
    return code;
}

template <typename T>
int batched_impl(tssvd_desc *d, int count, tssvd_opts *o)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSSVD_ECUDA;
    std::lock_guard<std::mutex> glk(g_batch_mu);
    if (ensure_workers(dev)) return TSSVD_ECUDA;
    WorkerStreams &W = g_workers[dev];
    cudaStream_t s = o->stream ? (cudaStream_t)o->stream : W.own;

    // modes (resolving TSSVD_AUTO per size class)
    std::vector<int> modes(count, o->mode);
    if (o->mode == TSSVD_AUTO) {
        for (int i = 0; i < count; i++) {
            const std::pair<int, int> key(log2_ceil(d[i].m), (int)((d[i].n + 31) / 32));
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                modes[i] = it->second;
                continue;
            }
            // time both FP64-accurate engines once on this member
            const int cand[2] = {TSSVD_FP64, TSSVD_FP64_TC};
            float best = 0.f;
            int bestm = TSSVD_FP64;
            size_t need = std::max(member_ws<T>(d[i], o, cand[0]), member_ws<T>(d[i], o, cand[1]));
            void *base = nullptr;
            std::unique_lock<std::mutex> lk;
            tssvd_opts o2 = *o;
            o2.workspace = nullptr;
            if (acquire_ws(&o2, need + 256, &base, lk)) return TSSVD_ENOMEM;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int c = 0; c < 2; c++) {
                for (int rep = 0; rep < 2; rep++) {  // the second run is timed
                    Bump ws(base, need + 256);
                    DevStatus *st = ws.take<DevStatus>(1);
                    cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
                    cudaEventRecord(e0, s);
                    cudaError_t e = ts_any<T, T>((const T *)d[i].A, d[i].m, d[i].n, d[i].lda, (T *)d[i].U,
                                                 d[i].n, (T *)d[i].S, (T *)d[i].V, d[i].n, o->passes,
                                                 o->scale, o->drop_tol, o->max_sweeps, ws, st, s, cand[c]);
                    cudaEventRecord(e1, s);
                    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaGetLastError();
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return TSSVD_ECUDA;
                    }
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (c == 0 || ms < best) {
                    best = ms;
                    bestm = cand[c];
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            g_tuned[key] = bestm;
            modes[i] = bestm;
        }
    }
    for (int i = 0; i < count; i++)
        if (check_member(d[i], modes[i])) return -(100 + i);

    Plan plan = make_plan<T>(d, count, o, modes);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(o, plan.total + 256, &base, lk);
    if (rc) return rc;
    base = (void *)(((size_t)base + 255) & ~(size_t)255);
    DevStatus *sts = (DevStatus *)base;
    std::vector<char *> slice_base(kWorkers);
    {
        size_t off = plan.status_bytes;
        for (int w = 0; w < kWorkers; w++) {
            slice_base[w] = (char *)base + off;
            off += plan.slice[w];
        }
    }

    // graph cache key: members, element type, options, stream, workspace
    std::vector<unsigned long long> key;
    key.push_back((unsigned long long)count);
    key.push_back((unsigned long long)sizeof(T));
    key.push_back((unsigned long long)(uintptr_t)base);
    key.push_back((unsigned long long)(uintptr_t)s);
    unsigned long long tolbits;
    std::memcpy(&tolbits, &o->drop_tol, 8);
    key.push_back(tolbits);
    key.push_back(((unsigned long long)o->passes << 32) | ((unsigned long long)o->scale << 16) |
                  (unsigned long long)o->max_sweeps);
    for (int i = 0; i < count; i++) {
        key.push_back((unsigned long long)(uintptr_t)d[i].A);
        key.push_back((unsigned long long)(uintptr_t)d[i].U);
        key.push_back((unsigned long long)(uintptr_t)d[i].S);
        key.push_back((unsigned long long)(uintptr_t)d[i].V);
        key.push_back((unsigned long long)d[i].m);
        key.push_back((unsigned long long)d[i].n);
        key.push_back((unsigned long long)d[i].lda);
        key.push_back((unsigned long long)modes[i]);
    }
    BatchGraph *g = nullptr;
    for (auto &bg : g_graphs)
        if (bg.key == key) g = &bg;
    if (!g) {
        const long long n0 = tssvd_launch_count();
        const int prof = tssvd_profile_enable(0);  // no event records inside the graph
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaEventRecord(W.fork, s);
        for (int w = 0; w < kWorkers && e == cudaSuccess; w++) e = cudaStreamWaitEvent(W.w[w], W.fork, 0);
        for (int i : plan.order) {
            if (e != cudaSuccess) break;
            const int w = plan.worker[i];
            cudaStream_t ws_ = W.w[w];
            Bump b(slice_base[w], plan.slice[w]);  // members of a worker reuse its slice
            e = cudaMemsetAsync(&sts[i], 0, sizeof(DevStatus), ws_);
            if (e == cudaSuccess)
                e = ts_any<T, T>((const T *)d[i].A, d[i].m, d[i].n, d[i].lda, (T *)d[i].U, d[i].n,
                                 (T *)d[i].S, (T *)d[i].V, d[i].n, o->passes, o->scale, o->drop_tol,
                                 o->max_sweeps, b, &sts[i], ws_, modes[i]);
        }
        for (int w = 0; w < kWorkers; w++) {
            cudaError_t e2 = cudaEventRecord(W.join[w], W.w[w]);
            if (e == cudaSuccess) e = e2;
            e2 = cudaStreamWaitEvent(s, W.join[w], 0);
            if (e == cudaSuccess) e = e2;
        }
        cudaError_t ec = cudaStreamEndCapture(s, &graph);
        tssvd_profile_enable(prof);
        if (e == cudaSuccess) e = ec;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            fprintf(stderr, "tssvd: batch capture failed: %s\n", cudaGetErrorString(e));
            cudaGetLastError();
            return TSSVD_ECUDA;
        }
        BatchGraph nb;
        nb.key = key;
        nb.exec = exec;
        nb.kernels = tssvd_launch_count() - n0;
        if (g_graphs.size() >= 8) {
            evict_tasks(g_graphs.back().key);
            cudaGraphExecDestroy(g_graphs.back().exec);
            g_graphs.pop_back();
        }
        g_graphs.insert(g_graphs.begin(), nb);
        g = &g_graphs.front();
    } else {
        add_launches(g->kernels);
    }
    return finish_batch(g, d, count, o, sts, modes, s);
}

// passes: 1 (Algorithm 3), 2 (Algorithm 4) or 3 (Algorithm 4 with its
// second pass run twice); the TSQR methods take 1 or 2 (max_passes 2).
int check_opts(const tssvd_opts *o, int max_passes = 3)
{
    if (!o) return 0;
    if (o->passes < 1 || o->passes > max_passes) return 0;
    if (!(o->drop_tol >= 0.0) || o->drop_tol >= 1.0) return 0;
    if (o->max_sweeps < 1 || o->max_sweeps > 1000) return 0;
    if (o->mode < TSSVD_FP64 || o->mode > TSSVD_FP64_TC) return 0;
    return 1;
}

// ts_svd (mu == nullptr) and ts_pca (mu != nullptr: column means into mu,
// then the TS-SVD of the centred copy A - 1 mu^T held in the workspace).
// `pca` shifts the argument numbers of the error codes past mu.
// comm (ts_svd_rowshard): A holds this rank's rows; the exchange steps go
// through the caller's all-reduce (its argument number is 8, opts 9).
template <typename T>
int ts_svd_entry(const T *A, int64_t m, int64_t n, int64_t lda, T *U, T *S, T *V,
                 tssvd_opts *opts, T *mu = nullptr, bool pca = false,
                 const tssvd_comm *comm = nullptr, bool sharded = false)
{
    const int sh = (pca || sharded) ? 1 : 0;
    if (!A) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1 || n > 16384) return -3;
    if (lda < n) return -4;
    if (pca && !mu) return -5;
    if (!U) return -5 - (pca ? 1 : 0);
    if (!S) return -6 - (pca ? 1 : 0);
    if (!V) return -7 - (pca ? 1 : 0);
    if (sharded && (!comm || comm->size < 1 || comm->rank < 0 || comm->rank >= comm->size))
        return -8;
    if (!check_opts(opts)) return -8 - sh;
    if ((opts->mode == TSSVD_BF16X3 || opts->mode == TSSVD_BF16X6) && n > 256) {
        fprintf(stderr, "tssvd: the mixed-precision modes take n <= 256 (n = %lld)\n",
                (long long)n);
        return -3;
    }
    cudaStream_t s = (cudaStream_t)opts->stream;

    Bump sz(nullptr, 0);
    sz.take<DevStatus>(1);
    if (pca) {
        sz.take<T>((size_t)m * n);
        sz.take<double>((size_t)colsum_rows(m, n) * n);
    }
    ts_any<T, T>(A, m, n, lda, U, n, S, V, n, opts->passes, opts->scale, opts->drop_tol,
                 opts->max_sweeps, sz, nullptr, s, opts->mode);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    DevStatus *st = ws.take<DevStatus>(1);
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return TSSVD_ECUDA;
    const T *X = A;
    i64 ldx = lda;
    cudaError_t e = cudaSuccess;
    if (pca) {
        T *C = ws.take<T>((size_t)m * n);
        double *P = ws.take<double>((size_t)colsum_rows(m, n) * n);
        if (ws.overflow) return TSSVD_ENOMEM;
        e = launch_col_means<T>(A, lda, m, n, P, mu, s);
        if (e == cudaSuccess) e = launch_center<T>(A, lda, m, n, mu, C, s);
        X = C;
        ldx = n;
    }
    t_comm_failed = 0;
    if (e == cudaSuccess)
        e = ts_any<T, T>(X, m, n, ldx, U, n, S, V, n, opts->passes, opts->scale, opts->drop_tol,
                         opts->max_sweeps, ws, st, s, opts->mode, comm);
    if (e != cudaSuccess) {
        if (t_comm_failed) {
            fprintf(stderr, "tssvd: the all-reduce of a row-sharded call failed\n");
            cudaGetLastError();
            return TSSVD_ECOMM;
        }
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TSSVD_ENOMEM : TSSVD_ECUDA;
    }
    DevStatus h;
    if (cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    std::vector<DevStatus> v(1, h);
    int code = summarise(v, opts->passes >= 2 ? 3 : 1, nullptr);
    opts->out_rank = h.rank;
    for (int i = 0; i < 4; i++) opts->sweeps[i] = h.sweeps[i];
    opts->ranks[0] = h.rank1;
    opts->ranks[1] = opts->passes >= 2 ? h.rank2 : h.rank1;
    if (code == TSSVD_OK && h.rank < n) code = TSSVD_RANKDEF;
    return code;
}

// ------------------------------------------------------------- low rank

// Number of per-sub-call status blocks used by lowrank: 2 per power step + 2.
cudaError_t tsqr_core(const double *X, i64 rows, i64 n, i64 ldx, const double *Mt, double *U,
                      i64 ldu, double *S, double *V, i64 ldv, int passes, double wp,
                      int max_sweeps, Bump &ws, DevStatus *st, cudaStream_t s, bool oz = false);

cudaError_t lowrank_core(const double *A, i64 m, i64 n, i64 lda, i64 k, i64 l, int iters,
                         const double *Omega, double *U, double *S, double *V, double tol,
                         int max_sweeps, Bump &ws, DevStatus *sts, cudaStream_t s,
                         int mode = TSSVD_FP64)
{
    const bool sizing = ws.sizing();
    const bool oz = mode == TSSVD_FP64_TC;
    double *Qt = ws.take<double>((size_t)n * l), *Y = ws.take<double>((size_t)m * l);
    double *Q = ws.take<double>((size_t)m * l), *Bt = ws.take<double>((size_t)n * l);
    double *U1 = ws.take<double>((size_t)n * l), *S1 = ws.take<double>(l);
    double *V1 = ws.take<double>((size_t)l * l), *V1s = ws.take<double>((size_t)l * l);
    double *Uf = ws.take<double>((size_t)m * l), *sgn = ws.take<double>(l);
    double *tS = ws.take<double>(l), *tV = ws.take<double>((size_t)l * l);
    const int spT = oz ? oz_tn_splits(m, (int)n, (int)l) : tn_splits(m, n, l, false);
    double *P = ws.take<double>((size_t)spT * n * l);
    const int gy = nn_grid_rows(m, l);
    double *NP = ws.take<double>((size_t)gy * l);
    // digit images of A (built once per call) and of the thin factors
    unsigned long long *bits = oz ? ws.take<unsigned long long>(n > l ? n : l) : nullptr;
    int *exA = oz ? ws.take<int>(n) : nullptr, *erA = oz ? ws.take<int>(m) : nullptr;
    int *exQ = oz ? ws.take<int>(l) : nullptr, *em = oz ? ws.take<int>(l) : nullptr;
    uint8_t *rimgA = oz ? ws.take<uint8_t>(oz_row_image_bytes(m, (int)n)) : nullptr;
    uint8_t *cimgA = oz ? ws.take<uint8_t>(oz_gram_image_bytes(m, (int)n)) : nullptr;
    uint8_t *cimgQ = oz ? ws.take<uint8_t>(oz_gram_image_bytes(m, (int)l)) : nullptr;
    uint8_t *bimg = oz ? ws.take<uint8_t>(oz_image_bytes((int)n, (int)l)) : nullptr;
    // sub-call workspaces are carved last and reused by every sub-call
    const size_t sub_off = ws.off;
    const i64 big = m > n ? m : n;
    {
        Bump probe(nullptr, 0);
        ts_any<double, double>(nullptr, big, l, l, (double *)nullptr, l, (double *)nullptr,
                               (double *)nullptr, l, 2, 0, tol, max_sweeps, probe, nullptr, s, mode);
        Bump probe1(nullptr, 0);
        ts_any<double, double>(nullptr, big, l, l, (double *)nullptr, l, (double *)nullptr,
                               (double *)nullptr, l, 1, 0, tol, max_sweeps, probe1, nullptr, s, mode);
        ws.take<char>((probe.off > probe1.off ? probe.off : probe1.off) + 256);
    }
    if (sizing) return cudaSuccess;
    if (ws.overflow) return cudaErrorMemoryAllocation;
    auto sub = [&](const double *Ain, i64 rows, double *Uo, double *So, double *Vo, int passes,
                   DevStatus *st) -> cudaError_t {
        Bump w(ws.base + ((sub_off + 255) & ~(size_t)255), ws.cap - ((sub_off + 255) & ~(size_t)255));
        return ts_any<double, double>(Ain, rows, l, l, Uo, l, So, Vo, l, passes, 0, tol, max_sweeps,
                                      w, st, s, mode);
    };
    // Y = A X (m x l) and C = A^T Z (n x l) on the selected engine
    auto AX = [&](const double *X, double *Yo, DevStatus *st) -> cudaError_t {
        if (!oz) return launch_nn<double, double>(A, lda, X, l, m, n, l, Yo, l, NP, s);
        CK(launch_oz_image(X, l, (int)n, (int)l, nullptr, em, bimg, s));
        return launch_oz_nn_run<double>(rimgA, m, (int)n, erA, bimg, em, (int)l, Yo, l, st, s);
    };
    auto AtZ = [&](const double *Z, double *Co, DevStatus *st) -> cudaError_t {
        if (!oz) {
            CK(launch_tn_partial<double, double>(A, lda, Z, l, m, n, l, spT, false, P, s));
        } else {
            CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * l, s));
            CK(launch_colmax<double>(Z, m, l, l, bits, s));
            CK(launch_oz_exp_from_bits(bits, (int)l, exQ, s));
            CK(launch_oz_col_image(Z, l, m, (int)l, exQ, cimgQ, s));
            CK(launch_oz_tn(cimgA, exA, (int)n, cimgQ, exQ, (int)l, m, spT, P, st, s));
        }
        return launch_tn_reduce(P, spT, n, l, nullptr, nullptr, false, Co, l, s);
    };

    int si = 0;
    if (oz) {
        CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s));
        CK(launch_colmax<double>(A, m, n, lda, bits, s));
        CK(launch_oz_exp_from_bits(bits, (int)n, exA, s));
        CK(launch_oz_rowexp<double>(A, lda, m, (int)n, nullptr, erA, s));
        CK(launch_oz_row_image<double>(A, lda, m, (int)n, nullptr, erA, rimgA, s));
        CK(launch_oz_col_image(A, lda, m, (int)n, exA, cimgA, s));
    }
    CK(cudaMemcpyAsync(Qt, Omega, sizeof(double) * n * l, cudaMemcpyDeviceToDevice, s));
    DevStatus *pst = sts + (2 * iters + 2);  // status of the products' waits
    for (int it = 0; it < iters; it++) {
        // Y_j = A Q~_{j-1}; Y_j = Q_j R_j (Algorithm 3).
        CK(AX(Qt, Y, pst));
        CK(sub(Y, m, Q, tS, tV, 1, sts + si++));
        // Y~_j = A^T Q_j; Y~_j = Q~_j R~_j (Algorithm 3).
        CK(AtZ(Q, Bt, pst));
        CK(sub(Bt, n, Qt, tS, tV, 1, sts + si++));
    }
    // Y = A Q~_i; Y = Q R with double orthonormalisation (Algorithm 4).
    CK(AX(Qt, Y, pst));
    CK(sub(Y, m, Q, tS, tV, 2, sts + si++));
    // Algorithm 6: B = Q^T A via B^T = A^T Q (n x l); B^T = U1 S1 V1^T, so
    // B = V1 S1 U1^T: U~ = V1 and V = U1.
    CK(AtZ(Q, Bt, pst));
    CK(sub(Bt, n, U1, S1, V1, 2, sts + si++));
    // Sign convention on the final V = U1; U = Q U~ = Q V1 diag(sgn).
    CK(launch_signs(U1, l, n, l, S1, sgn, s));
    CK(launch_scale2(V1, l, l, l, nullptr, sgn, V1s, l, s));
    CK(launch_nn<double, double>(Q, l, V1s, l, m, l, l, Uf, l, NP, s));
    CK(launch_convert<double>(Uf, l, m, k, U, k, s));
    CK(launch_convert<double>(U1, l, n, k, V, k, s));
    CK(launch_convert<double>(S1, l, 1, k, S, k, s));
    CK(launch_count_positive(S1, k, &pst->rank, s));
    return cudaSuccess;
}

template <typename T>
int backward_entry(const T *A, int64_t m, int64_t n, int64_t lda, const T *S, const T *V,
                   const T *dU, const T *dS, const T *dV, T *dA, tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1 || n > 16384) return -3;
    if (lda < n) return -4;
    if (!S) return -5;
    if (!V) return -6;
    if (!dA) return -10;
    if (!opts) return -11;
    cudaStream_t s = (cudaStream_t)opts->stream;
    const i64 nn = n * n;
    const int spJ = tn_splits(m, n, n, false);
    const int spK = tn_splits(n, n, n, false);
    const int sp = spJ > spK ? spJ : spK;
    const int gy = nn_grid_rows(m, n);
    const bool dbl = sizeof(T) == sizeof(double);
    // FP64_TC: the three tall products (U = A V S^-1, J = U^T dU, dA =
    // [U | dU] BB) on the digit-sliced tensor-core kernels
    const bool oz = opts->mode == TSSVD_FP64_TC;
    const int spO = oz ? oz_tn_splits(m, (int)n, (int)n) : 0;
    struct Bufs {
        double *Ub, *sinv, *M0, *J, *K, *Mc, *Vtr, *BB, *P, *NP, *Sd, *Vd, *dSd, *dVd, *dAd;
        DevStatus *st;
        int *er, *emM, *emB, *exU, *exD;
        unsigned long long *bits;
        uint8_t *big, *bimg;
        double *PO;
    } b;
    const size_t gib = oz ? oz_gram_image_bytes(m, (int)n) : 0;
    size_t bigb = 0;
    if (oz) {
        const size_t r1 = oz_row_image_bytes(m, (int)n), r2 = oz_row_image_bytes(m, 2 * (int)n);
        bigb = 2 * ((gib + 255) / 256 * 256);
        if (r1 > bigb) bigb = r1;
        if (r2 > bigb) bigb = r2;
    }
    auto carve = [&](Bump &w) {
        b.st = w.take<DevStatus>(1);
        if (oz) {
            b.er = w.take<int>(m);
            b.emM = w.take<int>(n);
            b.emB = w.take<int>(n);
            b.exU = w.take<int>(n);
            b.exD = w.take<int>(n);
            b.bits = w.take<unsigned long long>(2 * n);
            b.big = w.take<uint8_t>(bigb);
            b.bimg = w.take<uint8_t>(oz_image_bytes(2 * (int)n, (int)n));
            b.PO = w.take<double>((size_t)spO * nn);
        }
        b.Ub = w.take<double>((size_t)m * 2 * n);
        b.sinv = w.take<double>(n);
        b.M0 = w.take<double>(nn);
        b.J = w.take<double>(nn);
        b.K = w.take<double>(nn);
        b.Mc = w.take<double>(nn);
        b.Vtr = w.take<double>(nn);
        b.BB = w.take<double>(2 * nn);
        b.P = w.take<double>((size_t)sp * nn);
        b.NP = w.take<double>((size_t)gy * n);
        b.Sd = w.take<double>(n);
        b.Vd = w.take<double>(nn);
        b.dSd = w.take<double>(n);
        b.dVd = w.take<double>(nn);
        b.dAd = dbl ? nullptr : w.take<double>((size_t)m * n);
    };
    Bump sz(nullptr, 0);
    carve(sz);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    carve(ws);
    if (ws.overflow) return TSSVD_ENOMEM;
    auto body = [&]() -> cudaError_t {
        CK(cudaMemsetAsync(b.st, 0, sizeof(DevStatus), s));
        // FP64 copies of the small operands
        CK(launch_to_double<T>(S, n, 1, n, b.Sd, n, s));
        CK(launch_to_double<T>(V, n, n, n, b.Vd, n, s));
        if (dS) CK(launch_to_double<T>(dS, n, 1, n, b.dSd, n, s));
        if (dV) CK(launch_to_double<T>(dV, n, n, n, b.dVd, n, s));
        // sinv = 1/S (the discard rule with tol 0 inverts every S_j > 0)
        CK(launch_discard(b.Sd, n, 0.0, b.sinv, nullptr, s));
        // U = A V S^-1 (recomputed), the left half of [U | dU]
        CK(launch_scale2(b.Vd, n, n, n, nullptr, b.sinv, b.M0, n, s));
        if (oz) {
            CK(launch_oz_rowexp<T>(A, lda, m, (int)n, nullptr, b.er, s));
            CK(launch_oz_row_image<T>(A, lda, m, (int)n, nullptr, b.er, b.big, s));
            CK(launch_oz_image(b.M0, n, (int)n, (int)n, nullptr, b.emM, b.bimg, s));
            CK(launch_oz_nn_run<double>(b.big, m, (int)n, b.er, b.bimg, b.emM, (int)n, b.Ub, 2 * n,
                                        b.st, s));
        } else {
            CK(launch_nn<T, double>(A, lda, b.M0, n, m, n, n, b.Ub, 2 * n, b.NP, s));
        }
        if (dU) {
            CK(launch_to_double<T>(dU, n, m, n, b.Ub + n, 2 * n, s));
            // J = U^T dU
            if (oz) {
                uint8_t *imgD = b.big + (gib + 255) / 256 * 256;
                CK(cudaMemsetAsync(b.bits, 0, sizeof(unsigned long long) * 2 * n, s));
                CK(launch_colmax<double>(b.Ub, m, n, 2 * n, b.bits, s));
                CK(launch_colmax<double>(b.Ub + n, m, n, 2 * n, b.bits + n, s));
                CK(launch_oz_exp_from_bits(b.bits, (int)n, b.exU, s));
                CK(launch_oz_exp_from_bits(b.bits + n, (int)n, b.exD, s));
                CK(launch_oz_col_image(b.Ub, 2 * n, m, (int)n, b.exU, b.big, s));
                CK(launch_oz_col_image(b.Ub + n, 2 * n, m, (int)n, b.exD, imgD, s));
                CK(launch_oz_tn(b.big, b.exU, (int)n, imgD, b.exD, (int)n, m, spO, b.PO, b.st, s));
                CK(launch_tn_reduce(b.PO, spO, n, n, nullptr, nullptr, false, b.J, n, s));
            } else {
                CK(launch_tn_partial<double, double>(b.Ub, 2 * n, b.Ub + n, 2 * n, m, n, n, spJ,
                                                     false, b.P, s));
                CK(launch_tn_reduce(b.P, spJ, n, n, nullptr, nullptr, false, b.J, n, s));
            }
        } else {
            CK(cudaMemset2DAsync(b.Ub + n, sizeof(double) * 2 * n, 0, sizeof(double) * n, m, s));
        }
        if (dV) {
            // K = V^T dV
            CK(launch_tn_partial<double, double>(b.Vd, n, b.dVd, n, n, n, n, spK, false, b.P, s));
            CK(launch_tn_reduce(b.P, spK, n, n, nullptr, nullptr, false, b.K, n, s));
        }
        CK(launch_adjoint_core(dU ? b.J : nullptr, dV ? b.K : nullptr, b.Sd, dS ? b.dSd : nullptr,
                               n, b.Mc, s));
        // BB = [Core V^T ; S^-1 V^T]  (2n x n)
        CK(launch_transpose(b.Vd, n, n, n, nullptr, b.Vtr, n, s));
        CK(launch_nn<double, double>(b.Mc, n, b.Vtr, n, n, n, n, b.BB, n, b.NP, s));
        CK(launch_transpose(b.Vd, n, n, n, b.sinv, b.BB + nn, n, s));
        // dA = [U | dU] BB
        if (oz) {
            CK(launch_oz_rowexp<double>(b.Ub, 2 * n, m, 2 * (int)n, nullptr, b.er, s));
            CK(launch_oz_row_image<double>(b.Ub, 2 * n, m, 2 * (int)n, nullptr, b.er, b.big, s));
            CK(launch_oz_image(b.BB, n, 2 * (int)n, (int)n, nullptr, b.emB, b.bimg, s));
            CK(launch_oz_nn_run<T>(b.big, m, 2 * (int)n, b.er, b.bimg, b.emB, (int)n, dA, n, b.st,
                                   s));
        } else if (dbl) {
            CK(launch_nn<double, T>(b.Ub, 2 * n, b.BB, n, m, 2 * n, n, dA, n, b.NP, s));
        } else {
            CK(launch_nn<double, double>(b.Ub, 2 * n, b.BB, n, m, 2 * n, n, b.dAd, n, b.NP, s));
            CK(launch_convert<T>(b.dAd, n, m, n, dA, n, s));
        }
        return cudaSuccess;
    };
    cudaError_t e = body();
    if (e != cudaSuccess) {
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, &b.st->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    return err ? TSSVD_ETIMEOUT : TSSVD_OK;
}

// Adjoint of the rank-k SVD of Algorithm 8 (U m x k, S k, V n x k):
//   dA = [U | dU] [ (Core - S^-1 K^T) V^T + S^-1 dV^T ; S^-1 V^T ]
// with J = U^T dU, K = V^T dV and Core the thin adjoint's core (including
// its -J S^-1 term): the (I - U U^T) and (I - V V^T) projections folded into
// the k x k core and the k x n right factor, so the only m-sized work is
// one tall product (m x 2k by 2k x n) and J.
int lowrank_backward_entry(int64_t m, int64_t n, int64_t k, const double *U, const double *S,
                           const double *V, const double *dU, const double *dS,
                           const double *dV, double *dA, tssvd_opts *opts)
{
    if (m < 1) return -1;
    if (n < 1) return -2;
    if (k < 1 || k > m || k > n || k > 16384) return -3;
    if (!U) return -4;
    if (!S) return -5;
    if (!V) return -6;
    if (!dA) return -10;
    if (!opts) return -11;
    cudaStream_t s = (cudaStream_t)opts->stream;
    const i64 kk = k * k, k2 = 2 * k;
    const int spJ = tn_splits(m, k, k, false);
    const int spK = tn_splits(n, k, k, false);
    const int sp = spJ > spK ? spJ : spK;
    const int gy1 = nn_grid_rows(m, n), gy2 = nn_grid_rows(k, n);
    const int gy = gy1 > gy2 ? gy1 : gy2;
    const bool oz = opts->mode == TSSVD_FP64_TC;
    struct Bufs {
        double *Ub, *Sd, *sinv, *J, *K, *Mc, *Vtr, *BB, *P, *NP;
        DevStatus *st;
        int *er, *emB;
        uint8_t *big, *bimg;
    } b;
    auto carve = [&](Bump &w) {
        b.st = w.take<DevStatus>(1);
        if (oz) {
            b.er = w.take<int>(m);
            b.emB = w.take<int>(n);
            b.big = w.take<uint8_t>(oz_row_image_bytes(m, (int)k2));
            b.bimg = w.take<uint8_t>(oz_image_bytes((int)k2, (int)n));
        }
        b.Ub = w.take<double>((size_t)m * k2);
        b.Sd = w.take<double>(k);
        b.sinv = w.take<double>(k);
        b.J = w.take<double>(kk);
        b.K = w.take<double>(kk);
        b.Mc = w.take<double>(kk);
        b.Vtr = w.take<double>((size_t)k * n);
        b.BB = w.take<double>((size_t)k2 * n);
        b.P = w.take<double>((size_t)sp * kk);
        b.NP = w.take<double>((size_t)gy * n);
    };
    Bump sz(nullptr, 0);
    carve(sz);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    carve(ws);
    if (ws.overflow) return TSSVD_ENOMEM;
    auto body = [&]() -> cudaError_t {
        CK(cudaMemsetAsync(b.st, 0, sizeof(DevStatus), s));
        CK(cudaMemcpyAsync(b.Sd, S, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
        CK(launch_discard(b.Sd, k, 0.0, b.sinv, nullptr, s));
        // [U | dU]
        CK(launch_to_double<double>(U, k, m, k, b.Ub, k2, s));
        if (dU) {
            CK(launch_to_double<double>(dU, k, m, k, b.Ub + k, k2, s));
            CK(launch_tn_partial<double, double>(b.Ub, k2, b.Ub + k, k2, m, k, k, spJ, false, b.P,
                                                 s));
            CK(launch_tn_reduce(b.P, spJ, k, k, nullptr, nullptr, false, b.J, k, s));
        } else {
            CK(cudaMemset2DAsync(b.Ub + k, sizeof(double) * k2, 0, sizeof(double) * k, m, s));
        }
        if (dV) {
            CK(launch_tn_partial<double, double>(V, k, dV, k, n, k, k, spK, false, b.P, s));
            CK(launch_tn_reduce(b.P, spK, k, k, nullptr, nullptr, false, b.K, k, s));
        }
        CK(launch_adjoint_core(dU ? b.J : nullptr, dV ? b.K : nullptr, b.Sd, dS, k, b.Mc, s));
        if (dV) CK(launch_core_fix(b.Mc, b.K, b.sinv, k, s));
        // BB = [Mc V^T + S^-1 dV^T ; S^-1 V^T]  (2k x n)
        CK(launch_transpose(V, k, n, k, nullptr, b.Vtr, n, s));
        CK(launch_nn<double, double>(b.Mc, k, b.Vtr, n, k, k, n, b.BB, n, b.NP, s));
        if (dV) CK(launch_add_scaled_t(dV, k, n, k, b.sinv, b.BB, n, s));
        CK(launch_transpose(V, k, n, k, b.sinv, b.BB + (size_t)k * n, n, s));
        // dA = [U | dU] BB
        if (oz) {
            CK(launch_oz_rowexp<double>(b.Ub, k2, m, (int)k2, nullptr, b.er, s));
            CK(launch_oz_row_image<double>(b.Ub, k2, m, (int)k2, nullptr, b.er, b.big, s));
            CK(launch_oz_image(b.BB, n, (int)k2, (int)n, nullptr, b.emB, b.bimg, s));
            CK(launch_oz_nn_run<double>(b.big, m, (int)k2, b.er, b.bimg, b.emB, (int)n, dA, n,
                                        b.st, s));
        } else {
            CK(launch_nn<double, double>(b.Ub, k2, b.BB, n, m, k2, n, dA, n, b.NP, s));
        }
        return cudaSuccess;
    };
    cudaError_t e = body();
    if (e != cudaSuccess) {
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, &b.st->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    return err ? TSSVD_ETIMEOUT : TSSVD_OK;
}

// Algorithm 1 (passes = 1) or 2 (passes = 2) on X (rows x n, ldx), with
// the mixing Mt = O^T (n' x n', n' = n + (n & 1)) given: B* = X O^T (n odd
// padded to n'), B* = Q R by TSQR, discard of R's diagonal below |R_00| wp,
// [Q = Q2 R2, discard, T = R2 R], SVD of T by one-sided Jacobi, U = Q U~,
// V = O^T V~ (leading n rows and triplets).  st->rank, st->sweeps[2] and
// st->err are written.  oz: the two tall products (B* and U) as
// FP64-accurate digit products on the tensor cores.  Sizing when ws has no
// base.
cudaError_t tsqr_core(const double *X, i64 rows, i64 n, i64 ldx, const double *Mt, double *U,
                      i64 ldu, double *S, double *V, i64 ldv, int passes, double wp,
                      int max_sweeps, Bump &ws, DevStatus *st, cudaStream_t s, bool oz)
{
    const i64 np = n + (n & 1), nn = np * np;
    const int gy = nn_grid_rows(rows, np) > nn_grid_rows(np, np) ? nn_grid_rows(rows, np)
                                                                  : nn_grid_rows(np, np);
    int *keep = ws.take<int>(np), *perm_s = ws.take<int>(np);
    int *ctr = ws.take<int>((size_t)max_sweeps + 4);
    double *Bst = ws.take<double>((size_t)rows * np), *Q1 = ws.take<double>((size_t)rows * np);
    double *R1 = ws.take<double>(nn);
    double *Q2 = passes == 2 ? ws.take<double>((size_t)rows * np) : nullptr;
    double *R2 = passes == 2 ? ws.take<double>(nn) : nullptr;
    double *T = ws.take<double>(nn), *Xw = ws.take<double>(nn), *Jw = ws.take<double>(nn);
    double *Pm = ws.take<double>(nn), *Vo = ws.take<double>(nn), *Pp = ws.take<double>(nn);
    double *work = ws.take<double>(tsqr_workspace_doubles(rows, (int)np));
    double *NP = ws.take<double>((size_t)gy * np);
    double *norms = ws.take<double>(np), *sigma = ws.take<double>(np), *sgn = ws.take<double>(np);
    double *prm = ws.take<double>(jacobi_prm_doubles(np));
    int *er = oz ? ws.take<int>(rows) : nullptr, *em = oz ? ws.take<int>(np) : nullptr;
    uint8_t *aimg = oz ? ws.take<uint8_t>(oz_row_image_bytes(rows, (int)np)) : nullptr;
    uint8_t *bimg = oz ? ws.take<uint8_t>(oz_image_bytes((int)np, (int)np)) : nullptr;
    if (ws.sizing()) return cudaSuccess;
    if (ws.overflow) return cudaErrorMemoryAllocation;
    // C (rows x N) = Xa (rows x K) M (K x N)
    auto tall = [&](const double *Xa, i64 lda_, i64 K, const double *M, i64 ldm, i64 N, double *C,
                    i64 ldc) -> cudaError_t {
        if (!oz) return launch_nn<double, double>(Xa, lda_, M, ldm, rows, K, N, C, ldc, NP, s);
        CK(launch_oz_rowexp<double>(Xa, lda_, rows, (int)K, nullptr, er, s));
        CK(launch_oz_image(M, ldm, (int)K, (int)N, nullptr, em, bimg, s));
        return launch_oz_nn<double, double>(Xa, lda_, rows, (int)K, nullptr, er, aimg, bimg, em,
                                            (int)N, C, ldc, st, s);
    };
    // B* = X O^T = X Mt[0:n, :]
    CK(tall(X, ldx, n, Mt, np, np, Bst, np));
    CK(launch_tsqr(Bst, rows, (int)np, work, R1, Q1, s));
    CK(launch_tsqr_discard(R1, Q1, rows, (int)np, wp, keep, s));
    double *Qf = Q1;
    if (passes == 2) {
        CK(launch_tsqr(Q1, rows, (int)np, work, R2, Q2, s));
        CK(launch_tsqr_discard(R2, Q2, rows, (int)np, wp, keep, s));
        CK(launch_nn<double, double>(R2, np, R1, np, np, np, np, T, np, NP, s));
        Qf = Q2;
    } else {
        CK(cudaMemcpyAsync(T, R1, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    }
    // T = P Sigma V~^T by one-sided Jacobi on the columns of T^T
    CK(launch_orient_copy(nullptr, &st->rank2, T, np, Xw, &st->orient, s));
    CK(launch_jacobi(Xw, np, Jw, np, (int)np, (int)np, max_sweeps, ctr, prm, st, 2, s));
    CK(launch_jacobi_finalize(Xw, np, Jw, np, (int)np, (int)np, norms, perm_s, Pm, np, sigma, Vo,
                              np, s, &st->orient, prm));
    // V = (O^T V~)[0:n, 0:n] = Mt[0:n, :] V~[:, 0:n], then the sign rule
    CK(launch_nn<double, double>(Mt, np, Vo, np, n, np, n, V, ldv, NP, s));
    CK(launch_signs(V, ldv, n, n, sigma, sgn, s));
    CK(launch_count_positive(sigma, n, &st->rank, s));
    // U = Q (P[:, 0:n] diag(sgn))
    CK(launch_scale2(Pm, np, np, n, nullptr, sgn, Pp, n, s));
    CK(tall(Qf, np, np, Pp, n, n, U, ldu));
    CK(launch_convert<double>(sigma, np, 1, n, S, n, s));
    return cudaSuccess;
}

// The C entry of Algorithms 1 and 2: the mixing matrix from the caller's
// random draws, then tsqr_core.  wp = drop_tol^2 (drop_tol is the square
// root of the working precision, as for the Gram algorithms).
int tsqr_entry(const double *A, int64_t m, int64_t n, int64_t lda, const double *theta,
               const int64_t *perm, double *U, double *S, double *V, tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1 || n > 4096) return -3;
    if (lda < n) return -4;
    if (!theta) return -5;
    if (!perm) return -6;
    if (!U) return -7;
    if (!S) return -8;
    if (!V) return -9;
    if (!check_opts(opts, 2)) return -10;
    if (opts->mode != TSSVD_FP64 && opts->mode != TSSVD_FP64_TC) return -10;
    const bool oz = opts->mode == TSSVD_FP64_TC;
    cudaStream_t s = (cudaStream_t)opts->stream;
    const i64 np = n + (n & 1);
    const double wp = opts->drop_tol * opts->drop_tol;
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(1);
    sz.take<int>(1);
    sz.take<double>((size_t)np * np);
    tsqr_core(nullptr, m, n, n, nullptr, nullptr, n, nullptr, nullptr, n, opts->passes, wp,
              opts->max_sweeps, sz, nullptr, s, oz);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    DevStatus *st = ws.take<DevStatus>(1);
    int *bad = ws.take<int>(1);
    double *Mt = ws.take<double>((size_t)np * np);
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_mixing((int)(np / 2), theta, perm, Mt, bad, s);
    if (e == cudaSuccess)
        e = tsqr_core(A, m, n, lda, Mt, U, n, S, V, n, opts->passes, wp, opts->max_sweeps, ws, st,
                      s, oz);
    if (e != cudaSuccess) {
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TSSVD_ENOMEM : TSSVD_ECUDA;
    }
    DevStatus hst;
    int hbad = 0;
    if (cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    if (hbad) return -6;
    if (hst.err) return TSSVD_ETIMEOUT;
    opts->out_rank = hst.rank;
    for (int i = 0; i < 4; i++) opts->sweeps[i] = hst.sweeps[i];
    opts->ranks[0] = opts->ranks[1] = hst.rank;
    if (hst.sweeps[2] < 0) return TSSVD_ENOCONV;
    return hst.rank < n ? TSSVD_RANKDEF : TSSVD_OK;
}

// Algorithm 7: Algorithm 5 with Algorithm 1 in the power steps and
// Algorithm 2 in the last step, feeding Algorithm 6 (the SVD of B = Q^T A
// as the Algorithm 2 TS-SVD of B^T = A^T Q).  Discarded directions are
// removed: every step continues with the width the previous TS-SVD kept,
// read back from the device (2 iters + 2 short host synchronisations), and
// every TS-SVD takes the caller's draw for l columns restricted to its
// width.  The tall products A Q~ and A^T Q run in FP64 FMA or, with
// TSSVD_FP64_TC, on the digit-sliced tensor-core kernels (A's row and
// column digit images built once per call).
int lowrank_tsqr_entry(const double *A, int64_t m, int64_t n, int64_t lda, int64_t k, int64_t l,
                       int iters, const double *Omega, const double *theta,
                       const int64_t *perm, double *U, double *S, double *V, tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1) return -3;
    if (lda < n) return -4;
    if (k < 1 || k > l) return -5;
    if (l < 1 || l > m || l > n || l > 4096) return -6;
    if (iters < 0 || iters > 30) return -7;
    if (!Omega) return -8;
    if (!theta) return -9;
    if (!perm) return -10;
    if (!U) return -11;
    if (!S) return -12;
    if (!V) return -13;
    if (!check_opts(opts, 2)) return -14;
    if (opts->mode != TSSVD_FP64 && opts->mode != TSSVD_FP64_TC) return -14;
    cudaStream_t s = (cudaStream_t)opts->stream;
    const bool oz = opts->mode == TSSVD_FP64_TC;
    const i64 lp = l + (l & 1);
    const int hl = (int)(lp / 2);
    const double wp = opts->drop_tol * opts->drop_tol;
    const int nst = 2 * iters + 2;
    const i64 big = m > n ? m : n;
    const int sp = oz ? oz_tn_splits(m, (int)n, (int)l) : tn_splits(m, n, l, false);
    const int gy = nn_grid_rows(big, l);
    struct Bufs {
        DevStatus *st;
        int *bad;
        i64 *permw;
        double *thw, *Mt, *Qt, *Y, *Q, *Qc, *Bt, *U1, *S1, *V1, *V1s, *Uf, *tS, *tV, *sgn, *P, *NP;
        unsigned long long *bits;
        int *exA, *erA, *exQ, *em;
        uint8_t *rimgA, *cimgA, *cimgQ, *bimg;
        char *sub;
    } b = {};
    size_t sub_bytes = 0;
    {
        Bump probe(nullptr, 0);
        tsqr_core(nullptr, big, l, l, nullptr, nullptr, l, nullptr, nullptr, l, 2, wp,
                  opts->max_sweeps, probe, nullptr, s);
        sub_bytes = probe.off + 256;
    }
    auto carve = [&](Bump &w) {
        b.st = w.take<DevStatus>(nst + 1);
        b.bad = w.take<int>(1);
        b.permw = w.take<i64>(2 * (size_t)hl);
        b.thw = w.take<double>(2 * (size_t)hl);
        b.Mt = w.take<double>((size_t)lp * lp);
        b.Qt = w.take<double>((size_t)n * l);
        b.Y = w.take<double>((size_t)m * l);
        b.Q = w.take<double>((size_t)m * l);
        b.Qc = w.take<double>((size_t)m * l);
        b.Bt = w.take<double>((size_t)n * l);
        b.U1 = w.take<double>((size_t)n * l);
        b.S1 = w.take<double>(l);
        b.V1 = w.take<double>((size_t)l * l);
        b.V1s = w.take<double>((size_t)l * l);
        b.Uf = w.take<double>((size_t)m * l);
        b.tS = w.take<double>(l);
        b.tV = w.take<double>((size_t)l * l);
        b.sgn = w.take<double>(l);
        b.P = w.take<double>((size_t)sp * n * l);
        b.NP = w.take<double>((size_t)gy * l);
        if (oz) {
            b.bits = w.take<unsigned long long>(n > l ? n : l);
            b.exA = w.take<int>(n);
            b.erA = w.take<int>(m);
            b.exQ = w.take<int>(l);
            b.em = w.take<int>(l);
            b.rimgA = w.take<uint8_t>(oz_row_image_bytes(m, (int)n));
            b.cimgA = w.take<uint8_t>(oz_gram_image_bytes(m, (int)n));
            b.cimgQ = w.take<uint8_t>(oz_gram_image_bytes(m, (int)l));
            b.bimg = w.take<uint8_t>(oz_image_bytes((int)n, (int)l));
        }
        b.sub = w.take<char>(sub_bytes);
    };
    Bump sz(nullptr, 0);
    carve(sz);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    carve(ws);
    if (ws.overflow) return TSSVD_ENOMEM;
    int si = 0, code = TSSVD_OK;
    // one TS-SVD of X (rows x w, dense): the restricted draw, the mixing
    // matrix, tsqr_core; returns the kept width (or a negative status)
    auto ts = [&](const double *X, i64 rows, i64 w, int passes, double *Uo, double *So,
                  double *Vo) -> i64 {
        const int hw = (int)((w + 1) / 2);
        DevStatus *st = b.st + si++;
        Bump sw(b.sub, sub_bytes);
        cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
        if (e == cudaSuccess) e = launch_restrict_mix(theta, perm, hl, hw, b.thw, b.permw, b.bad, s);
        if (e == cudaSuccess) e = launch_mixing(hw, b.thw, b.permw, b.Mt, b.bad, s);
        if (e == cudaSuccess)
            e = tsqr_core(X, rows, w, w, b.Mt, Uo, w, So, Vo, w, passes, wp, opts->max_sweeps, sw,
                          st, s);
        if (e != cudaSuccess) return -TSSVD_ECUDA;
        DevStatus h;
        int hbad = 0;
        if (cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&hbad, b.bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return -TSSVD_ECUDA;
        if (hbad) return -100;
        if (h.err) return -TSSVD_ETIMEOUT;
        if (h.sweeps[2] < 0) code = TSSVD_ENOCONV;
        opts->sweeps[2] = h.sweeps[2];
        return h.rank;
    };
    auto fail = [&](i64 r) -> int {
        cudaGetLastError();
        return r == -100 ? -10 : (int)-r;
    };
    if (cudaMemsetAsync(b.bad, 0, sizeof(int), s) != cudaSuccess) return TSSVD_ECUDA;
    if (cudaMemcpyAsync(b.Qt, Omega, sizeof(double) * n * l, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return TSSVD_ECUDA;
    i64 w = l;
    auto err = [&](cudaError_t e) { return e == cudaSuccess; };
    DevStatus *pst = b.st + nst;  // the digit products' bounded waits
    if (cudaMemsetAsync(pst, 0, sizeof(DevStatus), s) != cudaSuccess) return TSSVD_ECUDA;
    // Y = A X (m x c, X n x c dense) and Co = A^T Z (n x c, Z m x c dense)
    auto AX = [&](const double *X, i64 c, double *Yo) -> cudaError_t {
        if (!oz) return launch_nn<double, double>(A, lda, X, c, m, n, c, Yo, c, b.NP, s);
        CK(launch_oz_image(X, c, (int)n, (int)c, nullptr, b.em, b.bimg, s));
        return launch_oz_nn_run<double>(b.rimgA, m, (int)n, b.erA, b.bimg, b.em, (int)c, Yo, c,
                                        pst, s);
    };
    auto AtZ = [&](const double *Z, i64 c, double *Co) -> cudaError_t {
        if (!oz) {
            CK(launch_tn_partial<double, double>(A, lda, Z, c, m, n, c, sp, false, b.P, s));
        } else {
            CK(cudaMemsetAsync(b.bits, 0, sizeof(unsigned long long) * c, s));
            CK(launch_colmax<double>(Z, m, c, c, b.bits, s));
            CK(launch_oz_exp_from_bits(b.bits, (int)c, b.exQ, s));
            CK(launch_oz_col_image(Z, c, m, (int)c, b.exQ, b.cimgQ, s));
            CK(launch_oz_tn(b.cimgA, b.exA, (int)n, b.cimgQ, b.exQ, (int)c, m, sp, b.P, pst, s));
        }
        return launch_tn_reduce(b.P, sp, n, c, nullptr, nullptr, false, Co, c, s);
    };
    if (oz) {
        auto images = [&]() -> cudaError_t {
            CK(cudaMemsetAsync(b.bits, 0, sizeof(unsigned long long) * n, s));
            CK(launch_colmax<double>(A, m, n, lda, b.bits, s));
            CK(launch_oz_exp_from_bits(b.bits, (int)n, b.exA, s));
            CK(launch_oz_rowexp<double>(A, lda, m, (int)n, nullptr, b.erA, s));
            CK(launch_oz_row_image<double>(A, lda, m, (int)n, nullptr, b.erA, b.rimgA, s));
            return launch_oz_col_image(A, lda, m, (int)n, b.exA, b.cimgA, s);
        };
        if (!err(images())) return TSSVD_ECUDA;
    }
    for (int it = 0; it < iters && w > 0; it++) {
        // Y = A Q~ (m x w); Y = Q R (Algorithm 1)
        if (!err(AX(b.Qt, w, b.Y))) return TSSVD_ECUDA;
        i64 r = ts(b.Y, m, w, 1, b.Q, b.tS, b.tV);
        if (r < 0) return fail(r);
        if (r == 0) {
            w = 0;
            break;
        }
        // Q (m x r) compacted, then Y~ = A^T Q (n x r); Y~ = Q~ R~ (Algorithm 1)
        if (cudaMemcpy2DAsync(b.Qc, sizeof(double) * r, b.Q, sizeof(double) * w,
                              sizeof(double) * r, m, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            !err(AtZ(b.Qc, r, b.Bt)))
            return TSSVD_ECUDA;
        const i64 r2 = ts(b.Bt, n, r, 1, b.U1, b.tS, b.tV);
        if (r2 < 0) return fail(r2);
        if (r2 > 0 && cudaMemcpy2DAsync(b.Qt, sizeof(double) * r2, b.U1, sizeof(double) * r,
                                        sizeof(double) * r2, n, cudaMemcpyDeviceToDevice,
                                        s) != cudaSuccess)
            return TSSVD_ECUDA;
        w = r2;
    }
    i64 rb = 0, wq = 0;
    if (w > 0) {
        // Y = A Q~; Y = Q R (Algorithm 2)
        if (!err(AX(b.Qt, w, b.Y))) return TSSVD_ECUDA;
        wq = ts(b.Y, m, w, 2, b.Q, b.tS, b.tV);
        if (wq < 0) return fail(wq);
        if (wq > 0) {
            // Algorithm 6: B^T = A^T Q (n x wq) = U1 S1 V1^T (Algorithm 2); U~ = V1, V = U1
            if (cudaMemcpy2DAsync(b.Qc, sizeof(double) * wq, b.Q, sizeof(double) * w,
                                  sizeof(double) * wq, m, cudaMemcpyDeviceToDevice,
                                  s) != cudaSuccess ||
                !err(AtZ(b.Qc, wq, b.Bt)))
                return TSSVD_ECUDA;
            rb = ts(b.Bt, n, wq, 2, b.U1, b.S1, b.V1);
            if (rb < 0) return fail(rb);
        }
    }
    // outputs: the sign rule on V = U1, U = Q V1 diag(sgn); zeros past rb
    const i64 kk = k < rb ? k : rb;
    bool ok = cudaMemsetAsync(U, 0, sizeof(double) * m * k, s) == cudaSuccess &&
              cudaMemsetAsync(V, 0, sizeof(double) * n * k, s) == cudaSuccess &&
              cudaMemsetAsync(S, 0, sizeof(double) * k, s) == cudaSuccess;
    if (ok && kk > 0) {
        ok = err(launch_signs(b.U1, wq, n, wq, b.S1, b.sgn, s)) &&
             err(launch_scale2(b.V1, wq, wq, wq, nullptr, b.sgn, b.V1s, wq, s)) &&
             err(launch_nn<double, double>(b.Qc, wq, b.V1s, wq, m, wq, wq, b.Uf, wq, b.NP, s)) &&
             cudaMemcpy2DAsync(U, sizeof(double) * k, b.Uf, sizeof(double) * wq,
                               sizeof(double) * kk, m, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
             cudaMemcpy2DAsync(V, sizeof(double) * k, b.U1, sizeof(double) * wq,
                               sizeof(double) * kk, n, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
             cudaMemcpyAsync(S, b.S1, sizeof(double) * kk, cudaMemcpyDeviceToDevice, s) ==
                 cudaSuccess;
    }
    int perr = 0;
    if (!ok ||
        cudaMemcpyAsync(&perr, &pst->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    if (perr) return TSSVD_ETIMEOUT;
    opts->out_rank = kk;
    opts->ranks[0] = (int)w;
    opts->ranks[1] = (int)wq;
    if (code == TSSVD_OK && kk < k) code = TSSVD_RANKDEF;
    return code;
}

// ------------------------------------------------------- host-buffer calls

// Copy streams and chunk events of the host-buffer calls, one set per
// device, created on first use and kept for the process.
constexpr int kHostMaxChunks = 64;
struct HostCopies {
    bool ready = false;
    cudaStream_t in, out;
    cudaEvent_t arrived[kHostMaxChunks], done[kHostMaxChunks], start, in_done, out_done;
};
HostCopies g_host[64];
std::mutex g_host_mu;

int ensure_host_copies(int dev)
{
    HostCopies &H = g_host[dev];
    if (H.ready) return 0;
    if (cudaStreamCreateWithFlags(&H.in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&H.out, cudaStreamNonBlocking) != cudaSuccess)
        return -1;
    cudaEvent_t *all[] = {&H.start, &H.in_done, &H.out_done};
    for (cudaEvent_t *e : all)
        if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return -1;
    for (int k = 0; k < kHostMaxChunks; k++)
        if (cudaEventCreateWithFlags(&H.arrived[k], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&H.done[k], cudaEventDisableTiming) != cudaSuccess)
            return -1;
    H.ready = true;
    return 0;
}

// Rows per chunk: about 256 MB of A, a multiple of 128 (U's row image is
// stored by 128-row tiles), at most kHostMaxChunks chunks.
i64 host_chunk_rows(i64 m, i64 n)
{
    i64 rows = ((i64)(256ll << 20) / (8 * n) + 127) / 128 * 128;
    const i64 least = ((m + kHostMaxChunks - 1) / kHostMaxChunks + 127) / 128 * 128;
    if (rows < least) rows = least;
    if (rows < 128) rows = 128;
    return rows;
}

bool host_overlaps(const tssvd_opts *o) { return o->mode == TSSVD_FP64_TC && o->passes >= 2; }

// Workspace of a host-buffer call: status, device copies of A and U, S, V,
// and the TS-SVD's own (with the chunked Gram partials when overlapping).
void host_sizes(Bump &b, i64 m, i64 n, const tssvd_opts *o, const HostIO *io)
{
    b.take<DevStatus>(1);
    b.take<double>((size_t)m * n);
    b.take<double>((size_t)m * n);
    b.take<double>(n);
    b.take<double>((size_t)n * n);
    if (host_overlaps(o))
        ts_core_oz<double, double>(nullptr, m, n, n, (double *)nullptr, n, (double *)nullptr,
                                   (double *)nullptr, n, o->passes, o->scale, o->drop_tol,
                                   o->max_sweeps, b, nullptr, nullptr, nullptr, 0, io);
    else
        ts_any<double, double>(nullptr, m, n, n, (double *)nullptr, n, (double *)nullptr,
                               (double *)nullptr, n, o->passes, o->scale, o->drop_tol,
                               o->max_sweeps, b, nullptr, nullptr, o->mode);
}

int ts_svd_host_entry(const double *A, i64 m, i64 n, i64 lda, double *U, double *S, double *V,
                      tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1 || n > 16384) return -3;
    if (lda < n) return -4;
    if (!U) return -5;
    if (!S) return -6;
    if (!V) return -7;
    if (!check_opts(opts)) return -8;
    if ((opts->mode == TSSVD_BF16X3 || opts->mode == TSSVD_BF16X6) && n > 256) {
        fprintf(stderr, "tssvd: the mixed-precision modes take n <= 256 (n = %lld)\n",
                (long long)n);
        return -3;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSSVD_ECUDA;
    std::lock_guard<std::mutex> hlk(g_host_mu);  // the chunk events are shared
    if (ensure_host_copies(dev)) return TSSVD_ECUDA;
    HostCopies &H = g_host[dev];
    cudaStream_t s = (cudaStream_t)opts->stream;
    const i64 rows = host_chunk_rows(m, n);
    const int chunks = (int)((m + rows - 1) / rows);
    HostIO io{chunks, rows, H.arrived, H.done, U, n, H.out};
    const bool ov = host_overlaps(opts);

    Bump sz(nullptr, 0);
    host_sizes(sz, m, n, opts, &io);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    DevStatus *st = ws.take<DevStatus>(1);
    double *Ad = ws.take<double>((size_t)m * n), *Ud = ws.take<double>((size_t)m * n);
    double *Sd = ws.take<double>(n), *Vd = ws.take<double>((size_t)n * n);
    auto fail = [&](cudaError_t e) {
        // copies may still be in flight on the copy streams: let them end
        // before the caller's buffers can go away
        cudaStreamSynchronize(H.in);
        cudaStreamSynchronize(H.out);
        cudaStreamSynchronize(s);
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TSSVD_ENOMEM : TSSVD_ECUDA;
    };
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    // A's chunks on the input stream, after the work already queued on s
    if (e == cudaSuccess) e = cudaEventRecord(H.start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(H.in, H.start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(H.out, H.start, 0);
    for (int k = 0; k < chunks && e == cudaSuccess; k++) {
        const i64 r0 = (i64)k * rows, rk = io_rows(&io, m, k);
        e = cudaMemcpy2DAsync(Ad + r0 * n, sizeof(double) * n, A + r0 * lda, sizeof(double) * lda,
                              sizeof(double) * n, rk, cudaMemcpyHostToDevice, H.in);
        if (e == cudaSuccess) e = cudaEventRecord(H.arrived[k], H.in);
    }
    if (e != cudaSuccess) return fail(e);
    if (ov) {
        // the first Gram consumes A's chunks as they land; U leaves in chunks
        e = ts_core_oz<double, double>(Ad, m, n, n, Ud, n, Sd, Vd, n, opts->passes, opts->scale,
                                       opts->drop_tol, opts->max_sweeps, ws, st, s, nullptr, 0,
                                       &io);
    } else {
        e = cudaEventRecord(H.in_done, H.in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, H.in_done, 0);
        if (e == cudaSuccess)
            e = ts_any<double, double>(Ad, m, n, n, Ud, n, Sd, Vd, n, opts->passes, opts->scale,
                                       opts->drop_tol, opts->max_sweeps, ws, st, s, opts->mode);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(U, Ud, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S, Sd, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(V, Vd, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(H.out_done, H.out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, H.out_done, 0);
    if (e != cudaSuccess) return fail(e);
    DevStatus h;
    if (cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cudaErrorUnknown);
    std::vector<DevStatus> v(1, h);
    int code = summarise(v, opts->passes >= 2 ? 3 : 1, nullptr);
    opts->out_rank = h.rank;
    for (int i = 0; i < 4; i++) opts->sweeps[i] = h.sweeps[i];
    opts->ranks[0] = h.rank1;
    opts->ranks[1] = opts->passes >= 2 ? h.rank2 : h.rank1;
    if (code == TSSVD_OK && h.rank < n) code = TSSVD_RANKDEF;
    return code;
}

}  // namespace
}  // namespace tssvd

using namespace tssvd;

extern "C" {

void tssvd_default_opts(tssvd_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->passes = 2;
    o->scale = 1;
    o->drop_tol = sqrt(1e-11);
    o->mode = TSSVD_FP64;
    o->max_sweeps = 50;
}

const char *tssvd_status_string(int st)
{
    switch (st) {
    case TSSVD_OK: return "ok";
    case TSSVD_ENOCONV: return "Jacobi solve did not converge within max_sweeps";
    case TSSVD_RANKDEF: return "numerically rank deficient; trailing outputs are zero";
    case TSSVD_ETIMEOUT: return "device-side wait timed out";
    case TSSVD_ECUDA: return "CUDA runtime error";
    case TSSVD_ENOMEM: return "workspace too small or allocation failed";
    case TSSVD_ECOMM: return "the all-reduce of a row-sharded call failed";
    default: return st < 0 ? "invalid argument" : "unknown status";
    }
}

size_t ts_svd_workspace_size(int64_t m, int64_t n, int elem_bytes, const tssvd_opts *opts)
{
    if (!opts || m < 1 || n < 1) return 0;
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(1);
    if (elem_bytes == 4)
        ts_any<float, float>(nullptr, m, n, n, (float *)nullptr, n, (float *)nullptr,
                             (float *)nullptr, n, opts->passes, opts->scale, opts->drop_tol,
                             opts->max_sweeps, sz, nullptr, nullptr, opts->mode);
    else
        ts_any<double, double>(nullptr, m, n, n, (double *)nullptr, n, (double *)nullptr,
                               (double *)nullptr, n, opts->passes, opts->scale, opts->drop_tol,
                               opts->max_sweeps, sz, nullptr, nullptr, opts->mode);
    return sz.off + 256;
}

int ts_svd(const double *A, int64_t m, int64_t n, int64_t lda, double *U, double *S, double *V,
           tssvd_opts *opts)
{
    return ts_svd_entry<double>(A, m, n, lda, U, S, V, opts);
}

size_t ts_svd_host_workspace_size(int64_t m, int64_t n, const tssvd_opts *opts)
{
    if (!opts || m < 1 || n < 1 || m < n) return 0;
    const i64 rows = host_chunk_rows(m, n);
    HostIO io{(int)((m + rows - 1) / rows), rows, nullptr, nullptr, nullptr, n, nullptr};
    Bump sz(nullptr, 0);
    host_sizes(sz, m, n, opts, &io);
    return sz.off + 256;
}

int ts_svd_host(const double *A, int64_t m, int64_t n, int64_t lda, double *U, double *S,
                double *V, tssvd_opts *opts)
{
    return ts_svd_host_entry(A, m, n, lda, U, S, V, opts);
}

int ts_svd_f32(const float *A, int64_t m, int64_t n, int64_t lda, float *U, float *S, float *V,
               tssvd_opts *opts)
{
    return ts_svd_entry<float>(A, m, n, lda, U, S, V, opts);
}

int ts_svd_rowshard(const double *A, int64_t m_local, int64_t n, int64_t lda, double *U,
                    double *S, double *V, const tssvd_comm *comm, tssvd_opts *opts)
{
    return ts_svd_entry<double>(A, m_local, n, lda, U, S, V, opts, nullptr, false, comm, true);
}

size_t ts_pca_workspace_size(int64_t m, int64_t n, int elem_bytes, const tssvd_opts *opts)
{
    if (!opts || m < 1 || n < 1) return 0;
    const size_t eb = elem_bytes == 4 ? 4 : 8;
    return ts_svd_workspace_size(m, n, elem_bytes, opts) + (size_t)m * n * eb +
           sizeof(double) * (size_t)colsum_rows(m, n) * n + 512;
}

int ts_pca(const double *A, int64_t m, int64_t n, int64_t lda, double *mu, double *U, double *S,
           double *V, tssvd_opts *opts)
{
    return ts_svd_entry<double>(A, m, n, lda, U, S, V, opts, mu, true);
}

int ts_pca_f32(const float *A, int64_t m, int64_t n, int64_t lda, float *mu, float *U, float *S,
               float *V, tssvd_opts *opts)
{
    return ts_svd_entry<float>(A, m, n, lda, U, S, V, opts, mu, true);
}

size_t lowrank_svd_workspace_size(int64_t m, int64_t n, int64_t l, const tssvd_opts *opts)
{
    if (!opts || m < 1 || n < 1 || l < 1) return 0;
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(64);
    lowrank_core(nullptr, m, n, n, l, l, 0, nullptr, nullptr, nullptr, nullptr, opts->drop_tol,
                 opts->max_sweeps, sz, nullptr, nullptr, opts->mode);
    return sz.off + 256;
}

int lowrank_svd(const double *A, int64_t m, int64_t n, int64_t lda, int64_t k, int64_t l,
                int iters, const double *Omega, double *U, double *S, double *V,
                tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1) return -3;
    if (lda < n) return -4;
    if (k < 1 || k > l) return -5;
    if (l < 1 || l > m || l > n || l > 16384) return -6;
    if (iters < 0 || iters > 30) return -7;
    if (!Omega) return -8;
    if (!U) return -9;
    if (!S) return -10;
    if (!V) return -11;
    if (!check_opts(opts)) return -12;
    cudaStream_t s = (cudaStream_t)opts->stream;
    if ((opts->mode == TSSVD_BF16X3 || opts->mode == TSSVD_BF16X6) && l > 256) return -6;
    const int nst = 2 * iters + 3;
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(nst);
    lowrank_core(A, m, n, lda, k, l, iters, Omega, U, S, V, opts->drop_tol, opts->max_sweeps, sz,
                 nullptr, s, opts->mode);
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    int rc = acquire_ws(opts, sz.off, &base, lk);
    if (rc) return rc;
    Bump ws(base, sz.off + 256);
    DevStatus *sts = ws.take<DevStatus>(nst);
    if (cudaMemsetAsync(sts, 0, sizeof(DevStatus) * nst, s) != cudaSuccess) return TSSVD_ECUDA;
    cudaError_t e = lowrank_core(A, m, n, lda, k, l, iters, Omega, U, S, V, opts->drop_tol,
                                 opts->max_sweeps, ws, sts, s, opts->mode);
    if (e != cudaSuccess) {
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TSSVD_ENOMEM : TSSVD_ECUDA;
    }
    std::vector<DevStatus> h(nst);
    if (cudaMemcpyAsync(h.data(), sts, sizeof(DevStatus) * nst, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    int code = TSSVD_OK;
    if (h[nst - 1].err) return TSSVD_ETIMEOUT;  // the products' own waits
    for (int i = 0; i < nst - 1; i++) {
        if (h[i].err) return TSSVD_ETIMEOUT;
        const int solves = (i < 2 * iters) ? 1 : 3;
        for (int j = 0; j < solves; j++)
            if (h[i].sweeps[j] < 0) code = TSSVD_ENOCONV;
    }
    const int rank = h[nst - 1].rank;
    opts->out_rank = rank;
    opts->ranks[0] = h[nst - 2].rank1;
    opts->ranks[1] = h[nst - 2].rank2;
    for (int i = 0; i < 4; i++) opts->sweeps[i] = h[nst - 2].sweeps[i];
    if (code == TSSVD_OK && rank < k) code = TSSVD_RANKDEF;
    return code;
}

int lowrank_svd_tsqr(const double *A, int64_t m, int64_t n, int64_t lda, int64_t k, int64_t l,
                     int iters, const double *Omega, const double *theta, const int64_t *perm,
                     double *U, double *S, double *V, tssvd_opts *opts)
{
    return lowrank_tsqr_entry(A, m, n, lda, k, l, iters, Omega, theta, perm, U, S, V, opts);
}

size_t ts_svd_batched_workspace_size(const tssvd_desc *descs, int count, int elem_bytes,
                                     const tssvd_opts *opts)
{
    if (!descs || count < 1 || !opts || (elem_bytes != 4 && elem_bytes != 8)) return 0;
    if (phased_applies(descs, count, opts))
        return (elem_bytes == 8 ? make_phased_plan<double>(descs, count)
                                : make_phased_plan<float>(descs, count)).total + 256;
    std::vector<int> modes(count, opts->mode == TSSVD_AUTO ? TSSVD_FP64_TC : opts->mode);
    // TSSVD_AUTO may pick either engine: size for the larger
    Plan p1 = elem_bytes == 8 ? make_plan<double>(descs, count, opts, modes)
                              : make_plan<float>(descs, count, opts, modes);
    if (opts->mode != TSSVD_AUTO) return p1.total + 256;
    std::vector<int> m2(count, TSSVD_FP64);
    Plan p2 = elem_bytes == 8 ? make_plan<double>(descs, count, opts, m2)
                              : make_plan<float>(descs, count, opts, m2);
    return std::max(p1.total, p2.total) + 256;
}

int ts_svd_batched(tssvd_desc *descs, int count, int elem_bytes, tssvd_opts *opts)
{
    if (!descs) return -1;
    if (count < 1) return -2;
    if (elem_bytes != 4 && elem_bytes != 8) return -3;
    if (!opts || opts->passes < 1 || opts->passes > 3 || !(opts->drop_tol >= 0.0) ||
        opts->drop_tol >= 1.0 || opts->max_sweeps < 1 || opts->max_sweeps > 1000 ||
        opts->mode < TSSVD_FP64 || opts->mode > TSSVD_AUTO)
        return -4;
    if (phased_applies(descs, count, opts))
        return elem_bytes == 8 ? batched_phased<double>(descs, count, opts)
                               : batched_phased<float>(descs, count, opts);
    return elem_bytes == 8 ? batched_impl<double>(descs, count, opts)
                           : batched_impl<float>(descs, count, opts);
}

size_t ts_gram_workspace_size(int64_t m, int64_t n)
{
    if (m < 1 || n < 1) return 0;
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(1);
    const int sp = tn_splits(m, n, n, true);
    const int tsp = tc_gram_splits(m);
    const int osp = oz_gram_splits(m, (int)n);
    int mx = sp > tsp ? sp : tsp;
    mx = mx > osp ? mx : osp;
    sz.take<double>((size_t)mx * n * n);
    sz.take<unsigned long long>(n);
    sz.take<int>(n);
    sz.take<uint8_t>(oz_gram_image_bytes(m, (int)n));
    return sz.off + 256;
}

// Reads the status block back; TSSVD_ETIMEOUT if a device wait expired.
int finish_call(DevStatus *st, cudaStream_t s)
{
    DevStatus h;
    if (cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    return h.err ? TSSVD_ETIMEOUT : TSSVD_OK;
}

int ts_gram(const double *A, int64_t m, int64_t n, int64_t lda, double *B, tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1 || n > 16384) return -3;
    if (lda < n) return -4;
    if (!B) return -5;
    if (!check_opts(opts)) return -6;
    const int terms = mode_terms(opts->mode);
    if (terms && n > 256) return -3;
    cudaStream_t s = (cudaStream_t)opts->stream;
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    const size_t need = ts_gram_workspace_size(m, n);
    int rc = acquire_ws(opts, need, &base, lk);
    if (rc) return rc;
    Bump ws(base, need + 256);
    DevStatus *st = ws.take<DevStatus>(1);
    const bool oz = opts->mode == TSSVD_FP64_TC;
    const int sp = oz ? oz_gram_splits(m, (int)n)
                      : (terms ? tc_gram_splits(m) : tn_splits(m, n, n, true));
    double *P = ws.take<double>((size_t)sp * n * n);
    unsigned long long *bits = ws.take<unsigned long long>(n);
    int *ex = ws.take<int>(n);
    uint8_t *gimg = ws.take<uint8_t>(oz_gram_image_bytes(m, (int)n));
    if (ws.overflow) return TSSVD_ENOMEM;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (oz) {
        if (e == cudaSuccess) e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long) * n, s);
        if (e == cudaSuccess) e = launch_colmax<double>(A, m, n, lda, bits, s);
        if (e == cudaSuccess) e = launch_oz_exp_from_bits(bits, (int)n, ex, s);
        if (e == cudaSuccess) e = launch_oz_gram<double>(A, lda, m, (int)n, ex, sp, gimg, P, st, s);
    } else if (e == cudaSuccess) {
        e = terms ? launch_tc_gram<double>(A, lda, m, (int)n, terms, sp, P, st, s)
                  : launch_tn_partial<double, double>(A, lda, A, lda, m, n, n, sp, true, P, s);
    }
    if (e == cudaSuccess) e = launch_tn_reduce(P, sp, n, n, nullptr, nullptr, true, B, n, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    return finish_call(st, s);
}

size_t ts_matmul_workspace_size(int64_t m, int64_t k, int64_t n)
{
    if (m < 1 || k < 1 || n < 1) return 0;
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(1);
    const size_t a = tc_split_b_bytes((int)k, (int)n, 3), b = oz_image_bytes((int)k, (int)n);
    sz.take<uint8_t>(a > b ? a : b);
    sz.take<double>((size_t)nn_grid_rows(m, n) * n);
    sz.take<int>(m);
    sz.take<int>(n);
    sz.take<uint8_t>(oz_row_image_bytes(m, (int)k));
    return sz.off + 256;
}

int ts_matmul(const double *A, int64_t m, int64_t k, int64_t lda, const double *M, int64_t n,
              int64_t ldm, double *C, int64_t ldc, tssvd_opts *opts)
{
    if (!A) return -1;
    if (m < 1) return -2;
    if (k < 1 || k > (1 << 20)) return -3;
    if (lda < k) return -4;
    if (!M) return -5;
    if (n < 1 || n > 16384) return -6;
    if (ldm < n) return -7;
    if (!C) return -8;
    if (ldc < n) return -9;
    if (!check_opts(opts)) return -10;
    const int terms = mode_terms(opts->mode);
    if (terms && n > 256) return -6;
    cudaStream_t s = (cudaStream_t)opts->stream;
    void *base = nullptr;
    std::unique_lock<std::mutex> lk;
    const size_t need = ts_matmul_workspace_size(m, k, n);
    int rc = acquire_ws(opts, need, &base, lk);
    if (rc) return rc;
    Bump ws(base, need + 256);
    DevStatus *st = ws.take<DevStatus>(1);
    const size_t ib1 = tc_split_b_bytes((int)k, (int)n, 3), ib2 = oz_image_bytes((int)k, (int)n);
    uint8_t *img = ws.take<uint8_t>(ib1 > ib2 ? ib1 : ib2);
    double *NP = ws.take<double>((size_t)nn_grid_rows(m, n) * n);
    int *er = ws.take<int>(m);
    int *em = ws.take<int>(n);
    uint8_t *aimg = ws.take<uint8_t>(oz_row_image_bytes(m, (int)k));
    if (ws.overflow) return TSSVD_ENOMEM;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (opts->mode == TSSVD_FP64_TC) {
        if (e == cudaSuccess) e = launch_oz_rowexp<double>(A, lda, m, (int)k, nullptr, er, s);
        if (e == cudaSuccess) e = launch_oz_image(M, ldm, (int)k, (int)n, nullptr, em, img, s);
        if (e == cudaSuccess)
            e = launch_oz_nn<double, double>(A, lda, m, (int)k, nullptr, er, aimg, img, em, (int)n,
                                             C, ldc, st, s);
    } else if (terms) {
        if (e == cudaSuccess) e = launch_tc_split_b(M, ldm, (int)k, (int)n, terms, img, s);
        if (e == cudaSuccess)
            e = launch_tc_nn<double>(A, lda, m, (int)k, img, (int)n, terms, C, ldc, st, s);
    } else if (e == cudaSuccess) {
        e = launch_nn<double, double>(A, lda, M, ldm, m, k, n, C, ldc, NP, s);
    }
    if (e != cudaSuccess) {
        fprintf(stderr, "tssvd: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    return finish_call(st, s);
}

int ts_svd_backward(const double *A, int64_t m, int64_t n, int64_t lda, const double *S,
                    const double *V, const double *dU, const double *dS, const double *dV,
                    double *dA, tssvd_opts *opts)
{
    return backward_entry<double>(A, m, n, lda, S, V, dU, dS, dV, dA, opts);
}

size_t ts_svd_tsqr_workspace_size(int64_t m, int64_t n, const tssvd_opts *opts)
{
    if (!opts || m < 1 || n < 1) return 0;
    const i64 np = n + (n & 1);
    Bump sz(nullptr, 0);
    sz.take<DevStatus>(1);
    sz.take<int>(1);
    sz.take<double>((size_t)np * np);
    tsqr_core(nullptr, m, n, n, nullptr, nullptr, n, nullptr, nullptr, n, opts->passes,
              opts->drop_tol * opts->drop_tol, opts->max_sweeps, sz, nullptr, nullptr,
              opts->mode == TSSVD_FP64_TC);
    return sz.off + 256;
}

int ts_svd_tsqr(const double *A, int64_t m, int64_t n, int64_t lda, const double *theta,
                const int64_t *perm, double *U, double *S, double *V, tssvd_opts *opts)
{
    return tsqr_entry(A, m, n, lda, theta, perm, U, S, V, opts);
}

int lowrank_svd_backward(int64_t m, int64_t n, int64_t k, const double *U, const double *S,
                         const double *V, const double *dU, const double *dS, const double *dV,
                         double *dA, tssvd_opts *opts)
{
    return lowrank_backward_entry(m, n, k, U, S, V, dU, dS, dV, dA, opts);
}

int ts_svd_backward_f32(const float *A, int64_t m, int64_t n, int64_t lda, const float *S,
                        const float *V, const float *dU, const float *dS, const float *dV,
                        float *dA, tssvd_opts *opts)
{
    return backward_entry<float>(A, m, n, lda, S, V, dU, dS, dV, dA, opts);
}

}  // extern "C"
