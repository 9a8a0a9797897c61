// Algorithms 1 and 2 (randomized TS-SVD via TSQR): the random mixing of
// Remark "randomness" as an explicit orthogonal matrix, Householder TSQR
// (leaf QRs of row blocks, a reduction tree over the stacked R factors,
// and Q formed explicitly back down the tree) and the discard of R's
// diagonal.  All in FP64 on the CUDA cores: the leaf QRs are bound by the
// FP64 pipe (2 b n^2 flops per block of b rows).
#include "common.cuh"

namespace tssvd {
namespace {

// Columns 2k and 2k+1 of the real form of Omega = D F S D~ F S~ (one block
// per complex column k), written transposed into Mt = O^T (n2 x n2):
// Mt[2k][2j] = Re w, Mt[2k][2j+1] = Im w, Mt[2k+1][2j] = -Im w,
// Mt[2k+1][2j+1] = Re w, w = Omega_jk.  F is the unitary DFT.  A
// permutation entry outside [0, h) sets bad (and is read as the identity),
// so no index leaves the shared arrays.
__global__ void mixing_kernel(int h, const double *__restrict__ th, const i64 *__restrict__ perm,
                              double *__restrict__ Mt, int *bad)
{
    extern __shared__ double mx_s[];
    double *xr = mx_s, *xi = mx_s + h, *yr = mx_s + 2 * h, *yi = mx_s + 3 * h;
    const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const i64 *p1 = perm, *p2 = perm + h;
    const double *t1 = th, *t2 = th + h;
    auto pidx = [&](const i64 *p, int a) -> int {
        const i64 v = p[a];
        if (v < 0 || v >= h) {
            atomicExch(bad, 1);
            return a;
        }
        return (int)v;
    };
    const double sc = rsqrt((double)h);
    // S~ e_k then F: (F S~ e_k)_a = exp(-2 pi i a q / h) / sqrt(h), q = the
    // position a' with p2[a'] = k, i.e. F applied to a unit vector at q
    for (int a = tid; a < h; a += nt) {
        xr[a] = (pidx(p2, a) == k) ? 1.0 : 0.0;
        xi[a] = 0.0;
    }
    __syncthreads();
    for (int pass = 0; pass < 2; pass++) {
        // y = F x
        for (int a = tid; a < h; a += nt) {
            double sr = 0.0, si = 0.0;
            for (int b = 0; b < h; b++) {
                const double xb = xr[b], xib = xi[b];
                if (xb == 0.0 && xib == 0.0) continue;
                const i64 r = ((i64)a * b) % h;
                double s, c;
                sincospi(-2.0 * (double)r / (double)h, &s, &c);
                sr = fma(xb, c, fma(-xib, s, sr));
                si = fma(xb, s, fma(xib, c, si));
            }
            yr[a] = sr * sc;
            yi[a] = si * sc;
        }
        __syncthreads();
        if (pass == 0) {
            // D~ then S: x_a = (D~ y)_{p1[a]}
            for (int a = tid; a < h; a += nt) {
                const int q = pidx(p1, a);
                double s, c;
                sincos(t2[q], &s, &c);
                xr[a] = yr[q] * c - yi[q] * s;
                xi[a] = yr[q] * s + yi[q] * c;
            }
            __syncthreads();
        }
    }
    const int n2 = 2 * h;
    for (int j = tid; j < h; j += nt) {
        double s, c;
        sincos(t1[j], &s, &c);
        const double wr = yr[j] * c - yi[j] * s, wi = yr[j] * s + yi[j] * c;
        Mt[(i64)(2 * k) * n2 + 2 * j] = wr;
        Mt[(i64)(2 * k) * n2 + 2 * j + 1] = wi;
        Mt[(i64)(2 * k + 1) * n2 + 2 * j] = -wi;
        Mt[(i64)(2 * k + 1) * n2 + 2 * j + 1] = wr;
    }
}

constexpr int kQrThreads = 256;

// Block reduction of one value per thread (all threads get the sum).
__device__ __forceinline__ double qr_block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kQrThreads / 32; w++) t += red[w];
    return t;
}

// Householder QR of row block blk of X (rows [r0, r1), n columns, in
// place): reflection j is I - tau_j v v^T with v_j = 1 and v below the
// diagonal stored in X; R (upper triangle of the block's first n rows) is
// copied, with zeros below, into rows [blk n, blk n + n) of Rs.  Each
// step reduces column j's norm, forms the reflection, then w = v^T X (for
// the trailing columns, warps on interleaved rows, lanes on columns) and
// the rank-one update.
__global__ void __launch_bounds__(kQrThreads) geqr2_kernel(double *__restrict__ X, i64 ldx,
                                                          i64 m, int n, i64 b, int nblk,
                                                          double *__restrict__ tau,
                                                          double *__restrict__ Rs)
{
    extern __shared__ double qr_s[];  // [8][n] partial w, then w
    __shared__ double red[kQrThreads / 32];
    __shared__ double step_s[2];      // tau_j, 1 / (alpha - beta)
    const int blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const i64 r0 = (i64)blk * b;
    const i64 r1 = (blk == nblk - 1) ? m : r0 + b;
    const i64 rows = r1 - r0;
    double *Xb = X + r0 * ldx;
    const int kq = rows < n ? (int)rows : n;
    for (int j = 0; j < kq; j++) {
        // ---- the reflection for column j (rows j .. rows-1)
        double ss = 0.0;
        for (i64 i = j + 1 + tid; i < rows; i += kQrThreads) {
            const double x = Xb[i * ldx + j];
            ss = fma(x, x, ss);
        }
        const double xn2 = qr_block_sum(ss, red);
        if (tid == 0) {
            const double alpha = Xb[(i64)j * ldx + j];
            if (xn2 == 0.0) {
                step_s[0] = 0.0;
                step_s[1] = 0.0;
            } else {
                const double beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
                step_s[0] = (beta - alpha) / beta;
                step_s[1] = 1.0 / (alpha - beta);
                Xb[(i64)j * ldx + j] = beta;
            }
            tau[(i64)blk * n + j] = step_s[0];
        }
        __syncthreads();
        const double tj = step_s[0], scv = step_s[1];
        if (tj == 0.0) continue;  // uniform across the block
        for (i64 i = j + 1 + tid; i < rows; i += kQrThreads) Xb[i * ldx + j] *= scv;
        __syncthreads();
        // ---- w_c = X[j][c] + sum_{i>j} v_i X[i][c], c > j
        for (int c = j + 1 + lane; c < n; c += 32) {
            double acc = 0.0;
            for (i64 i = j + 1 + warp; i < rows; i += kQrThreads / 32)
                acc = fma(Xb[i * ldx + j], Xb[i * ldx + c], acc);
            qr_s[warp * n + c] = acc;
        }
        __syncthreads();
        for (int c = j + 1 + tid; c < n; c += kQrThreads) {
            double w = Xb[(i64)j * ldx + c];
            for (int q = 0; q < kQrThreads / 32; q++) w += qr_s[q * n + c];
            qr_s[c] = w;  // row 0 of the partials is no longer needed for c
        }
        __syncthreads();
        // ---- X[i][c] -= tau v_i w_c for i >= j, c > j
        for (int c = j + 1 + lane; c < n; c += 32) {
            const double tw = tj * qr_s[c];
            if (warp == 0) Xb[(i64)j * ldx + c] -= tw;
            for (i64 i = j + 1 + warp; i < rows; i += kQrThreads / 32)
                Xb[i * ldx + c] = fma(-tw, Xb[i * ldx + j], Xb[i * ldx + c]);
        }
        __syncthreads();
    }
    for (int j = kq; j < n; j++)
        if (tid == 0) tau[(i64)blk * n + j] = 0.0;
    // R into the stacked array (zeros below the diagonal and past kq rows)
    double *R = Rs + (i64)blk * n * n;
    for (int e = tid; e < n * n; e += kQrThreads) {
        const int i = e / n, c = e % n;
        R[e] = (i <= c && i < kq) ? Xb[(i64)i * ldx + c] : 0.0;
    }
}

// Q of row block blk: Y = H_0 ... H_{n-1} [C; 0] with C = rows
// [blk n, blk n + n) of Cin (the block's slice of the next level's Q, or
// the identity at the top), written to rows [r0, r1) of Qout.
__global__ void __launch_bounds__(kQrThreads) org2r_kernel(const double *__restrict__ X, i64 ldx,
                                                          i64 m, int n, i64 b, int nblk,
                                                          const double *__restrict__ tau,
                                                          const double *__restrict__ Cin,
                                                          double *__restrict__ Qout, i64 ldq)
{
    extern __shared__ double qr_s[];
    const int blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const i64 r0 = (i64)blk * b;
    const i64 r1 = (blk == nblk - 1) ? m : r0 + b;
    const i64 rows = r1 - r0;
    const double *Xb = X + r0 * ldx;
    double *Y = Qout + r0 * ldq;
    const int kq = rows < n ? (int)rows : n;
    for (i64 e = tid; e < rows * n; e += kQrThreads) {
        const i64 i = e / n;
        const int c = (int)(e - i * n);
        Y[i * ldq + c] = (i < n) ? (Cin ? Cin[((i64)blk * n + i) * n + c] : (i == c ? 1.0 : 0.0))
                                 : 0.0;
    }
    __syncthreads();
    for (int j = kq - 1; j >= 0; j--) {
        const double tj = tau[(i64)blk * n + j];
        if (tj == 0.0) continue;
        for (int c = lane; c < n; c += 32) {
            double acc = 0.0;
            for (i64 i = j + 1 + warp; i < rows; i += kQrThreads / 32)
                acc = fma(Xb[i * ldx + j], Y[i * ldq + c], acc);
            qr_s[warp * n + c] = acc;
        }
        __syncthreads();
        for (int c = tid; c < n; c += kQrThreads) {
            double w = Y[(i64)j * ldq + c];
            for (int q = 0; q < kQrThreads / 32; q++) w += qr_s[q * n + c];
            qr_s[c] = w;
        }
        __syncthreads();
        for (int c = lane; c < n; c += 32) {
            const double tw = tj * qr_s[c];
            if (warp == 0) Y[(i64)j * ldq + c] -= tw;
            for (i64 i = j + 1 + warp; i < rows; i += kQrThreads / 32)
                Y[i * ldq + c] = fma(-tw, Xb[i * ldx + j], Y[i * ldq + c]);
        }
        __syncthreads();
    }
}

// Discard of Algorithms 1 and 2: row j of R and column j of Q are zeroed
// when |R_jj| < |R_00| wp or R_jj == 0.  keep[j] receives 0/1.
__global__ void tsqr_keep_kernel(const double *R, int n, double wp, int *keep)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double d = fabs(R[(i64)j * n + j]), thr = fabs(R[0]) * wp;
    keep[j] = (d > 0.0 && !(d < thr)) ? 1 : 0;
}

__global__ void tsqr_mask_kernel(double *R, double *Q, i64 m, int n, const int *keep)
{
    const i64 total = m * n + (i64)n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        if (e < m * n) {
            const int c = (int)(e % n);
            if (!keep[c]) Q[e] = 0.0;
        } else {
            const i64 f = e - m * n;
            if (!keep[f / n]) R[f] = 0.0;
        }
    }
}

// The mixing draw for w columns from the draw for l >= w columns (h and hw
// complex entries): the first hw phases of each set and each permutation
// restricted to 0..hw-1 (its entries below hw, in their order).  One
// thread: h is at most a few thousand.  An entry outside [0, h) sets bad.
__global__ void restrict_mix_kernel(const double *th, const i64 *perm, int h, int hw,
                                    double *thw, i64 *permw, int *bad)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int a = 0; a < hw; a++) {
        thw[a] = th[a];
        thw[hw + a] = th[h + a];
    }
    for (int set = 0; set < 2; set++) {
        int c = 0;
        for (int a = 0; a < h; a++) {
            const i64 v = perm[(i64)set * h + a];
            if (v < 0 || v >= h) {
                *bad = 1;
                continue;
            }
            if (v < hw && c < hw) permw[(i64)set * hw + c++] = v;
        }
        for (; c < hw; c++) permw[(i64)set * hw + c] = c;  // only after a bad entry
    }
}

}  // namespace

// ------------------------------------------------------------ launchers

cudaError_t launch_restrict_mix(const double *th, const i64 *perm, int h, int hw, double *thw,
                                i64 *permw, int *bad, cudaStream_t s)
{
    restrict_mix_kernel<<<1, 32, 0, s>>>(th, perm, h, hw, thw, permw, bad);
    return cudaGetLastError();
}

cudaError_t launch_mixing(int h, const double *th, const i64 *perm, double *Mt, int *bad,
                          cudaStream_t s)
{
    ProfScope ps_("mixing", s);
    const size_t smem = sizeof(double) * 4 * (size_t)h;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(mixing_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    mixing_kernel<<<h, 128, smem, s>>>(h, th, perm, Mt, bad);
    return cudaGetLastError();
}

// Row-block size of a TSQR level with `rows` rows: at least n rows per
// block (so every block has a full n x n R), about 4n.
i64 tsqr_block_rows(i64 rows, int n)
{
    i64 b = 4 * (i64)n;
    if (b < 256) b = 256;
    if (b > rows) b = rows;
    return b;
}

int tsqr_blocks(i64 rows, int n)
{
    const i64 b = tsqr_block_rows(rows, n);
    i64 nb = rows / b;
    return nb < 1 ? 1 : (int)nb;
}

// Levels of the reduction tree: level 0 is X (m rows), level l + 1 the
// stacked R factors of level l (blocks(l) * n rows), up to one block.
int tsqr_levels(i64 m, int n, i64 *rows_out, int max_levels)
{
    int L = 0;
    i64 rows = m;
    while (L < max_levels) {
        rows_out[L++] = rows;
        const int nb = tsqr_blocks(rows, n);
        if (nb == 1) break;
        rows = (i64)nb * n;
    }
    return L;
}

size_t tsqr_workspace_doubles(i64 m, int n)
{
    i64 rows[64];
    const int L = tsqr_levels(m, n, rows, 64);
    size_t d = 0;
    for (int l = 0; l < L; l++) {
        const int nb = tsqr_blocks(rows[l], n);
        d += (size_t)nb * n;                     // tau
        d += (size_t)nb * n * n;                 // stacked R (next level's X)
        if (l > 0) d += (size_t)rows[l] * n;     // Q of this level
    }
    return d + 64 * (size_t)L;
}

cudaError_t launch_tsqr(double *X, i64 m, int n, double *work, double *R, double *Q,
                        cudaStream_t s)
{
    i64 rows[64];
    const int L = tsqr_levels(m, n, rows, 64);
    double *taus[64], *Rst[64], *Qs[64];
    double *w = work;
    for (int l = 0; l < L; l++) {
        const int nb = tsqr_blocks(rows[l], n);
        taus[l] = w;
        w += (size_t)nb * n + 8;
        Rst[l] = w;
        w += (size_t)nb * n * n + 8;
        Qs[l] = (l == 0) ? Q : w;
        if (l > 0) w += (size_t)rows[l] * n + 8;
    }
    const size_t smem = sizeof(double) * (kQrThreads / 32) * (size_t)n;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(geqr2_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(org2r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e != cudaSuccess) return e;
    }
    // factorization up the tree
    for (int l = 0; l < L; l++) {
        double *Xl = (l == 0) ? X : Rst[l - 1];
        const int nb = tsqr_blocks(rows[l], n);
        const i64 b = tsqr_block_rows(rows[l], n);
        ProfScope ps_("tsqr_geqr2", s);
        geqr2_kernel<<<nb, kQrThreads, smem, s>>>(Xl, n, rows[l], n, b, nb, taus[l], Rst[l]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // R = the top block's R
    cudaError_t e = cudaMemcpyAsync(R, Rst[L - 1], sizeof(double) * (size_t)n * n,
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // Q down the tree
    for (int l = L - 1; l >= 0; l--) {
        double *Xl = (l == 0) ? X : Rst[l - 1];
        const int nb = tsqr_blocks(rows[l], n);
        const i64 b = tsqr_block_rows(rows[l], n);
        ProfScope ps_("tsqr_org2r", s);
        org2r_kernel<<<nb, kQrThreads, smem, s>>>(Xl, n, rows[l], n, b, nb, taus[l],
                                                   l == L - 1 ? nullptr : Qs[l + 1], Qs[l], n);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_tsqr_discard(double *R, double *Q, i64 m, int n, double wp, int *keep,
                                cudaStream_t s)
{
    ProfScope ps_("tsqr_discard", s);
    tsqr_keep_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, n, wp, keep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    i64 blocks = (m * n + (i64)n * n + 255) / 256;
    if (blocks > (i64)num_sms() * 8) blocks = (i64)num_sms() * 8;
    tsqr_mask_kernel<<<(unsigned)blocks, 256, 0, s>>>(R, Q, m, n, keep);
    return cudaGetLastError();
}

}  // namespace tssvd
