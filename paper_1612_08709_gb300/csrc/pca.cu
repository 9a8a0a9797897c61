// Column means and explicit centering for the PCA entry point: the
// principal components of A are the singular triplets of the centred matrix
// A - 1 mu^T (mu = column means), which the TS-SVD then takes as its input.
// Both kernels are single passes over the m rows and bound by HBM.
#include "common.cuh"

namespace tssvd {
namespace {

inline int ceil_div_i(i64 a, i64 b) { return (int)((a + b - 1) / b); }

// The sums are of the deviations from the first row, A_ij - A_0j (the
// shifted-data form of the mean): their size, and so their rounding error,
// scales with the spread of the column rather than its offset, which
// matters when the means dominate the data.  The shift is added back once,
// in mean_reduce_kernel.
//
// Block (cx, g) sums 32 columns over a fixed row range in FP64; P[g][j]
// receives its partial.  Warps take interleaved rows and their partials
// are added in warp order, so the result does not depend on scheduling.
template <typename T>
__global__ void __launch_bounds__(256) colsum_kernel(const T *__restrict__ A, i64 lda, i64 m,
                                                     i64 n, i64 rows_per,
                                                     double *__restrict__ P)
{
    __shared__ double red[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const i64 c = (i64)blockIdx.x * 32 + lane;
    const i64 r0 = (i64)blockIdx.y * rows_per;
    const i64 r1 = r0 + rows_per < m ? r0 + rows_per : m;
    double acc0 = 0.0, acc1 = 0.0;
    if (c < n) {
        const double ref = (double)A[c];
        i64 r = r0 + warp;
        for (; r + 8 < r1; r += 16) {
            acc0 += (double)A[r * lda + c] - ref;
            acc1 += (double)A[(r + 8) * lda + c] - ref;
        }
        if (r < r1) acc0 += (double)A[r * lda + c] - ref;
    }
    red[warp][lane] = acc0 + acc1;
    __syncthreads();
    if (warp == 0 && c < n) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w][lane];
        P[(i64)blockIdx.y * n + c] = t;
    }
}

// mu_j = A_0j + (sum of the g partials of column j, in order) / m, stored
// as T.
template <typename T>
__global__ void mean_reduce_kernel(const T *__restrict__ A, const double *__restrict__ P, int g,
                                   i64 n, i64 m, T *__restrict__ mu)
{
    const i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int b = 0; b < g; b++) s += P[(i64)b * n + j];
    mu[j] = (T)((double)A[j] + s / (double)m);
}

// C = A - 1 mu^T (C dense, leading dimension n).  One warp per row, rows
// grid-strided; the difference is taken in FP64 and rounded once to T, with
// the stored (rounded) means, so that A = 1 mu^T + C holds for the values
// the caller receives up to that one rounding.
template <typename T>
__global__ void __launch_bounds__(256) center_kernel(const T *__restrict__ A, i64 lda, i64 m,
                                                     i64 n, const T *__restrict__ mu,
                                                     T *__restrict__ C)
{
    const int lane = threadIdx.x & 31;
    const i64 w0 = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const i64 nw = ((i64)gridDim.x * blockDim.x) >> 5;
    for (i64 r = w0; r < m; r += nw) {
        const T *a = A + r * lda;
        T *c = C + r * n;
#pragma unroll 4
        for (i64 j = lane; j < n; j += 32) c[j] = (T)((double)a[j] - (double)mu[j]);
    }
}

}  // namespace

int colsum_rows(i64 m, i64 n)
{
    const int cx = ceil_div_i(n, 32);
    i64 gy = ((i64)num_sms() * 8 + cx - 1) / cx;
    const i64 max_gy = (m + 255) / 256;
    if (gy > max_gy) gy = max_gy;
    if (gy < 1) gy = 1;
    if (gy > 65535) gy = 65535;
    return (int)gy;
}

template <typename T>
cudaError_t launch_col_means(const T *A, i64 lda, i64 m, i64 n, double *P, T *mu, cudaStream_t s)
{
    const int cx = ceil_div_i(n, 32);
    const int gy = colsum_rows(m, n);
    const i64 rows_per = (m + gy - 1) / gy;
    {
        ProfScope ps_("colsum", s);
        colsum_kernel<T><<<dim3(cx, gy), 256, 0, s>>>(A, lda, m, n, rows_per, P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    ProfScope ps_("mean_reduce", s);
    mean_reduce_kernel<T><<<ceil_div_i(n, 128), 128, 0, s>>>(A, P, gy, n, m, mu);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_center(const T *A, i64 lda, i64 m, i64 n, const T *mu, T *C, cudaStream_t s)
{
    i64 blocks = (i64)num_sms() * 8;
    const i64 need = (m + 7) / 8;  // 8 warps (rows) per block
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    ProfScope ps_("center", s);
    center_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(A, lda, m, n, mu, C);
    return cudaGetLastError();
}

template cudaError_t launch_col_means<double>(const double *, i64, i64, i64, double *, double *,
                                              cudaStream_t);
template cudaError_t launch_col_means<float>(const float *, i64, i64, i64, double *, float *,
                                             cudaStream_t);
template cudaError_t launch_center<double>(const double *, i64, i64, i64, const double *,
                                           double *, cudaStream_t);
template cudaError_t launch_center<float>(const float *, i64, i64, i64, const float *, float *,
                                          cudaStream_t);

}  // namespace tssvd
