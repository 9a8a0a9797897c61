// Small device-side steps between the tall passes: the discard rule, the
// diagonal scalings, the assembly of R, the sign convention and type
// conversions.  Everything stays on the device so a call needs no host
// round trip between its passes.
#include "common.cuh"

namespace tssvd {

namespace {

inline unsigned grid_for(i64 total, int per_sm = 8)
{
    i64 b = (total + 255) / 256;
    i64 cap = (i64)num_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Single CTA: smax, then r = 1 + last index kept by the rule (Algorithms 3
// and 4, discard steps: a norm strictly below smax * tol is numerically
// zero).  Columns before r are kept even if an intermediate norm falls
// under the threshold at rounding level.
__global__ void discard_kernel(const double *sig, i64 n, double tol, double *inv, int *rank_out)
{
    __shared__ double smax_s[32];
    __shared__ long long last_s[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mx = 0.0;
    for (i64 j = threadIdx.x; j < n; j += blockDim.x) mx = sig[j] > mx ? sig[j] : mx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if (lane == 0) smax_s[warp] = mx;
    __syncthreads();
    double smax = 0.0;
    for (int w = 0; w < nw; w++) smax = smax_s[w] > smax ? smax_s[w] : smax;
    const double thr = smax * tol;
    long long last = -1;
    for (i64 j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = sig[j];
        if (v > 0.0 && !(v < thr)) last = j > last ? j : last;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long v = __shfl_xor_sync(0xffffffffu, last, o);
        last = v > last ? v : last;
    }
    if (lane == 0) last_s[warp] = last;
    __syncthreads();
    long long r = -1;
    for (int w = 0; w < nw; w++) r = last_s[w] > r ? last_s[w] : r;
    r += 1;
    for (i64 j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = sig[j];
        inv[j] = (j < r && v > 0.0) ? 1.0 / v : 0.0;
    }
    if (threadIdx.x == 0 && rank_out) *rank_out = (int)r;
}

__global__ void scale2_kernel(const double *M, i64 ldm, i64 rows, i64 cols, const double *rs,
                              const double *cs, double *out, i64 ldo)
{
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / cols, j = e % cols;
        double v = M[i * ldm + j];
        if (rs) v *= rs[i];
        if (cs) v *= cs[j];
        out[i * ldo + j] = v;
    }
}

__global__ void build_g_kernel(const double *sig, const double *keep, const double *Vt, i64 ldv,
                               const double *d, i64 n, double *G)
{
    const i64 total = n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 b = e / n, c = e % n;
        const double sb = keep[b] != 0.0 ? sig[b] : 0.0;
        const double dc = d ? d[c] : 1.0;
        G[b * n + c] = sb * Vt[c * ldv + b] * dc;
    }
}

// One warp per column: argmax |V[:, j]| (lowest index on ties).
__global__ void signs_kernel(double *V, i64 ldv, i64 rows, i64 cols, const double *sig,
                             double *sgn)
{
    const i64 j = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= cols) return;
    double best = -1.0;
    i64 bi = 0;
    for (i64 i = lane; i < rows; i += 32) {
        const double a = fabs(V[i * ldv + j]);
        if (a > best) {
            best = a;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    bi = __shfl_sync(0xffffffffu, (long long)bi, 0);
    double s = V[bi * ldv + j] < 0.0 ? -1.0 : 1.0;
    if (sig && !(sig[j] > 0.0)) s = 0.0;
    for (i64 i = lane; i < rows; i += 32) V[i * ldv + j] *= s;
    if (lane == 0) sgn[j] = s;
}

__global__ void count_positive_kernel(const double *sig, i64 n, int *out)
{
    __shared__ int cnt_s[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int c = 0;
    for (i64 j = threadIdx.x; j < n; j += blockDim.x) c += sig[j] > 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt_s[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < nw; w++) t += cnt_s[w];
        *out = t;
    }
}

template <typename T>
__global__ void convert_kernel(const double *src, i64 lds, i64 rows, i64 cols, T *dst, i64 ldd)
{
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / cols, j = e % cols;
        dst[i * ldd + j] = (T)src[i * lds + j];
    }
}

template <typename TS>
__global__ void to_double_kernel(const TS *src, i64 lds, i64 rows, i64 cols, double *dst,
                                 i64 ldd)
{
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / cols, j = e % cols;
        dst[i * ldd + j] = (double)src[i * lds + j];
    }
}

template <typename T>
__global__ void scale_cols_inplace_kernel(T *U, i64 ldu, i64 rows, i64 cols, const double *cs)
{
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / cols, j = e % cols;
        U[i * ldu + j] = (T)((double)U[i * ldu + j] * cs[j]);
    }
}

__global__ void diag_sqrt_kernel(const double *G, i64 ldg, i64 n, double *out)
{
    const i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        const double v = G[j * ldg + j];
        out[j] = v > 0.0 ? sqrt(v) : 0.0;
    }
}

__global__ void keepval_kernel(const double *val, const double *keep, i64 n, double *out)
{
    const i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = (keep[j] != 0.0) ? (val ? val[j] : 1.0) : 0.0;
}

__global__ void transpose_kernel(const double *src, i64 lds, i64 rows, i64 cols, const double *rs,
                                 double *dst, i64 ldd)
{
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / cols, j = e % cols;  // dst[j][i] = src[i][j] * rs[j]
        dst[j * ldd + i] = src[i * lds + j] * (rs ? rs[j] : 1.0);
    }
}

// Core of the thin-SVD adjoint (n x n):
// M_ij = F_ij (J_ij - J_ji) s_j + s_i F_ij (K_ij - K_ji) - J_ij / s_j, i != j
// M_ii = dS_i - J_ii / s_i,  F_ij = 1/(s_j^2 - s_i^2).
__global__ void adjoint_core_kernel(const double *J, const double *K, const double *s,
                                    const double *dS, i64 n, double *M)
{
    const i64 total = n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / n, j = e % n;
        double v = 0.0;
        const double jij = J ? J[i * n + j] : 0.0;
        if (i != j) {
            const double F = 1.0 / (s[j] * s[j] - s[i] * s[i]);
            if (J) v += F * (jij - J[j * n + i]) * s[j];
            if (K) v += s[i] * F * (K[i * n + j] - K[j * n + i]);
        } else if (dS) {
            v += dS[i];
        }
        v -= jij / s[j];
        M[e] = v;
    }
}

// M[a][b] -= K[b][a] * sinv[a] (k x k): the -S^-1 K^T term of the rank-k
// adjoint's core.
__global__ void core_fix_kernel(double *M, const double *K, const double *sinv, i64 k)
{
    const i64 total = k * k;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 a = e / k, b = e - a * k;
        M[e] -= K[b * k + a] * sinv[a];
    }
}

// X[a][j] += sinv[a] * D[j][a] (X k x n, D n x k): adds S^-1 D^T.
__global__ void add_scaled_t_kernel(const double *D, i64 ldd, i64 n, i64 k, const double *sinv,
                                    double *X, i64 ldx)
{
    const i64 total = k * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 a = e / n, j = e - a * n;
        X[a * ldx + j] += sinv[a] * D[j * ldd + a];
    }
}

// Every block derives the orientation itself (n exponents: cheap), so one
// launch both decides and copies.
__global__ void orient_copy_kernel(const double *d, const int *rank2, const double *R, i64 n,
                                   double *X, int *orient)
{
    __shared__ int lo_s, hi_s;
    if (threadIdx.x == 0) {
        lo_s = 1 << 20;
        hi_s = -1;
    }
    __syncthreads();
    if (d) {
        int lo = 1 << 20, hi = -1;
        for (i64 j = threadIdx.x; j < n; j += blockDim.x) {
            const int e = (int)((__double_as_longlong(d[j]) >> 52) & 0x7ff);
            lo = e < lo ? e : lo;
            hi = e > hi ? e : hi;
        }
        atomicMin(&lo_s, lo);
        atomicMax(&hi_s, hi);
    }
    __syncthreads();
    const int flip = (d && *rank2 == n && hi_s - lo_s > kOrientBits) ? 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *orient = flip;
    const i64 nn = n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / n, j = e - i * n;
        X[e] = flip ? R[j * n + i] : R[e];
    }
}

}  // namespace

cudaError_t launch_orient_copy(const double *d, const int *rank2, const double *R, i64 n,
                               double *X, int *orient, cudaStream_t s)
{
    i64 blocks = (n * n + 255) / 256;
    if (blocks > (i64)num_sms() * 4) blocks = (i64)num_sms() * 4;
    if (blocks < 1) blocks = 1;
    ProfScope ps_("orient_copy", s);
    orient_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>(d, rank2, R, n, X, orient);
    return cudaGetLastError();
}

cudaError_t launch_core_fix(double *M, const double *K, const double *sinv, i64 k, cudaStream_t s)
{
    ProfScope ps_("core_fix", s);
    core_fix_kernel<<<grid_for(k * k), 256, 0, s>>>(M, K, sinv, k);
    return cudaGetLastError();
}

cudaError_t launch_add_scaled_t(const double *D, i64 ldd, i64 n, i64 k, const double *sinv,
                                double *X, i64 ldx, cudaStream_t s)
{
    ProfScope ps_("add_scaled_t", s);
    add_scaled_t_kernel<<<grid_for(k * n), 256, 0, s>>>(D, ldd, n, k, sinv, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_diag_sqrt(const double *G, i64 ldg, i64 n, double *out, cudaStream_t s)
{
    ProfScope ps_("diag_sqrt", s);
    diag_sqrt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G, ldg, n, out);
    return cudaGetLastError();
}

namespace {
__global__ void bits_max_kernel(unsigned long long *dst, const unsigned long long *src, i64 n)
{
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (i64)gridDim.x * blockDim.x)
        if (src[j] > dst[j]) dst[j] = src[j];
}
}  // namespace

cudaError_t launch_bits_max(unsigned long long *dst, const unsigned long long *src, i64 n,
                            cudaStream_t s)
{
    ProfScope ps_("bits_max", s);
    bits_max_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

cudaError_t launch_keepval(const double *val, const double *keep, i64 n, double *out,
                           cudaStream_t s)
{
    ProfScope ps_("keepval", s);
    keepval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(val, keep, n, out);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const double *src, i64 lds, i64 rows, i64 cols, const double *rs,
                             double *dst, i64 ldd, cudaStream_t s)
{
    ProfScope ps_("transpose", s);
    transpose_kernel<<<grid_for(rows * cols), 256, 0, s>>>(src, lds, rows, cols, rs, dst, ldd);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_core(const double *J, const double *K, const double *sv,
                                const double *dS, i64 n, double *M, cudaStream_t s)
{
    ProfScope ps_("adjoint_core", s);
    adjoint_core_kernel<<<grid_for(n * n), 256, 0, s>>>(J, K, sv, dS, n, M);
    return cudaGetLastError();
}

cudaError_t launch_discard(const double *sig, i64 n, double tol, double *inv, int *rank_out,
                           cudaStream_t s)
{
    ProfScope ps_("discard", s);
    discard_kernel<<<1, 1024, 0, s>>>(sig, n, tol, inv, rank_out);
    return cudaGetLastError();
}

cudaError_t launch_scale2(const double *M, i64 ldm, i64 rows, i64 cols, const double *rs,
                          const double *cs, double *out, i64 ldo, cudaStream_t s)
{
    ProfScope ps_("scale2", s);
    scale2_kernel<<<grid_for(rows * cols), 256, 0, s>>>(M, ldm, rows, cols, rs, cs, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_build_g(const double *sig, const double *keep, const double *Vt, i64 ldv,
                           const double *d, i64 n, double *G, cudaStream_t s)
{
    ProfScope ps_("build_g", s);
    build_g_kernel<<<grid_for(n * n), 256, 0, s>>>(sig, keep, Vt, ldv, d, n, G);
    return cudaGetLastError();
}

cudaError_t launch_signs(double *V, i64 ldv, i64 rows, i64 cols, const double *sig, double *sgn,
                         cudaStream_t s)
{
    const i64 threads = cols * 32;
    ProfScope ps_("signs", s);
    signs_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(V, ldv, rows, cols, sig, sgn);
    return cudaGetLastError();
}

cudaError_t launch_count_positive(const double *sig, i64 n, int *rank_out, cudaStream_t s)
{
    ProfScope ps_("count_positive", s);
    count_positive_kernel<<<1, 1024, 0, s>>>(sig, n, rank_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert(const double *src, i64 lds, i64 rows, i64 cols, T *dst, i64 ldd,
                           cudaStream_t s)
{
    ProfScope ps_("convert", s);
    convert_kernel<T><<<grid_for(rows * cols), 256, 0, s>>>(src, lds, rows, cols, dst, ldd);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_cols_inplace(T *U, i64 ldu, i64 rows, i64 cols, const double *cs,
                                      cudaStream_t s)
{
    ProfScope ps_("scale_cols", s);
    scale_cols_inplace_kernel<T><<<grid_for(rows * cols, 16), 256, 0, s>>>(U, ldu, rows, cols, cs);
    return cudaGetLastError();
}

template <typename TS>
cudaError_t launch_to_double(const TS *src, i64 lds, i64 rows, i64 cols, double *dst, i64 ldd,
                             cudaStream_t s)
{
    ProfScope ps_("to_double", s);
    to_double_kernel<TS><<<grid_for(rows * cols, 16), 256, 0, s>>>(src, lds, rows, cols, dst, ldd);
    return cudaGetLastError();
}

template cudaError_t launch_convert<double>(const double *, i64, i64, i64, double *, i64,
                                            cudaStream_t);
template cudaError_t launch_convert<float>(const double *, i64, i64, i64, float *, i64,
                                           cudaStream_t);
template cudaError_t launch_scale_cols_inplace<double>(double *, i64, i64, i64, const double *,
                                                       cudaStream_t);
template cudaError_t launch_scale_cols_inplace<float>(float *, i64, i64, i64, const double *,
                                                      cudaStream_t);
template cudaError_t launch_to_double<double>(const double *, i64, i64, i64, double *, i64,
                                              cudaStream_t);
template cudaError_t launch_to_double<float>(const float *, i64, i64, i64, double *, i64,
                                             cudaStream_t);

}  // namespace tssvd
