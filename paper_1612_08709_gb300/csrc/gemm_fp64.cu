// FP64 tall products on the CUDA cores (DFMA) and the MaxEntry scan.
//
// GB300 runs FP64 at about 1.2 TFLOP/s (DFMA; its f64 mma.sync is slower),
// so these kernels are bound by the FP64 pipe at any tile shape that keeps
// a few DFMA per shared-memory load: 64 x 64 output tiles, 16-deep K
// slabs, 4 x 4 outputs per thread.  HBM traffic is 8 bytes per FP64 input
// element read once per tile column, far below the 6.8 TB/s roofline.
//
// All reductions are deterministic: split-K partials and per-CTA column
// sums are written to scratch and summed in a fixed order by a second
// kernel (the GPU analogue of the paper's aggregation of per-partition
// Gram matrices, Section 2).
#include <float.h>

#include "common.cuh"

namespace tssvd {

namespace {

constexpr int TB = 64;        // output tile edge
constexpr int KB = 16;        // K slab depth
constexpr int NTHR = 256;     // threads per CTA (16 x 16, 4 x 4 outputs each)

template <typename T>
__device__ __forceinline__ double ld_as_double(const T *p)
{
    return (double)__ldg(p);
}

// ------------------------------------------------------------- colmax
// Column maxima of |A| as bit patterns: non-negative doubles order like
// their bit patterns, so the maxima are integer maxima of the patterns with
// the sign cleared (no FP64 compare, which is slow on this part).  Each
// warp covers 32 columns; rows are strided over the 8 warps, four loads in
// flight per thread.
__device__ __forceinline__ unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// |v| as the bit pattern of the double of the same value, by integer
// operations (FP32 subnormals go through the conversion).
__device__ __forceinline__ unsigned long long abs_bits(float v)
{
    const uint32_t b = __float_as_uint(v) & 0x7FFFFFFFu;
    const uint32_t ef = b >> 23;
    if (ef == 0) return b == 0 ? 0ull : abs_bits((double)__uint_as_float(b));
    if (ef == 0xFF) return 0x7FF0000000000000ull | ((unsigned long long)(b & 0x7FFFFF) << 29);
    return ((unsigned long long)(ef + (1023 - 127)) << 52) | ((unsigned long long)(b & 0x7FFFFF) << 29);
}

template <typename T>
__global__ void __launch_bounds__(256) colmax_kernel(const T *__restrict__ A, i64 m, i64 n,
                                                     i64 lda, i64 rows_per_chunk,
                                                     unsigned long long *bits)
{
    __shared__ unsigned long long red[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const i64 c = (i64)blockIdx.x * 32 + lane;
    const i64 r0 = (i64)blockIdx.y * rows_per_chunk;
    const i64 r1 = r0 + rows_per_chunk < m ? r0 + rows_per_chunk : m;
    unsigned long long mx = 0;
    if (c < n) {
        i64 r = r0 + warp;
        for (; r + 24 < r1; r += 32) {
            const unsigned long long a = abs_bits(__ldg(A + r * lda + c));
            const unsigned long long b = abs_bits(__ldg(A + (r + 8) * lda + c));
            const unsigned long long d = abs_bits(__ldg(A + (r + 16) * lda + c));
            const unsigned long long f = abs_bits(__ldg(A + (r + 24) * lda + c));
            const unsigned long long ab = a > b ? a : b, df = d > f ? d : f;
            const unsigned long long x = ab > df ? ab : df;
            mx = x > mx ? x : mx;
        }
        for (; r < r1; r += 8) {
            const unsigned long long a = abs_bits(__ldg(A + r * lda + c));
            mx = a > mx ? a : mx;
        }
    }
    red[warp][lane] = mx;
    __syncthreads();
    if (warp == 0 && c < n) {
        unsigned long long v = red[0][lane];
        for (int w = 1; w < 8; w++) v = red[w][lane] > v ? red[w][lane] : v;
        atomicMax(bits + c, v);
    }
}

__global__ void pow2_kernel(const unsigned long long *bits, i64 n, double *d, double *dinv)
{
    i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double mx = __longlong_as_double((long long)bits[j]);
    double dj = 1.0;
    if (mx > 0.0 && mx <= DBL_MAX) {
        int e;
        double f = frexp(mx, &e);  // mx = f * 2^e, f in [0.5, 1)
        dj = (f == 0.5) ? mx : ldexp(1.0, e);
    }
    d[j] = dj;
    dinv[j] = 1.0 / dj;  // exact: dj is a power of two
}

// ---------------------------------------------------------- A^T B partials
__device__ __forceinline__ void upper_tile(int t, int T, int &ti, int &tj)
{
    ti = 0;
    while (t >= T - ti) {
        t -= T - ti;
        ti++;
    }
    tj = ti + t;
}

template <typename TA, typename TB_>
__global__ void __launch_bounds__(NTHR) tn_partial_kernel(const TA *__restrict__ A, i64 lda,
                                                          const TB_ *__restrict__ B, i64 ldb,
                                                          i64 K, i64 M, i64 N, i64 kchunk,
                                                          int tiles_n, int upper,
                                                          double *__restrict__ P)
{
    __shared__ double As[KB][TB];
    __shared__ double Bs[KB][TB];
    int ti, tj;
    if (upper)
        upper_tile(blockIdx.x, tiles_n, ti, tj);
    else {
        ti = blockIdx.x / tiles_n;
        tj = blockIdx.x % tiles_n;
    }
    const i64 i0 = (i64)ti * TB, j0 = (i64)tj * TB;
    const i64 kb = (i64)blockIdx.y * kchunk;
    const i64 ke = kb + kchunk < K ? kb + kchunk : K;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    for (i64 k0 = kb; k0 < ke; k0 += KB) {
#pragma unroll
        for (int q = 0; q < (KB * TB) / NTHR; q++) {
            const int e = threadIdx.x + NTHR * q;
            const int kk = e / TB, c = e % TB;
            const i64 kr = k0 + kk;
            double a = 0.0, b = 0.0;
            if (kr < ke) {
                if (i0 + c < M) a = ld_as_double(A + kr * lda + i0 + c);
                if (j0 + c < N) b = ld_as_double(B + kr * ldb + j0 + c);
            }
            As[kk][c] = a;
            Bs[kk][c] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KB; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *Ps = P + (i64)blockIdx.y * M * N;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const i64 row = i0 + ty + 16 * i;
        if (row >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const i64 col = j0 + tx + 16 * j;
            if (col < N) Ps[row * N + col] = acc[i][j];
        }
    }
}

__global__ void tn_reduce_kernel(const double *__restrict__ P, int splits, i64 M, i64 N,
                                 const double *rs, const double *cs, int sym,
                                 double *__restrict__ C, i64 ldc)
{
    const i64 total = M * N;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e / N, j = e % N;
        if (sym && i > j) continue;
        double acc = 0.0;
        for (int s = 0; s < splits; s++) acc += P[(i64)s * total + e];
        if (rs) acc *= rs[i];
        if (cs) acc *= cs[j];
        C[i * ldc + j] = acc;
        if (sym && i != j) C[j * ldc + i] = acc;
    }
}

// ------------------------------------------------------- tall A * B (+norms)
template <typename TA, typename TC>
__global__ void __launch_bounds__(NTHR) nn_kernel(const TA *__restrict__ A, i64 lda,
                                                  const double *__restrict__ B, i64 ldb, i64 m,
                                                  i64 K, i64 N, TC *__restrict__ C, i64 ldc,
                                                  double *__restrict__ NP)
{
    __shared__ double As[KB][TB + 1];
    __shared__ double Bs[KB][TB];
    __shared__ double red[16][TB + 1];
    const i64 j0 = (i64)blockIdx.x * TB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const i64 nrt = (m + TB - 1) / TB;
    double ss[4] = {0.0, 0.0, 0.0, 0.0};

    for (i64 rt = blockIdx.y; rt < nrt; rt += gridDim.y) {
        const i64 r0 = rt * TB;
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
        for (i64 k0 = 0; k0 < K; k0 += KB) {
#pragma unroll
            for (int q = 0; q < (KB * TB) / NTHR; q++) {
                const int e = threadIdx.x + NTHR * q;
                {
                    const int row = e / KB, kk = e % KB;
                    double v = 0.0;
                    if (r0 + row < m && k0 + kk < K) v = ld_as_double(A + (r0 + row) * lda + k0 + kk);
                    As[kk][row] = v;
                }
                {
                    const int kk = e / TB, c = e % TB;
                    double v = 0.0;
                    if (k0 + kk < K && j0 + c < N) v = __ldg(B + (k0 + kk) * ldb + j0 + c);
                    Bs[kk][c] = v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KB; kk++) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const i64 row = r0 + ty + 16 * i;
            if (row >= m) continue;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const i64 col = j0 + tx + 16 * j;
                if (col < N) {
                    if (C) C[row * ldc + col] = (TC)acc[i][j];
                    ss[j] = fma(acc[i][j], acc[i][j], ss[j]);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) red[ty][tx + 16 * j] = ss[j];
    __syncthreads();
    if (threadIdx.x < TB) {
        double s = 0.0;
        for (int t = 0; t < 16; t++) s += red[t][threadIdx.x];
        const i64 col = j0 + threadIdx.x;
        if (col < N) NP[(i64)blockIdx.y * N + col] = s;
    }
}

// Column sums of squares of X (m x n): block (cx, g) covers 32 columns and
// a fixed row range; NP[g][j] receives its partial (deterministic).
__global__ void __launch_bounds__(256) colsumsq_kernel(const double *__restrict__ X, i64 ldx, i64 m,
                                                       i64 n, i64 rows_per,
                                                       double *__restrict__ NP)
{
    __shared__ double red[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const i64 c = (i64)blockIdx.x * 32 + lane;
    const i64 r0 = (i64)blockIdx.y * rows_per;
    const i64 r1 = r0 + rows_per < m ? r0 + rows_per : m;
    double acc = 0.0;
    if (c < n)
        for (i64 r = r0 + warp; r < r1; r += 8) {
            const double v = X[r * ldx + c];
            acc = fma(v, v, acc);
        }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && c < n) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w][lane];
        NP[(i64)blockIdx.y * n + c] = t;
    }
}

__global__ void norms_reduce_kernel(const double *__restrict__ NP, int g, i64 N,
                                    double *__restrict__ out, int take_sqrt)
{
    i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int b = 0; b < g; b++) s += NP[(i64)b * N + j];
    out[j] = take_sqrt ? sqrt(s) : s;
}

__global__ void sqrt_inplace_kernel(double *x, i64 N)
{
    i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) x[j] = sqrt(x[j]);
}

// Row-streaming column maxima (n <= 32 * 16): every warp reads whole rows,
// which are contiguous, and lane l keeps the maxima of columns l + 32 c in
// registers, so a warp has 2 * NCH independent loads in flight per step
// whatever n is.  Warps take interleaved rows of the block's range; the
// block's maxima (|x| as bit patterns, integer compares only) go to bits
// by atomicMax.  (Column sums stay on the column-strip kernels: they need
// FP64 operations per element, which bound them above the HBM time on this
// part, and those kernels keep more warps resident to issue them.)
template <typename T, int NCH>
__global__ void __launch_bounds__(256) colmax_rows_kernel(const T *__restrict__ A, i64 lda, i64 m,
                                                          int n, i64 rows_per,
                                                          unsigned long long *__restrict__ bits)
{
    __shared__ unsigned long long red[8][32 * NCH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const i64 r0 = (i64)blockIdx.x * rows_per;
    const i64 r1 = r0 + rows_per < m ? r0 + rows_per : m;
    unsigned long long mx[NCH];
#pragma unroll
    for (int c = 0; c < NCH; c++) mx[c] = 0ull;
    i64 r = r0 + warp;
    for (; r + 8 < r1; r += 16) {
        const T *a0 = A + r * lda, *a1 = a0 + 8 * lda;
        T v0[NCH], v1[NCH];
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            const int col = lane + 32 * c;
            v0[c] = col < n ? a0[col] : (T)0;
            v1[c] = col < n ? a1[col] : (T)0;
        }
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            const unsigned long long b0 = abs_bits(v0[c]), b1 = abs_bits(v1[c]);
            const unsigned long long b = b0 > b1 ? b0 : b1;
            mx[c] = b > mx[c] ? b : mx[c];
        }
    }
    if (r < r1) {
        const T *a0 = A + r * lda;
#pragma unroll
        for (int c = 0; c < NCH; c++) {
            const int col = lane + 32 * c;
            const unsigned long long b = abs_bits(col < n ? a0[col] : (T)0);
            mx[c] = b > mx[c] ? b : mx[c];
        }
    }
#pragma unroll
    for (int c = 0; c < NCH; c++) red[warp][lane + 32 * c] = mx[c];
    __syncthreads();
    for (int col = threadIdx.x; col < n; col += 256) {
        unsigned long long v = 0ull;
        for (int w = 0; w < 8; w++) v = red[w][col] > v ? red[w][col] : v;
        atomicMax(bits + col, v);
    }
}

inline int ceil_div_i(i64 a, i64 b) { return (int)((a + b - 1) / b); }

}  // namespace

// ------------------------------------------------------------ launchers

int colstat_blocks(i64 m, i64 n)
{
    if (n > 32 * kColStatMaxCh) return 0;
    // three 256-thread blocks per SM stay resident at up to 85 registers
    // (n <= 256), one wave
    i64 g = (i64)num_sms() * 3;
    const i64 cap = (m + 63) / 64;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

template <typename T>
cudaError_t launch_colmax_rows(const T *A, i64 lda, i64 m, i64 n, unsigned long long *bits,
                               cudaStream_t s)
{
    const int g = colstat_blocks(m, n);
    const i64 rows_per = (m + g - 1) / g;
    const int nch = (int)((n + 31) / 32);
    ProfScope ps_("colmax", s);
#define TSSVD_COLMAX(NC) colmax_rows_kernel<T, NC><<<g, 256, 0, s>>>(A, lda, m, (int)n, rows_per, bits)
    if (nch <= 1)
        TSSVD_COLMAX(1);
    else if (nch <= 2)
        TSSVD_COLMAX(2);
    else if (nch <= 4)
        TSSVD_COLMAX(4);
    else if (nch <= 8)
        TSSVD_COLMAX(8);
    else
        TSSVD_COLMAX(16);
#undef TSSVD_COLMAX
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_colmax(const T *A, i64 m, i64 n, i64 lda, unsigned long long *bits,
                          cudaStream_t s)
{
    if (n <= 32 * kColStatMaxCh) return launch_colmax_rows<T>(A, lda, m, n, bits, s);
    const int cx = ceil_div_i(n, 32);
    i64 target = (i64)num_sms() * 8;
    i64 ry = target / cx;
    if (ry < 1) ry = 1;
    i64 max_ry = (m + 255) / 256;
    if (ry > max_ry) ry = max_ry;
    if (ry > 65535) ry = 65535;
    i64 rows_per = (m + ry - 1) / ry;
    ry = (m + rows_per - 1) / rows_per;
    ProfScope ps_("colmax", s);
    colmax_kernel<T><<<dim3(cx, (unsigned)ry), 256, 0, s>>>(A, m, n, lda, rows_per, bits);
    return cudaGetLastError();
}

cudaError_t launch_pow2_scale(const unsigned long long *bits, i64 n, double *d, double *dinv,
                              cudaStream_t s)
{
    ProfScope ps_("pow2", s);
    pow2_kernel<<<ceil_div_i(n, 256), 256, 0, s>>>(bits, n, d, dinv);
    return cudaGetLastError();
}

int tn_splits(i64 K, i64 M, i64 N, bool upper_only)
{
    const int tm = ceil_div_i(M, TB), tn = ceil_div_i(N, TB);
    const i64 tiles = upper_only ? (i64)tm * (tm + 1) / 2 : (i64)tm * tn;
    // CTAs of the partial kernel resident per SM (looked up once).
    static int per_sm = 0;
    if (!per_sm) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tn_partial_kernel<double, double>,
                                                          NTHR, 0) != cudaSuccess ||
            b < 1) {
            cudaGetLastError();
            b = 1;
        }
        per_sm = b;
    }
    // About four waves' worth of CTAs, the count whose last wave is fullest
    // (waves / splits smallest, smaller counts winning within 3%), each
    // split keeping at least 256 rows.
    const i64 slots = (i64)num_sms() * per_sm;
    i64 max_sp = (K + 255) / 256;
    i64 cap = (4 * slots + tiles - 1) / tiles;
    if (cap > max_sp) cap = max_sp;
    if (cap > 65535) cap = 65535;
    if (cap < 1) cap = 1;
    i64 best = 1;
    double best_cost = (double)((tiles + slots - 1) / slots);
    for (i64 sp = 2; sp <= cap; sp++) {
        const double cost = (double)((tiles * sp + slots - 1) / slots) / (double)sp;
        if (cost < best_cost * 0.97) {
            best_cost = cost;
            best = sp;
        }
    }
    return (int)best;
}

template <typename TA, typename TB_>
cudaError_t launch_tn_partial(const TA *A, i64 lda, const TB_ *B, i64 ldb, i64 K, i64 M, i64 N,
                              int splits, bool upper_only, double *P, cudaStream_t s)
{
    const int tm = ceil_div_i(M, TB), tn = ceil_div_i(N, TB);
    const i64 tiles = upper_only ? (i64)tm * (tm + 1) / 2 : (i64)tm * tn;
    i64 kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + KB - 1) / KB * KB;
    if (kchunk < KB) kchunk = KB;
    ProfScope ps_((upper_only ? "tn_gram" : (K > 4 * M ? "tn_tall" : "tn_small")), s);
    tn_partial_kernel<TA, TB_><<<dim3((unsigned)tiles, (unsigned)splits), NTHR, 0, s>>>(
        A, lda, B, ldb, K, M, N, kchunk, tn, upper_only ? 1 : 0, P);
    return cudaGetLastError();
}

cudaError_t launch_tn_reduce(const double *P, int splits, i64 M, i64 N, const double *rs,
                             const double *cs, bool sym, double *C, i64 ldc, cudaStream_t s)
{
    i64 total = M * N;
    i64 blocks = (total + 255) / 256;
    if (blocks > (i64)num_sms() * 16) blocks = (i64)num_sms() * 16;
    if (blocks < 1) blocks = 1;
    ProfScope ps_("tn_reduce", s);
    tn_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, splits, M, N, rs, cs, sym ? 1 : 0, C, ldc);
    return cudaGetLastError();
}

int nn_grid_rows(i64 m, i64 N)
{
    const int gx = ceil_div_i(N, TB);
    i64 gy = ((i64)num_sms() * 4 + gx - 1) / gx;
    const i64 nrt = (m + TB - 1) / TB;
    if (gy > nrt) gy = nrt;
    if (gy < 1) gy = 1;
    if (gy > 65535) gy = 65535;
    return (int)gy;
}

template <typename TA, typename TC>
cudaError_t launch_nn(const TA *A, i64 lda, const double *B, i64 ldb, i64 m, i64 K, i64 N, TC *C,
                      i64 ldc, double *NP, cudaStream_t s)
{
    const int gx = ceil_div_i(N, TB);
    const int gy = nn_grid_rows(m, N);
    ProfScope ps_((m > 4 * K ? "nn_tall" : "nn_small"), s);
    nn_kernel<TA, TC><<<dim3(gx, gy), NTHR, 0, s>>>(A, lda, B, ldb, m, K, N, C, ldc, NP);
    return cudaGetLastError();
}

int colsumsq_rows(i64 m, i64 n)
{
    const int cx = ceil_div_i(n, 32);
    i64 gy = ((i64)num_sms() * 8 + cx - 1) / cx;
    const i64 max_gy = (m + 255) / 256;
    if (gy > max_gy) gy = max_gy;
    if (gy < 1) gy = 1;
    if (gy > 65535) gy = 65535;
    return (int)gy;
}

cudaError_t launch_colsumsq(const double *X, i64 ldx, i64 m, i64 n, double *NP, cudaStream_t s)
{
    const int cx = ceil_div_i(n, 32);
    const int gy = colsumsq_rows(m, n);
    const i64 rows_per = (m + gy - 1) / gy;
    ProfScope ps_("colsumsq", s);
    colsumsq_kernel<<<dim3(cx, gy), 256, 0, s>>>(X, ldx, m, n, rows_per, NP);
    return cudaGetLastError();
}

cudaError_t launch_norms_reduce(const double *NP, int g, i64 N, double *out, cudaStream_t s)
{
    ProfScope ps_("norms_reduce", s);
    norms_reduce_kernel<<<ceil_div_i(N, 256), 256, 0, s>>>(NP, g, N, out, 1);
    return cudaGetLastError();
}

cudaError_t launch_sumsq_reduce(const double *NP, int g, i64 N, double *out, cudaStream_t s)
{
    ProfScope ps_("norms_reduce", s);
    norms_reduce_kernel<<<ceil_div_i(N, 256), 256, 0, s>>>(NP, g, N, out, 0);
    return cudaGetLastError();
}

cudaError_t launch_sqrt_inplace(double *x, i64 N, cudaStream_t s)
{
    ProfScope ps_("sqrt", s);
    sqrt_inplace_kernel<<<ceil_div_i(N, 256), 256, 0, s>>>(x, N);
    return cudaGetLastError();
}

template cudaError_t launch_colmax<double>(const double *, i64, i64, i64, unsigned long long *,
                                           cudaStream_t);
template cudaError_t launch_colmax<float>(const float *, i64, i64, i64, unsigned long long *,
                                          cudaStream_t);
template cudaError_t launch_tn_partial<double, double>(const double *, i64, const double *, i64,
                                                       i64, i64, i64, int, bool, double *,
                                                       cudaStream_t);
template cudaError_t launch_tn_partial<float, float>(const float *, i64, const float *, i64, i64,
                                                     i64, i64, int, bool, double *,
                                                     cudaStream_t);
template cudaError_t launch_tn_partial<float, double>(const float *, i64, const double *, i64,
                                                      i64, i64, i64, int, bool, double *,
                                                      cudaStream_t);
template cudaError_t launch_nn<double, double>(const double *, i64, const double *, i64, i64, i64,
                                               i64, double *, i64, double *, cudaStream_t);
template cudaError_t launch_nn<float, double>(const float *, i64, const double *, i64, i64, i64,
                                              i64, double *, i64, double *, cudaStream_t);
template cudaError_t launch_nn<double, float>(const double *, i64, const double *, i64, i64, i64,
                                              i64, float *, i64, double *, cudaStream_t);
template cudaError_t launch_nn<float, float>(const float *, i64, const double *, i64, i64, i64,
                                             i64, float *, i64, double *, cudaStream_t);

}  // namespace tssvd
