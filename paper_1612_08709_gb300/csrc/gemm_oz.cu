// FP64-accurate tall products on the tcgen05 tensor cores (digit-sliced
// products in the manner of the Ozaki scheme: Ozaki, Ogita, Oishi & Rump,
// "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication", Numer. Algorithms 59, 2012).
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the FP64-accurate products
// (every product of the FP64-accurate mode, and the second
// orthonormalisation pass) are emulated on the BF16 tensor cores:
//
//  * Each operand row (the index that is not summed over) has a power-of-two
//    scale 2^e bounding its entries.  Relative to it a value is cut into
//    seven signed base-128 digits: |v| 2^-e = sum_s d_s 2^(-7(s+1)) + tail,
//    0 <= d_0 <= 128, 0 <= d_s <= 127, |tail| < 2^-49.  The digits are
//    small integers, exact in bfloat16, and are extracted with integer
//    operations on the FP64 bit pattern (no FP64 arithmetic).
//  * A product sum_k a_k b_k becomes sum over digit pairs (s, t) with
//    s + t <= 6 (28 pairs; dropped pairs weigh < 2^-49) of
//    2^(ea+eb-14-7(s+t)) sum_k da_s db_t.  Pairs with the same level
//    L = s + t share one FP32 accumulator in tensor memory (7 levels x 64
//    columns).  Every term is an integer below 2^14 and a level sums at most
//    7 * 128 of them per chunk of 128 rows, so the FP32 sums are exact
//    (< 2^24).
//  * After each 128-row chunk the epilogue warps combine the seven exact
//    level sums with error-free FP32 transformations (TwoSum) into a
//    double-FP32 value and add it to a double-FP32 running sum kept in
//    registers (about 48 significant bits); FP64 is used only once per
//    output element, to scale and store the result.
//
// Warp roles, stages and bounded mbarrier waits as in gemm_tc.cu.
#include "tc_ptx.cuh"

namespace tssvd {

namespace {

using namespace tc;

constexpr int kDig = 7;           // digits per value
constexpr int kLevels = 7;        // levels s + t = 0..6
constexpr int kNT = 64;           // output columns per CTA tile (N of the MMA)
constexpr int kBK = 32;           // rows (Gram) or k (A*M) per stage
constexpr int kChunkStages = 4;   // 128 rows/k per exact FP32 chunk
constexpr int kStages = 2;
constexpr uint32_t kATerm = 128 * kBK * 2;  // 8 KB: one digit of the 128-row operand
constexpr uint32_t kBTerm = kNT * kBK * 2;  // 4 KB: one digit of the 64-row operand
constexpr uint32_t kStageBytes = kDig * (kATerm + kBTerm);

// Exponent of the bit pattern (unbiased), and the 53-bit significand.
__device__ __forceinline__ void dsplit(double v, int &ev, unsigned long long &mant, uint32_t &sign)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    sign = (uint32_t)(b >> 63);
    const int ef = (int)((b >> 52) & 0x7FF);
    if (ef == 0 || ef == 0x7FF) {  // zero, subnormal (negligible), inf/nan
        ev = -100000;
        mant = 0;
        return;
    }
    ev = ef - 1023;
    mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
}

// bfloat16 bit pattern of the signed integer +-d, 0 <= d <= 128.
__device__ __forceinline__ uint32_t bf16_of_int(uint32_t d, uint32_t sign)
{
    if (d == 0) return 0;
    const uint32_t p = 31 - __clz(d);  // 0..7
    return (sign << 15) | ((127 + p) << 7) | ((d << (7 - p)) & 0x7F);
}

// Seven digits of v relative to 2^e (|v| <= 2^e), for a value that is
// prescaled by 2^p first (p added to its exponent).  out[s] = bf16 bits.
__device__ __forceinline__ void digits7(double v, int e, int p, uint32_t (&out)[kDig])
{
    int ev;
    unsigned long long mant;
    uint32_t sign;
    dsplit(v, ev, mant, sign);
    // F = floor(|v| 2^(p-e) 2^49) = mant >> (e - ev - p + 3)
    const int sh = e - (ev + p) + 3;
    unsigned long long F = 0;
    if (mant != 0) {
        if (sh >= 64)
            F = 0;
        else if (sh >= 0)
            F = mant >> sh;
        else
            F = mant << (-sh);  // only when |v 2^p| > 2^e: a scale error; keep bits
    }
    out[0] = bf16_of_int((uint32_t)(F >> 42) & 0xFF, sign);
#pragma unroll
    for (int s = 1; s < kDig; s++) out[s] = bf16_of_int((uint32_t)(F >> (42 - 7 * s)) & 0x7F, sign);
}

__device__ __forceinline__ void digits7(float v, int e, int p, uint32_t (&out)[kDig])
{
    digits7((double)v, e, p, out);
}

// Store 8 values' digits (one 16-byte vector per digit).
__device__ __forceinline__ void store_digits8(uint8_t *base, uint32_t term_stride, uint32_t off,
                                              const uint32_t (&d)[8][kDig])
{
#pragma unroll
    for (int s = 0; s < kDig; s++) {
        uint4 v;
        v.x = d[0][s] | (d[1][s] << 16);
        v.y = d[2][s] | (d[3][s] << 16);
        v.z = d[4][s] | (d[5][s] << 16);
        v.w = d[6][s] | (d[7][s] << 16);
        *reinterpret_cast<uint4 *>(base + (size_t)s * term_stride + off) = v;
    }
}

// Error-free sum of two floats: s + err == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err)
{
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// 8 consecutive FP32 TMEM columns of this thread's lane (no wait).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Drain: add sum_L acc_L 2^-7L (exact level sums in TMEM) to the running
// double-FP32 sums (hi, lo) of this thread's row, 64 columns.
__device__ __forceinline__ void drain_levels(uint32_t tmem_row, float (&hi)[kNT], float (&lo)[kNT])
{
#pragma unroll
    for (int g = 0; g < kNT / 8; g++) {
        uint32_t lv[kLevels][8];
#pragma unroll
        for (int L = 0; L < kLevels; L++) tmem_ld8_nowait(tmem_row + (uint32_t)(L * kNT + g * 8), lv[L]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; c++) {
            float s = __uint_as_float(lv[0][c]), e = 0.f;
#pragma unroll
            for (int L = 1; L < kLevels; L++) {
                float t, er;
                // 2^(-7L) exactly: the level's weight relative to level 0
                const float w = __uint_as_float((uint32_t)(127 - 7 * L) << 23);
                two_sum(s, __uint_as_float(lv[L][c]) * w, t, er);
                s = t;
                e += er;
            }
            float t, er;
            two_sum(hi[g * 8 + c], s, t, er);
            hi[g * 8 + c] = t;
            lo[g * 8 + c] += er + e;
        }
    }
}

// MMAs of one stage: both 16-deep halves, all 28 digit pairs.
__device__ __forceinline__ void issue_stage(uint32_t abase, uint32_t bbase, uint32_t tmem,
                                            uint32_t &started)
{
    const uint32_t idesc = idesc_bf16(128, kNT);
#pragma unroll
    for (int h = 0; h < kBK / 16; h++) {
#pragma unroll
        for (int s = 0; s < kDig; s++) {
#pragma unroll
            for (int t = 0; t < kDig - s; t++) {
                const int L = s + t;
                const uint64_t ad = sdesc(abase + s * kATerm + h * (128 * 32), 128, 256);
                const uint64_t bd = sdesc(bbase + t * kBTerm + h * (kNT * 32), 128, 256);
                const uint32_t acc = (started >> L) & 1u;
                mma_bf16(tmem + (uint32_t)(L * kNT), ad, bd, idesc, acc);
                started |= 1u << L;
            }
        }
    }
}

// Upper tiles of the Gram: i-blocks of 128 (ti), j-blocks of 64 (tj) that
// contain some i <= j.
__device__ __forceinline__ bool gram_tile(int t, int n, int &ti, int &tj)
{
    const int TI = (n + 127) / 128, TJ = (n + kNT - 1) / kNT;
    int c = 0;
    for (int a = 0; a < TI; a++)
        for (int b = 0; b < TJ; b++)
            if (b * kNT + kNT - 1 >= a * 128) {
                if (c == t) {
                    ti = a;
                    tj = b;
                    return true;
                }
                c++;
            }
    return false;
}

// ----------------------------------------------------------------- Gram
// P[split][i][j] (n x n, FP64) for the (i, j) of the CTA's tile:
// sum over the split's rows of X[k][i] X[k][j]; ex[c] bounds column c.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
    oz_gram_kernel(const T *__restrict__ X, i64 ldx, i64 m, int n, const int *__restrict__ ex,
                   i64 rows_per_split, double *__restrict__ P, DevStatus *st)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int exs[128 + kNT];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = &st->err;
    int ti = 0, tj = 0;
    gram_tile(blockIdx.x, n, ti, tj);
    const int i0 = ti * 128, j0 = tj * kNT;
    const i64 r0 = (i64)blockIdx.y * rows_per_split;
    const i64 r1 = r0 + rows_per_split < m ? r0 + rows_per_split : m;
    const int nkb = r1 > r0 ? (int)((r1 - r0 + kBK - 1) / kBK) : 0;
    const int nchunks = (nkb + kChunkStages - 1) / kChunkStages;

    for (int c = threadIdx.x; c < 128 + kNT; c += blockDim.x) {
        const int col = c < 128 ? i0 + c : j0 + c - 128;
        exs[c] = col < n ? ex[col] : 0;
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full_bar[s], kProducers);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, kEpilogue);
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) tmem_alloc(&tmem_base_s, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp < 4) {
        const int tid = threadIdx.x;
        for (int kb = 0; kb < nkb; kb++) {
            const int s = kb % kStages;
            if (!mbar_wait(&empty_bar[s], ((kb / kStages) & 1) ^ 1, err)) break;
            uint8_t *stage = smem_raw + (size_t)s * kStageBytes;
            const i64 k0 = r0 + (i64)kb * kBK;
            // items: (operand row c of 192, 8-row chunk q of 4)
            for (int it = tid; it < (128 + kNT) * (kBK / 8); it += kProducers) {
                const int c = it % (128 + kNT), q = it / (128 + kNT);
                const int col = c < 128 ? i0 + c : j0 + c - 128;
                const int e = exs[c];
                uint32_t d[8][kDig];
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    const i64 k = k0 + 8 * q + r;
                    const T v = (col < n && k < r1) ? X[k * ldx + col] : (T)0;
                    digits7(v, e, 0, d[r]);
                }
                if (c < 128) {
                    const uint32_t off = (uint32_t)(q >> 1) * (128 * 32) + (uint32_t)(c >> 3) * 256 +
                                         (uint32_t)(q & 1) * 128 + (uint32_t)(c & 7) * 16;
                    store_digits8(stage, kATerm, off, d);
                } else {
                    const int cb = c - 128;
                    const uint32_t off = (uint32_t)(q >> 1) * (kNT * 32) + (uint32_t)(cb >> 3) * 256 +
                                         (uint32_t)(q & 1) * 128 + (uint32_t)(cb & 7) * 16;
                    store_digits8(stage + kDig * kATerm, kBTerm, off, d);
                }
            }
            fence_proxy_async();
            mbar_arrive(&full_bar[s]);
        }
    } else if (warp < 8) {
        const int ew = warp - 4;
        float hi[kNT], lo[kNT];
#pragma unroll
        for (int j = 0; j < kNT; j++) {
            hi[j] = 0.f;
            lo[j] = 0.f;
        }
        const uint32_t trow = tmem + ((uint32_t)(ew * 32) << 16);
        bool ok = true;
        for (int ch = 0; ch < nchunks; ch++) {
            if (!mbar_wait(&acc_full, ch & 1, err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            drain_levels(trow, hi, lo);
            tc_fence_before();
            mbar_arrive(&acc_empty);
        }
        if (ok) {
            const int il = ew * 32 + lane;
            const int i = i0 + il;
            if (i < n) {
                double *Prow = P + (i64)blockIdx.y * n * n + (i64)i * n;
                const int ei = exs[il];
#pragma unroll
                for (int jj = 0; jj < kNT; jj++) {
                    const int j = j0 + jj;
                    if (j < n) Prow[j] = ldexp((double)hi[jj] + (double)lo[jj], ei + exs[128 + jj] - 14);
                }
            }
        }
    } else {
        if (lane == 0) {
            int kb = 0;
            bool ok = true;
            for (int ch = 0; ch < nchunks && ok; ch++) {
                if (ch > 0) {
                    if (!mbar_wait(&acc_empty, (ch - 1) & 1, err)) break;
                    tc_fence_after();
                }
                uint32_t started = 0;
                const int kb_end = (ch + 1) * kChunkStages < nkb ? (ch + 1) * kChunkStages : nkb;
                for (; kb < kb_end; kb++) {
                    const int s = kb % kStages;
                    if (!mbar_wait(&full_bar[s], (kb / kStages) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = saddr(smem_raw + (size_t)s * kStageBytes);
                    issue_stage(base, base + kDig * kATerm, tmem, started);
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full);
            }
            mma_commit(&done_bar);
            mbar_wait_drain(&done_bar, 0);
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 8) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- A * M
// C[r][j] = sum_k A[r][k] M[k][j] for the CTA's tiles (128 rows x 64
// columns, persistent over tiles with the column tile fastest).  A's
// column k is prescaled by 2^pk[k] (exact) and its row r is bounded by
// 2^er[r]; img holds the digits of diag(2^-pk) M per (column tile, 32-deep
// k block), 7 x 4 KB each, with the column exponents em.
template <typename T, typename TC>
__global__ void __launch_bounds__(kThreads, 1)
    oz_nn_kernel(const T *__restrict__ A, i64 lda, i64 m, int K, const int *__restrict__ pk,
                 const int *__restrict__ er, const uint8_t *__restrict__ img,
                 const int *__restrict__ em, int N, TC *__restrict__ C, i64 ldc, DevStatus *st)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = &st->err;
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    const int nchunks = (nkb + kChunkStages - 1) / kChunkStages;
    const int TN = (N + kNT - 1) / kNT;
    const i64 ntiles = (m + 127) / 128 * TN;
    const int my_tiles =
        (i64)blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const size_t img_tile = (size_t)nkb * kDig * kBTerm;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full_bar[s], kProducers);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, kEpilogue);
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) tmem_alloc(&tmem_base_s, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp < 4) {
        const int tid = threadIdx.x;
        int f = 0, last_copy = -1;
        bool ok = true;
        for (int ti = 0; ti < my_tiles && ok; ti++) {
            const i64 t = (i64)blockIdx.x + (i64)ti * gridDim.x;
            const i64 rbase = (t / TN) * 128;
            const int nt = (int)(t % TN);
            for (int kb = 0; kb < nkb; kb++, f++) {
                const int s = f % kStages;
                if (!mbar_wait(&empty_bar[s], ((f / kStages) & 1) ^ 1, err)) {
                    ok = false;
                    break;
                }
                uint8_t *stage = smem_raw + (size_t)s * kStageBytes;
                if (tid == 0) {
                    const uint32_t bytes = kDig * kBTerm;
                    mbar_expect_tx(&full_bar[s], bytes);
                    bulk_g2s(stage + kDig * kATerm, img + (size_t)nt * img_tile + (size_t)kb * bytes,
                             bytes, &full_bar[s]);
                    last_copy = f;
                }
                const int k0 = kb * kBK;
                // items: (row r of 128, 8-k chunk q of 4)
                for (int it = tid; it < 128 * (kBK / 8); it += kProducers) {
                    const int r = it >> 2, q = it & 3;
                    const i64 row = rbase + r;
                    const int e = row < m ? er[row] : 0;
                    uint32_t d[8][kDig];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int k = k0 + 8 * q + u;
                        const bool in = row < m && k < K;
                        const T v = in ? A[row * lda + k] : (T)0;
                        digits7(v, e, (in && pk) ? pk[k] : 0, d[u]);
                    }
                    const uint32_t off = (uint32_t)(q >> 1) * (128 * 32) + (uint32_t)(r >> 3) * 256 +
                                         (uint32_t)(q & 1) * 128 + (uint32_t)(r & 7) * 16;
                    store_digits8(stage, kATerm, off, d);
                }
                fence_proxy_async();
                mbar_arrive(&full_bar[s]);
            }
        }
        if (tid == 0 && last_copy >= 0)
            mbar_wait_drain(&full_bar[last_copy % kStages], (last_copy / kStages) & 1);
    } else if (warp < 8) {
        const int ew = warp - 4;
        const uint32_t trow = tmem + ((uint32_t)(ew * 32) << 16);
        int ch_global = 0;
        bool ok = true;
        for (int ti = 0; ti < my_tiles && ok; ti++) {
            const i64 t = (i64)blockIdx.x + (i64)ti * gridDim.x;
            const i64 row = (t / TN) * 128 + ew * 32 + lane;
            const int nt = (int)(t % TN);
            float hi[kNT], lo[kNT];
#pragma unroll
            for (int j = 0; j < kNT; j++) {
                hi[j] = 0.f;
                lo[j] = 0.f;
            }
            for (int ch = 0; ch < nchunks; ch++, ch_global++) {
                if (!mbar_wait(&acc_full, ch_global & 1, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                drain_levels(trow, hi, lo);
                tc_fence_before();
                mbar_arrive(&acc_empty);
            }
            if (!ok) break;
            if (row < m) {
                const int e = er[row];
#pragma unroll
                for (int jj = 0; jj < kNT; jj++) {
                    const int j = nt * kNT + jj;
                    if (j < N) C[row * ldc + j] = (TC)ldexp((double)hi[jj] + (double)lo[jj], e + em[j] - 14);
                }
            }
        }
    } else {
        if (lane == 0) {
            int f = 0, ch_global = 0;
            bool ok = true;
            for (int ti = 0; ti < my_tiles && ok; ti++) {
                for (int ch = 0; ch < nchunks && ok; ch++, ch_global++) {
                    if (ch_global > 0) {
                        if (!mbar_wait(&acc_empty, (ch_global - 1) & 1, err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    uint32_t started = 0;
                    const int kb_end = (ch + 1) * kChunkStages < nkb ? (ch + 1) * kChunkStages : nkb;
                    for (int kb = ch * kChunkStages; kb < kb_end; kb++, f++) {
                        const int s = f % kStages;
                        if (!mbar_wait(&full_bar[s], (f / kStages) & 1, err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = saddr(smem_raw + (size_t)s * kStageBytes);
                        issue_stage(base, base + kDig * kATerm, tmem, started);
                        mma_commit(&empty_bar[s]);
                    }
                    if (!ok) break;
                    mma_commit(&acc_full);
                }
            }
            mma_commit(&done_bar);
            mbar_wait_drain(&done_bar, 0);
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 8) tmem_dealloc(tmem, kTmemCols);
}

// Column exponents of diag(2^-pk) M (K x N): em[j] = smallest e with
// |M[k][j] 2^-pk[k]| <= 2^e for all k (one warp per column).
__global__ void oz_colexp_kernel(const double *__restrict__ M, i64 ldm, int K, int N,
                                 const int *__restrict__ pk, int *__restrict__ em)
{
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= N) return;
    int mx = -100000;
    for (int k = lane; k < K; k += 32) {
        int ev;
        unsigned long long mant;
        uint32_t sign;
        dsplit(M[(i64)k * ldm + j], ev, mant, sign);
        if (mant) {
            // |v| < 2^(ev+1); exact powers of two need only 2^ev
            const int e = (mant == (1ull << 52)) ? ev : ev + 1;
            const int eff = e - (pk ? pk[k] : 0);
            mx = eff > mx ? eff : mx;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if (lane == 0) em[j] = mx < -1000 ? 0 : mx;
}

// Digit image of diag(2^-pk) M: per column tile nt and 32-deep k block kb,
// 7 digit blocks of 64 rows (j) x 32 k in the K-major no-swizzle layout.
__global__ void oz_image_kernel(const double *__restrict__ M, i64 ldm, int K, int N,
                                const int *__restrict__ pk, const int *__restrict__ em,
                                uint8_t *__restrict__ img)
{
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    const int TN = (N + kNT - 1) / kNT;
    const i64 total = (i64)TN * nkb * kNT * (kBK / 8);
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const int jj = (int)(e % kNT);
        const int q = (int)((e / kNT) % (kBK / 8));
        const int kb = (int)((e / (kNT * (kBK / 8))) % nkb);
        const int nt = (int)(e / ((i64)kNT * (kBK / 8) * nkb));
        const int j = nt * kNT + jj;
        const int ej = j < N ? em[j] : 0;
        uint32_t d[8][kDig];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = kb * kBK + 8 * q + u;
            const bool in = k < K && j < N;
            digits7(in ? M[(i64)k * ldm + j] : 0.0, ej, (in && pk) ? -pk[k] : 0, d[u]);
        }
        uint8_t *blk = img + ((size_t)nt * nkb + kb) * kDig * kBTerm;
        const uint32_t off = (uint32_t)(q >> 1) * (kNT * 32) + (uint32_t)(jj >> 3) * 256 +
                             (uint32_t)(q & 1) * 128 + (uint32_t)(jj & 7) * 16;
        store_digits8(blk, kBTerm, off, d);
    }
}

// Row exponents of A diag(2^pk): er[r] = smallest e bounding the row.
template <typename T>
__global__ void oz_rowexp_kernel(const T *__restrict__ A, i64 lda, i64 m, int K,
                                 const int *__restrict__ pk, int *__restrict__ er)
{
    const i64 r = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= m) return;
    int mx = -100000;
    for (int k = lane; k < K; k += 32) {
        int ev;
        unsigned long long mant;
        uint32_t sign;
        dsplit((double)A[r * lda + k], ev, mant, sign);
        if (mant) {
            const int e = (mant == (1ull << 52)) ? ev : ev + 1;
            const int eff = e + (pk ? pk[k] : 0);
            mx = eff > mx ? eff : mx;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if (lane == 0) er[r] = mx < -1000 ? 0 : mx;
}

// Exponents from MaxEntry bit patterns: ex[j] = log2 of the smallest power
// of two >= max |X[:, j]| (0 for a zero column).
__global__ void oz_exp_from_bits_kernel(const unsigned long long *bits, int n, int *ex)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int ev;
    unsigned long long mant;
    uint32_t sign;
    dsplit(__longlong_as_double((long long)bits[j]), ev, mant, sign);
    ex[j] = mant == 0 ? 0 : ((mant == (1ull << 52)) ? ev : ev + 1);
}

// pk[k] = round(log2(s[k])) as an integer (0 when s[k] <= 0): the
// power-of-two prescale nearest to a column scaling s.
__global__ void oz_pow2_of_kernel(const double *s, int n, int *pk)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int ev;
    unsigned long long mant;
    uint32_t sign;
    dsplit(s[j], ev, mant, sign);
    // round to nearest power: up when the significand exceeds sqrt(2)
    const unsigned long long sqrt2_mant = 0x16A09E667F3BCDull;  // sqrt(2) * 2^52
    pk[j] = mant == 0 ? 0 : (mant > sqrt2_mant ? ev + 1 : ev);
}

__global__ void neg_int_kernel(const int *in, int n, int *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = -in[j];
}

inline unsigned grid_cap(i64 total, int per_sm = 8)
{
    i64 b = (total + 255) / 256;
    const i64 cap = (i64)num_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

int oz_gram_tiles(int n)
{
    const int TI = (n + 127) / 128, TJ = (n + kNT - 1) / kNT;
    int c = 0;
    for (int a = 0; a < TI; a++)
        for (int b = 0; b < TJ; b++)
            if (b * kNT + kNT - 1 >= a * 128) c++;
    return c;
}

int oz_gram_splits(i64 m, int n)
{
    const int tiles = oz_gram_tiles(n);
    i64 sp = ((i64)num_sms() + tiles - 1) / tiles;
    const i64 max_sp = (m + 255) / 256;
    if (sp > max_sp) sp = max_sp;
    return sp < 1 ? 1 : (int)sp;
}

size_t oz_image_bytes(int K, int N)
{
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    const int TN = (N + kNT - 1) / kNT;
    return (size_t)TN * nkb * kDig * kBTerm;
}

template <typename T>
cudaError_t launch_oz_gram(const T *X, i64 ldx, i64 m, int n, const int *ex, int splits,
                           double *P, DevStatus *st, cudaStream_t s)
{
    i64 rows = (m + splits - 1) / splits;
    rows = (rows + 127) / 128 * 128;
    const size_t smem = (size_t)kStages * kStageBytes;
    auto k = oz_gram_kernel<T>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    ProfScope ps_("oz_gram", s);
    k<<<dim3(oz_gram_tiles(n), splits), kThreads, smem, s>>>(X, ldx, m, n, ex, rows, P, st);
    return cudaGetLastError();
}

cudaError_t launch_oz_image(const double *M, i64 ldm, int K, int N, const int *pk, int *em,
                            uint8_t *img, cudaStream_t s)
{
    {
        ProfScope ps_("oz_colexp", s);
        oz_colexp_kernel<<<(unsigned)((N * 32 + 255) / 256), 256, 0, s>>>(M, ldm, K, N, pk, em);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int KP = (K + 15) / 16 * 16;
    const i64 total = (i64)((N + kNT - 1) / kNT) * ((KP + kBK - 1) / kBK) * kNT * (kBK / 8);
    ProfScope ps_("oz_image", s);
    oz_image_kernel<<<grid_cap(total), 256, 0, s>>>(M, ldm, K, N, pk, em, img);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oz_rowexp(const T *A, i64 lda, i64 m, int K, const int *pk, int *er,
                             cudaStream_t s)
{
    ProfScope ps_("oz_rowexp", s);
    const i64 threads = m * 32;
    oz_rowexp_kernel<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(A, lda, m, K, pk, er);
    return cudaGetLastError();
}

template <typename T, typename TC>
cudaError_t launch_oz_nn(const T *A, i64 lda, i64 m, int K, const int *pk, const int *er,
                         const uint8_t *img, const int *em, int N, TC *C, i64 ldc, DevStatus *st,
                         cudaStream_t s)
{
    const size_t smem = (size_t)kStages * kStageBytes;
    auto k = oz_nn_kernel<T, TC>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const i64 ntiles = (m + 127) / 128 * ((N + kNT - 1) / kNT);
    const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
    ProfScope ps_("oz_nn", s);
    k<<<grid, kThreads, smem, s>>>(A, lda, m, K, pk, er, img, em, N, C, ldc, st);
    return cudaGetLastError();
}

cudaError_t launch_oz_exp_from_bits(const unsigned long long *bits, int n, int *ex, cudaStream_t s)
{
    ProfScope ps_("oz_exp", s);
    oz_exp_from_bits_kernel<<<(n + 255) / 256, 256, 0, s>>>(bits, n, ex);
    return cudaGetLastError();
}

cudaError_t launch_oz_pow2_of(const double *sc, int n, int *pk, cudaStream_t s)
{
    ProfScope ps_("oz_pow2", s);
    oz_pow2_of_kernel<<<(n + 255) / 256, 256, 0, s>>>(sc, n, pk);
    return cudaGetLastError();
}

cudaError_t launch_neg_int(const int *in, int n, int *out, cudaStream_t s)
{
    ProfScope ps_("neg_int", s);
    neg_int_kernel<<<(n + 255) / 256, 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

template cudaError_t launch_oz_gram<double>(const double *, i64, i64, int, const int *, int,
                                            double *, DevStatus *, cudaStream_t);
template cudaError_t launch_oz_gram<float>(const float *, i64, i64, int, const int *, int,
                                           double *, DevStatus *, cudaStream_t);
template cudaError_t launch_oz_rowexp<double>(const double *, i64, i64, int, const int *, int *,
                                              cudaStream_t);
template cudaError_t launch_oz_rowexp<float>(const float *, i64, i64, int, const int *, int *,
                                             cudaStream_t);
template cudaError_t launch_oz_nn<double, double>(const double *, i64, i64, int, const int *,
                                                  const int *, const uint8_t *, const int *, int,
                                                  double *, i64, DevStatus *, cudaStream_t);
template cudaError_t launch_oz_nn<float, double>(const float *, i64, i64, int, const int *,
                                                 const int *, const uint8_t *, const int *, int,
                                                 double *, i64, DevStatus *, cudaStream_t);
template cudaError_t launch_oz_nn<double, float>(const double *, i64, i64, int, const int *,
                                                 const int *, const uint8_t *, const int *, int,
                                                 float *, i64, DevStatus *, cudaStream_t);

}  // namespace tssvd
