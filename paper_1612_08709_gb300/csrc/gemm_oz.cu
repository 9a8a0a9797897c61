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
//    scale 2^e bounding its entries.  Relative to it a value is rounded to
//    49 fractional bits and written as seven balanced base-128 digits:
//    v 2^-e = sum_s d_s 2^(-7(s+1)) + r, |d_0| <= 129, |d_s| <= 64,
//    |r| <= 2^-50.  The digits are small integers, exact in bfloat16, and
//    are extracted with integer operations on the bit pattern (no FP64
//    arithmetic).  Balanced digits and rounding keep the neglected parts
//    free of sign bias, so their errors do not add up along a long sum.
//  * A product sum_k a_k b_k becomes sum over digit pairs (s, t) with
//    s + t <= 6 (28 pairs; the dropped ones weigh about 2^-49) of
//    2^(ea+eb-14-7(s+t)) sum_k da_s db_t.  Pairs with the same level
//    L = s + t share one FP32 accumulator in tensor memory (7 levels x 64
//    columns).  A row adds at most 129^2 = 16641 to level 0 and
//    2*129*64 + (L-1)*64^2 <= 36992 to level L >= 1, so over a chunk of 448
//    rows every level sum stays below 2^24 and is exact.
//  * After each chunk the epilogue warps combine the seven level sums with
//    error-free FP32 transformations (TwoSum) into a double-FP32 value and
//    add it to an FP64 running sum per output: two FP64 additions per
//    output and chunk (the FP32 -> FP64 widening and the power-of-two
//    scales are integer operations on the bit patterns, since FP64 issue
//    is scarce on this part).  A product with a single chunk (k <= 448)
//    keeps the double-FP32 values in registers and releases tensor memory
//    to the next tile before it widens, scales and stores them.
// Each operand is first cut into a digit image in global memory (once per
// product), laid out exactly as the shared-memory tiles, so the product
// kernels only stage tiles with bulk copies (TMA) and issue MMAs.  Stages
// and bounded mbarrier waits as in gemm_tc.cu.
#include "tc_ptx.cuh"

namespace tssvd {

namespace {

using namespace tc;

constexpr int kDig = 7;           // digits per value
constexpr int kLevels = 7;        // levels s + t = 0..6
constexpr int kNT = 64;           // output columns per CTA tile (N of the MMA)
constexpr int kBK = 32;           // rows (Gram) or k (A*M) per stage
constexpr int kChunkStages = 14;  // 448 rows/k per FP32 chunk (every level exact)
constexpr uint32_t kATerm = 128 * kBK * 2;  // 8 KB: one digit of the 128-row operand
constexpr uint32_t kBTerm = kNT * kBK * 2;  // 4 KB: one digit of the 64-row operand
// The products stream 16-deep halves of the 32-deep blocks: a stage holds
// the seven 4 KB A digits and the 14 KB stacked B digits of one half.
constexpr uint32_t kStageBytes = kDig * (kATerm / 2) + kDig * (kBTerm / 2);  // 42 KB
constexpr int kChunkUnits = 2 * kChunkStages;  // halves per FP32 chunk
// The A*M product runs three stages and stages its 128 x 64 output tile in
// shared memory (rows padded to 65 eight-byte slots): the drain parks each
// output's double-FP32 value there (or adds it to an FP64 sum when k spans
// several chunks), releases tensor memory, and the results then leave as
// whole 256-byte row segments.  Rolled loops keep the epilogue small (an
// unrolled one overflows the instruction cache).
constexpr int kStagesNN = 3;
constexpr int kStgLd = kNT + 1;
constexpr size_t kNNSmem = (size_t)kStagesNN * kStageBytes + 128 * kStgLd * sizeof(double);
// Optional fused column statistics of the A*M output (N <= kFuseMaxN):
// per-warp FP64 sums of squares (deterministic order) and column maxima of
// |C| as bit patterns, in shared memory after the staging tile.
constexpr int kFuseMaxN = 512;
constexpr size_t kNNSmemTotal = kNNSmem + (size_t)kFuseMaxN * (4 * sizeof(double) + 8);
// The Gram-type product (oz_tn) uses the same three stages and staging tile
// (its drain parks each chunk's double-FP32 values there).
constexpr int kStagesTN = 3;
constexpr size_t kTNSmem = (size_t)kStagesTN * kStageBytes + 128 * kStgLd * sizeof(double);

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

// The same for a float: 24-bit significand.
__device__ __forceinline__ void fsplit(float v, int &ev, unsigned long long &mant, uint32_t &sign)
{
    const uint32_t b = __float_as_uint(v);
    sign = b >> 31;
    const int ef = (int)((b >> 23) & 0xFF);
    if (ef == 0 || ef == 0xFF) {
        ev = -100000;
        mant = 0;
        return;
    }
    ev = ef - 127;
    mant = (unsigned long long)((b & 0x7FFFFFu) | (1u << 23));
}

// Seven balanced base-128 digits of a value |v| = mant 2^(q) (q = its
// exponent minus the significand bits), prescaled by 2^p, relative to 2^e:
// F = round(|v| 2^(p - e) 2^49) is written as sum_s d_s 2^(7(6-s)) with the
// six low digits in [-64, 63] (the leading digit takes the carry, <= 129),
// so the dropped digit pairs and the rounding of F carry no sign bias.
// The recoding is one addition: with B = 64 (1 + 2^7 + ... + 2^35),
// F + B = sum (d_s + 64) 2^(7(6-s)) + d_0 2^42, so each low digit is a
// 7-bit field of F + B minus 64.  Each digit then becomes a bfloat16 bit
// pattern: d + 1.5 * 2^23 is formed exactly in the FP32 bit pattern, the
// bias is subtracted in FP32 (exact), and an integer of at most 8
// significant bits keeps all of them in bfloat16's upper half; the value's
// sign is the bfloat16 sign bit (a zero digit of a negative value becomes
// -0, which multiplies like 0).
__device__ __forceinline__ void digits_from(unsigned long long mant, int q, uint32_t vsign, int e,
                                           int p, uint32_t (&out)[kDig])
{
    unsigned long long F = 0;
    if (mant != 0) {
        const int sh = q + p - e + 49;  // F = mant * 2^sh
        if (sh >= 0)
            F = sh < __clzll((long long)mant) ? (mant << sh) : 0;  // overflow only for a wrong scale
        else if (sh > -64)
            F = (mant + (1ull << (-sh - 1))) >> (-sh);
    }
    const unsigned long long G = F + 0x20408102040ull;
    const uint32_t sgn = vsign << 15;
#pragma unroll
    for (int s = 1; s < kDig; s++) {
        const int d = (int)((G >> (7 * (kDig - 1 - s))) & 127u) - 64;
        out[s] = (__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16) ^ sgn;
    }
    const int d0 = (int)((G >> 42) & 0xFFu);
    out[0] = (__float_as_uint(__int_as_float(0x4B400000 + d0) - 12582912.0f) >> 16) ^ sgn;
}

__device__ __forceinline__ void digits7(double v, int e, int p, uint32_t (&out)[kDig])
{
    int ev;
    unsigned long long mant;
    uint32_t sign;
    dsplit(v, ev, mant, sign);
    digits_from(mant, ev - 52, sign, e, p, out);
}

__device__ __forceinline__ void digits7(float v, int e, int p, uint32_t (&out)[kDig])
{
    int ev;
    unsigned long long mant;
    uint32_t sign;
    fsplit(v, ev, mant, sign);
    digits_from(mant, ev - 23, sign, e, p, out);
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

// Exact FP32 -> FP64 widening by integer operations (for zero and normal
// floats; the level sums and their TwoSum errors are multiples of 2^-42
// far inside FP32's normal range, so no subnormal reaches this).  Written
// without branches so that independent widenings interleave.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t b = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned long long ex = (unsigned long long)(((b >> 23) & 0xFF) + (1023 - 127));
    const unsigned long long w =
        sign | (ex << 52) | ((unsigned long long)(b & 0x7FFFFF) << 29);
    return (b & 0x7FFFFFFFu) ? __longlong_as_double((long long)w) : 0.0;
}

// x 2^k by an integer add to the exponent field, without branches; `bad`
// is set when the result would leave the normal range (then the caller
// redoes the value with scale2k_safe).
__device__ __forceinline__ double scale2k_fast(double x, int k, bool &bad)
{
    const long long b = __double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7FF);
    bad |= ef != 0 && ((unsigned)(ef + k - 1) >= 2046u || ef == 0x7FF);
    return ef == 0 ? x : __longlong_as_double(b + ((long long)k << 52));
}

__device__ __noinline__ double scale2k_safe(double x, int k) { return ldexp(x, k); }

// x 2^k for results written once per tile (the Gram partials).
__device__ __forceinline__ double scale2k(double x, int k)
{
    bool bad = false;
    const double r = scale2k_fast(x, k, bad);
    return bad ? scale2k_safe(x, k) : r;
}

// 8 consecutive FP32 TMEM columns of this thread's lane (no wait).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// The drain of one 8-column group g: load_group issues the loads of the
// seven level sums of columns 8g .. 8g+7 of this thread's TMEM lane (no
// wait); park_group combines them with TwoSum into double-FP32 values and
// parks them in the staging row (or adds them to its FP64 sums).
__device__ __forceinline__ void load_group(uint32_t tmem_row, int g, uint32_t (&lv)[kLevels][8])
{
#pragma unroll
    for (int L = 0; L < kLevels; L++) tmem_ld8_nowait(tmem_row + (uint32_t)(L * kNT + g * 8), lv[L]);
}

__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Wait for the outstanding TMEM loads, then pass the registers of lv
// through empty asm statements: their values now depend on code after the
// wait, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&lv)[kLevels][8])
{
    tmem_wait_ld();
#pragma unroll
    for (int L = 0; L < kLevels; L++)
#pragma unroll
        for (int c = 0; c < 8; c++) asm volatile("" : "+r"(lv[L][c]));
}

__device__ __forceinline__ void park_group(const uint32_t (&lv)[kLevels][8], int g, bool single,
                                           double *stg, float2 *stg2, int lane)
{
#pragma unroll
    for (int c = 0; c < 8; c++) {
        float s = __uint_as_float(lv[kLevels - 1][c]) *
                  __uint_as_float((uint32_t)(127 - 7 * (kLevels - 1)) << 23);
        float e = 0.f;
#pragma unroll
        for (int L = kLevels - 2; L >= 0; L--) {
            float t, er;
            const float w = __uint_as_float((uint32_t)(127 - 7 * L) << 23);
            two_sum(__uint_as_float(lv[L][c]) * w, s, t, er);
            s = t;
            e += er;
        }
        const int col = g * 8 + c;
        if (single)
            stg2[lane * kStgLd + col] = make_float2(s, e);
        else
            stg[lane * kStgLd + col] += widen(s) + widen(e);
    }
}

// B operand of a 16-deep half: the digit blocks t = 0..6 (64 rows each)
// stacked into one 448-row K-major operand at t * (kBTerm / 2), so 8-row
// groups are 256 bytes apart across digit boundaries.  kBHalf is its size
// (and the stride between halves in the B digit image of oz_image).
constexpr uint32_t kBHalf = kDig * (kBTerm / 2);

// MMAs of one stage (a 16-deep half).  For A digit s one MMA (two when
// wider than 256) multiplies A_s by the stacked B digits t = 0..6-s into
// tensor-memory columns (s + t) * 64: level L = s + t receives every
// A_s B_t with s + t = L, 10 MMAs of N <= 256 instead of 28 of N = 64
// (the same products, 43% fewer operand bytes read from shared memory).
// At the first half of a chunk the s = 0 MMAs, which cover all seven
// levels, overwrite the accumulators; every later MMA accumulates.
__device__ __forceinline__ void issue_stage(uint32_t abase, uint32_t bbase, uint32_t tmem,
                                            uint32_t &started)
{
#pragma unroll
    for (int s = 0; s < kDig; s++) {
        const uint64_t ad = sdesc(abase + s * (kATerm / 2), 128, 256);
        const int width = (kDig - s) * kNT;
#pragma unroll
        for (int n0 = 0; n0 < width; n0 += 256) {
            const int w = width - n0 < 256 ? width - n0 : 256;
            const uint64_t bd = sdesc(bbase + (uint32_t)(n0 / 8) * 256, 128, 256);
            const uint32_t acc = (started != 0u || s > 0) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(s * kNT + n0), ad, bd, idesc_bf16(128, w), acc);
        }
    }
    started = 1u;
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

// Threads of the digit-product kernels: warps 0-3 drain TMEM (lane
// quarters 0-3), warp 4 stages operands with bulk copies, warp 5 issues
// the MMAs.  Six warps keep at most two per SM sub-partition, so the
// epilogue's 64 FP64 running sums fit in registers.
constexpr int kOzThreads = 192;

// Padded column count of a Gram digit image (whole 128-column tiles).
__host__ __device__ __forceinline__ int gram_npad(int n) { return (n + 127) / 128 * 128; }

// Gram digit image of X (m x n): per 32-row block kb and digit s, two
// 16-row halves of npad/8 groups of 8 columns (256 bytes each, K-major
// no-swizzle core layout).  Block (kb, s, h) starts at
// ((kb * 7 + s) * 2 + h) * npad * 32 bytes.
template <typename T>
__global__ void oz_gram_image_kernel(const T *__restrict__ X, i64 ldx, i64 m, int n,
                                     const int *__restrict__ ex, uint8_t *__restrict__ img)
{
    const int npad = gram_npad(n);
    const i64 nkb = (m + kBK - 1) / kBK;
    const i64 ngrp = nkb * (kBK / 8);  // 8-row groups
    // (c, group) walk: one 32-bit division per step while the group index
    // fits, the carry form of it afterwards
    const i64 stride = (i64)gridDim.x * blockDim.x;
    const i64 e0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    i64 g = e0 / npad;
    int c = (int)(e0 - g * npad);
    const i64 gstep = stride / npad;
    const int cstep = (int)(stride - gstep * npad);
    static_assert(kBK / 8 == 4, "four 8-row groups per block");
    // the next step's eight values are loaded before this step's digits are
    // formed, so every thread keeps a group of loads in flight
    auto load8 = [&](i64 gg, int cc, T (&v)[8]) {
        const i64 k0 = (gg >> 2) * kBK + 8 * (int)(gg & 3);
#pragma unroll
        for (int r = 0; r < 8; r++)
            v[r] = (cc < n && k0 + r < m) ? X[(k0 + r) * ldx + cc] : (T)0;
    };
    T cur[8];
    if (g < ngrp) load8(g, c, cur);
    const uint32_t half = (uint32_t)npad * 32;
    while (g < ngrp) {
        i64 gn = g + gstep;
        int cn = c + cstep;
        if (cn >= npad) {
            cn -= npad;
            gn++;
        }
        T nxt[8];
        if (gn < ngrp) load8(gn, cn, nxt);
        const int q = (int)(g & 3);
        const i64 kb = g >> 2;
        uint8_t *base = img + (size_t)kb * kDig * 2 * half + (size_t)(q >> 1) * half;
        const uint32_t off = (uint32_t)(c >> 3) * 256 + (uint32_t)(q & 1) * 128 + (uint32_t)(c & 7) * 16;
        if (c < n) {
            const int ec = ex[c];
            uint32_t d[8][kDig];
#pragma unroll
            for (int r = 0; r < 8; r++) digits7(cur[r], ec, 0, d[r]);
            store_digits8(base, 2 * half, off, d);
        } else {
            // padding columns: all digits zero
#pragma unroll
            for (int sd = 0; sd < kDig; sd++)
                *reinterpret_cast<uint4 *>(base + (size_t)sd * 2 * half + off) = make_uint4(0, 0, 0, 0);
        }
        g = gn;
        c = cn;
#pragma unroll
        for (int r = 0; r < 8; r++) cur[r] = nxt[r];
    }
}

// Row-operand digit image of A diag(2^pk) (m x K): per 128-row tile and
// 32-deep k block, 7 digits x 2 halves x 16 groups (56 KB contiguous).
template <typename T>
__global__ void oz_row_image_kernel(const T *__restrict__ A, i64 lda, i64 m, int K,
                                    const int *__restrict__ pk, const int *__restrict__ er,
                                    uint8_t *__restrict__ img)
{
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    const i64 mpad = (m + 127) / 128 * 128;
    // e = (kb * mpad + row) * 4 + q; the stride is a multiple of 4, so q
    // is fixed per thread and (kb, row) advance by carries, not divisions
    static_assert(kBK / 8 == 4, "four 8-deep groups per k block");
    const i64 stride4 = (i64)gridDim.x * blockDim.x / 4;
    const i64 e0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = (int)(e0 & 3);
    const i64 g0 = e0 >> 2;
    int kb = (int)(g0 / mpad);
    i64 row = g0 - (i64)kb * mpad;
    const int kstep = (int)(stride4 / mpad);
    const i64 rstep = stride4 - (i64)kstep * mpad;
    // the next step's eight values are loaded before this step's digits
    auto load8 = [&](int kk, i64 rr, T (&v)[8]) {
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = kk * kBK + 8 * q + u;
            v[u] = (rr < m && k < K) ? A[rr * lda + k] : (T)0;
        }
    };
    T cur[8];
    if (kb < nkb) load8(kb, row, cur);
    while (kb < nkb) {
        i64 rn = row + rstep;
        int kn = kb + kstep;
        if (rn >= mpad) {
            rn -= mpad;
            kn++;
        }
        T nxt[8];
        if (kn < nkb) load8(kn, rn, nxt);
        const int ei = row < m ? er[row] : 0;
        uint32_t d[8][kDig];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = kb * kBK + 8 * q + u;
            digits7(cur[u], ei, (pk && k < K) ? pk[k] : 0, d[u]);
        }
        const i64 rt = row >> 7;
        const int r = (int)(row & 127);
        uint8_t *base = img + ((size_t)rt * nkb + kb) * kDig * kATerm + (size_t)(q >> 1) * (kATerm / 2);
        const uint32_t off = (uint32_t)(r >> 3) * 256 + (uint32_t)(q & 1) * 128 + (uint32_t)(r & 7) * 16;
        store_digits8(base, kATerm, off, d);
        row = rn;
        kb = kn;
#pragma unroll
        for (int u = 0; u < 8; u++) cur[u] = nxt[u];
    }
}

// ------------------------------------------------------------ A^T B / Gram
// P[split][i][j] (M x N, FP64) for the (i, j) of the CTA's tile: sum over
// the split's rows k of X[k][i] Y[k][j], from the column digit images of X
// (m x M, exponents exa) and Y (m x N, exponents exb).  With upper (X = Y,
// the Gram matrix) only tiles holding some i <= j are computed.
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_tn_kernel(const uint8_t *__restrict__ aimg, const int *__restrict__ exa, int M,
                 const uint8_t *__restrict__ bimg, const int *__restrict__ exb, int N, int upper,
                 i64 m, i64 rows_per_split, double *__restrict__ P, DevStatus *st)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStagesTN], empty_bar[kStagesTN];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = &st->err;
    int ti = 0, tj = 0;
    if (upper) {
        gram_tile(blockIdx.x, M, ti, tj);
    } else {
        const int TJ = (N + kNT - 1) / kNT;
        ti = blockIdx.x / TJ;
        tj = blockIdx.x % TJ;
    }
    const int i0 = ti * 128, j0 = tj * kNT;
    const uint32_t half_a = (uint32_t)gram_npad(M) * 32, half_b = (uint32_t)gram_npad(N) * 32;
    const i64 kb0 = (i64)blockIdx.y * (rows_per_split / kBK);
    const i64 kbm = (m + kBK - 1) / kBK;
    i64 kb1 = kb0 + rows_per_split / kBK;
    if (kb1 > kbm) kb1 = kbm;
    const int nkb = kb1 > kb0 ? (int)(kb1 - kb0) : 0;
    const int nunits = 2 * nkb;
    const int nchunks = (nunits + kChunkUnits - 1) / kChunkUnits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesTN; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 128);
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) tmem_alloc(&tmem_base_s, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 4) {
        // ---------------- bulk-copy producer
        if (lane == 0) {
            int last = -1;
            for (int u = 0; u < nunits; u++) {
                const int s = u % kStagesTN;
                if (!mbar_wait(&empty_bar[s], ((u / kStagesTN) & 1) ^ 1, err)) break;
                uint8_t *stage = smem_raw + (size_t)s * kStageBytes;
                mbar_arrive_expect_tx(&full_bar[s], kStageBytes);
                const int h = u & 1;
                const uint8_t *ablk = aimg + (size_t)(kb0 + (u >> 1)) * kDig * 2 * half_a;
                const uint8_t *bblk = bimg + (size_t)(kb0 + (u >> 1)) * kDig * 2 * half_b;
#pragma unroll 1
                for (int d = 0; d < kDig; d++) {
                    bulk_g2s(stage + d * (kATerm / 2),
                             ablk + (size_t)(d * 2 + h) * half_a + (size_t)(i0 / 8) * 256,
                             kATerm / 2, &full_bar[s]);
                    bulk_g2s(stage + kDig * (kATerm / 2) + d * (kBTerm / 2),
                             bblk + (size_t)(d * 2 + h) * half_b + (size_t)(j0 / 8) * 256,
                             kBTerm / 2, &full_bar[s]);
                }
                last = u;
            }
            if (last >= 0) mbar_wait_drain(&full_bar[last % kStagesTN], (last / kStagesTN) & 1);
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- epilogue: per chunk, drain the level sums into
        // this thread's staging row as double-FP32 values, release tensor
        // memory, then add the row into the FP64 running sums (overlapping
        // the next chunk's MMAs)
        double acc[kNT];
#pragma unroll
        for (int j = 0; j < kNT; j++) acc[j] = 0.0;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        double *stg = reinterpret_cast<double *>(smem_raw + (size_t)kStagesTN * kStageBytes) +
                      warp * 32 * kStgLd;
        float2 *stg2 = reinterpret_cast<float2 *>(stg);
        bool ok = true;
        for (int ch = 0; ch < nchunks; ch++) {
            if (!mbar_wait(&acc_full, ch & 1, err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            uint32_t la[kLevels][8], lb[kLevels][8];
            load_group(trow, 0, la);
            tmem_wait_ld(la);
#pragma unroll 1
            for (int g = 0; g < kNT / 8; g += 2) {
                load_group(trow, g + 1, lb);
                park_group(la, g, true, stg, stg2, lane);
                tmem_wait_ld(lb);
                if (g + 2 < kNT / 8) load_group(trow, g + 2, la);
                park_group(lb, g + 1, true, stg, stg2, lane);
                tmem_wait_ld(la);
            }
            tc_fence_before();
            mbar_arrive(&acc_empty);
#pragma unroll
            for (int c = 0; c < kNT; c++) {
                const float2 f = stg2[lane * kStgLd + c];
                acc[c] += widen(f.x);
                acc[c] += widen(f.y);
            }
        }
        if (ok) {
            const int il = warp * 32 + lane;
            const int i = i0 + il;
            if (i < M) {
                double *Prow = P + (i64)blockIdx.y * M * N + (i64)i * N;
                const int ei = exa[i];
#pragma unroll
                for (int jj = 0; jj < kNT; jj++) {
                    const int j = j0 + jj;
                    if (j < N) Prow[j] = scale2k(acc[jj], ei + exb[j] - 14);
                }
            }
        }
    } else {
        // ---------------- MMA issuer
        if (lane == 0) {
            int u = 0;
            bool ok = true;
            for (int ch = 0; ch < nchunks && ok; ch++) {
                if (ch > 0) {
                    if (!mbar_wait(&acc_empty, (ch - 1) & 1, err)) break;
                    tc_fence_after();
                }
                uint32_t started = 0;
                const int u_end = (ch + 1) * kChunkUnits < nunits ? (ch + 1) * kChunkUnits : nunits;
                for (; u < u_end; u++) {
                    const int s = u % kStagesTN;
                    if (!mbar_wait(&full_bar[s], (u / kStagesTN) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = saddr(smem_raw + (size_t)s * kStageBytes);
                    issue_stage(base, base + kDig * (kATerm / 2), tmem, started);
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
    if (warp == 5) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------- A * M
// C[r][j] = sum_k A[r][k] M[k][j] from the row image of A diag(2^pk) and
// the image of diag(2^-pk) M; tiles of 128 rows x 64 columns, persistent,
// column tile fastest.
template <typename TC>
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_nn_kernel(const uint8_t *__restrict__ aimg, i64 m, int K, const int *__restrict__ er,
                 const uint8_t *__restrict__ bimg, const int *__restrict__ em, int N,
                 TC *__restrict__ C, i64 ldc, DevStatus *st, unsigned long long *colmax_out,
                 double *colsq_out)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStagesNN], empty_bar[kStagesNN];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = &st->err;
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    const int nunits = KP / 16;  // 16-deep halves holding some k < K
    const int nchunks = (nunits + kChunkUnits - 1) / kChunkUnits;
    const int TN = (N + kNT - 1) / kNT;
    const i64 ntiles = (m + 127) / 128 * TN;
    const int my_tiles =
        (i64)blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const size_t btile = (size_t)nkb * kDig * kBTerm;
    double *csq = reinterpret_cast<double *>(smem_raw + kNNSmem);  // [4][kFuseMaxN]
    unsigned long long *cmx = reinterpret_cast<unsigned long long *>(csq + 4 * kFuseMaxN);
    const bool fuse = (colmax_out || colsq_out) && N <= kFuseMaxN;
    if (fuse)
        for (int i = threadIdx.x; i < 5 * kFuseMaxN; i += blockDim.x) {
            if (i < 4 * kFuseMaxN)
                csq[i] = 0.0;
            else
                cmx[i - 4 * kFuseMaxN] = 0ull;
        }

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesNN; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 128);
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) tmem_alloc(&tmem_base_s, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 4) {
        if (lane == 0) {
            int f = 0, last = -1;
            bool ok = true;
            for (int ti = 0; ti < my_tiles && ok; ti++) {
                const i64 t = (i64)blockIdx.x + (i64)ti * gridDim.x;
                const i64 rt = t / TN;
                const int nt = (int)(t % TN);
                for (int u = 0; u < nunits; u++, f++) {
                    const int s = f % kStagesNN;
                    if (!mbar_wait(&empty_bar[s], ((f / kStagesNN) & 1) ^ 1, err)) {
                        ok = false;
                        break;
                    }
                    uint8_t *stage = smem_raw + (size_t)s * kStageBytes;
                    mbar_arrive_expect_tx(&full_bar[s], kStageBytes);
                    const int kb = u >> 1, h = u & 1;
                    const uint8_t *ablk = aimg + ((size_t)rt * nkb + kb) * kDig * kATerm;
#pragma unroll 1
                    for (int d = 0; d < kDig; d++)
                        bulk_g2s(stage + d * (kATerm / 2), ablk + d * kATerm + h * (kATerm / 2),
                                 kATerm / 2, &full_bar[s]);
                    bulk_g2s(stage + kDig * (kATerm / 2),
                             bimg + (size_t)nt * btile + (size_t)kb * kDig * kBTerm + h * kBHalf,
                             kBHalf, &full_bar[s]);
                    last = f;
                }
            }
            if (last >= 0) mbar_wait_drain(&full_bar[last % kStagesNN], (last / kStagesNN) & 1);
        }
        __syncwarp();
    } else if (warp < 4) {
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        // this warp's 32 staging rows (row `lane` is this thread's TMEM lane)
        double *stg = reinterpret_cast<double *>(smem_raw + (size_t)kStagesNN * kStageBytes) +
                      warp * 32 * kStgLd;
        float2 *stg2 = reinterpret_cast<float2 *>(stg);
        int ch_global = 0;
        bool ok = true;
        for (int ti = 0; ti < my_tiles && ok; ti++) {
            const i64 t = (i64)blockIdx.x + (i64)ti * gridDim.x;
            const i64 row0 = (t / TN) * 128 + warp * 32;
            const int nt = (int)(t % TN);
            const bool single = nchunks == 1;
            if (!single)
                for (int c = 0; c < kNT; c++) stg[lane * kStgLd + c] = 0.0;
            for (int ch = 0; ch < nchunks; ch++, ch_global++) {
                if (!mbar_wait(&acc_full, ch_global & 1, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // the loads of group g + 1 are in flight while group g is
                // combined (two register sets, alternating)
                uint32_t la[kLevels][8], lb[kLevels][8];
                load_group(trow, 0, la);
                tmem_wait_ld(la);
#pragma unroll 1
                for (int g = 0; g < kNT / 8; g += 2) {
                    load_group(trow, g + 1, lb);
                    park_group(la, g, single, stg, stg2, lane);
                    tmem_wait_ld(lb);
                    if (g + 2 < kNT / 8) load_group(trow, g + 2, la);
                    park_group(lb, g + 1, single, stg, stg2, lane);
                    tmem_wait_ld(la);
                }
                tc_fence_before();
                mbar_arrive(&acc_empty);
            }
            if (!ok) break;
            // tensor memory is free: widen, scale and store row segments.
            // Lane l owns column j = c0 + l; row exponents are loaded once
            // (lane r holds row r's) and broadcast; eight rows are formed in
            // registers before their stores, so the chains overlap.
            __syncwarp();
            const int erl = row0 + lane < m ? er[row0 + lane] : 0;
            bool bad = false;
#pragma unroll 1
            for (int c0 = 0; c0 < kNT; c0 += 32) {
                const int j = nt * kNT + c0 + lane;
                const int ej = j < N ? em[j] - 14 : 0;
                double sq = 0.0;
                unsigned long long mx = 0ull;
#pragma unroll 1
                for (int r0 = 0; r0 < 32; r0 += 8) {
                    double v[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int r = r0 + q;
                        double x;
                        if (single) {
                            const float2 f = stg2[r * kStgLd + c0 + lane];
                            x = widen(f.x) + widen(f.y);
                        } else {
                            x = stg[r * kStgLd + c0 + lane];
                        }
                        v[q] = scale2k_fast(x, __shfl_sync(0xffffffffu, erl, r) + ej, bad);
                    }
                    if (j < N) {
#pragma unroll
                        for (int q = 0; q < 8; q++)
                            if (row0 + r0 + q < m) {
                                C[(row0 + r0 + q) * ldc + j] = (TC)v[q];
                                if (fuse) {
                                    sq = fma(v[q], v[q], sq);
                                    const unsigned long long ab =
                                        (unsigned long long)__double_as_longlong(v[q]) &
                                        0x7FFFFFFFFFFFFFFFull;
                                    mx = ab > mx ? ab : mx;
                                }
                            }
                    }
                }
                if (fuse && j < N) {
                    csq[warp * kFuseMaxN + j] += sq;
                    if (mx) atomicMax(cmx + j, mx);
                }
            }
            if (__any_sync(0xffffffffu, bad)) {
                // some result left the normal range: redo the tile's stores
                // with the library scaling (never for data of sane range)
                for (int c0 = 0; c0 < kNT; c0 += 32) {
                    const int j = nt * kNT + c0 + lane;
                    const int ej = j < N ? em[j] - 14 : 0;
                    for (int r = 0; r < 32; r++) {
                        double x;
                        if (single) {
                            const float2 f = stg2[r * kStgLd + c0 + lane];
                            x = widen(f.x) + widen(f.y);
                        } else {
                            x = stg[r * kStgLd + c0 + lane];
                        }
                        const int k = __shfl_sync(0xffffffffu, erl, r) + ej;
                        if (j < N && row0 + r < m) C[(row0 + r) * ldc + j] = (TC)scale2k_safe(x, k);
                    }
                }
            }
            __syncwarp();
        }
        if (fuse) {
            // the CTA's column statistics (epilogue warps only)
            asm volatile("bar.sync 1, 128;" ::: "memory");
            for (int jj = threadIdx.x; jj < N; jj += 128) {
                if (colsq_out)
                    colsq_out[(i64)blockIdx.x * N + jj] =
                        ((csq[jj] + csq[kFuseMaxN + jj]) + csq[2 * kFuseMaxN + jj]) +
                        csq[3 * kFuseMaxN + jj];
                if (colmax_out && cmx[jj]) atomicMax(colmax_out + jj, cmx[jj]);
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
                    const int u_end = (ch + 1) * kChunkUnits < nunits ? (ch + 1) * kChunkUnits : nunits;
                    for (int u = ch * kChunkUnits; u < u_end; u++, f++) {
                        const int s = f % kStagesNN;
                        if (!mbar_wait(&full_bar[s], (f / kStagesNN) & 1, err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = saddr(smem_raw + (size_t)s * kStageBytes);
                        issue_stage(base, base + kDig * (kATerm / 2), tmem, started);
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
    if (warp == 5) tmem_dealloc(tmem, kTmemCols);
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
// for each 16-deep half the 7 digit blocks of 64 rows (j) x 16 k stacked
// in the K-major no-swizzle layout (the stage's B operand, see kBHalf).
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
        const uint32_t off = (uint32_t)(q >> 1) * kBHalf + (uint32_t)(jj >> 3) * 256 +
                             (uint32_t)(q & 1) * 128 + (uint32_t)(jj & 7) * 16;
        store_digits8(blk, kBTerm / 2, off, d);
    }
}

// Row exponents of A diag(2^pk): er[r] = smallest e bounding the row.
template <typename T>
__global__ void oz_rowexp_kernel(const T *__restrict__ A, i64 lda, i64 m, int K,
                                 const int *__restrict__ pk, int *__restrict__ er)
{
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 r = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += warps) {
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

// Row splits for a grid of `tiles` output tiles at one CTA per SM: the
// count whose last wave is fullest (waves / splits smallest), smaller counts
// winning within 3%, each split keeping at least 1024 rows.
static int balanced_splits(i64 m, int tiles)
{
    const int sms = num_sms();
    i64 cap = ((i64)sms + tiles - 1) / tiles;
    if (cap < 16) cap = 16;
    const i64 max_rows = (m + 1023) / 1024;
    if (cap > max_rows) cap = max_rows;
    if (cap < 1) cap = 1;
    int best = 1;
    double best_cost = (double)(((i64)tiles + sms - 1) / sms);
    for (i64 sp = 2; sp <= cap; sp++) {
        const double cost = (double)(((i64)tiles * sp + sms - 1) / sms) / (double)sp;
        if (cost < best_cost * 0.97) {
            best_cost = cost;
            best = (int)sp;
        }
    }
    return best;
}

int oz_gram_splits(i64 m, int n) { return balanced_splits(m, oz_gram_tiles(n)); }

size_t oz_image_bytes(int K, int N)
{
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    const int TN = (N + kNT - 1) / kNT;
    return (size_t)TN * nkb * kDig * kBTerm;
}

size_t oz_gram_image_bytes(i64 m, int n)
{
    return (size_t)((m + kBK - 1) / kBK) * kDig * 2 * (size_t)gram_npad(n) * 32;
}

size_t oz_row_image_bytes(i64 m, int K)
{
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + kBK - 1) / kBK;
    return (size_t)((m + 127) / 128) * nkb * kDig * kATerm;
}

template <typename T>
cudaError_t oz_col_image(const T *X, i64 ldx, i64 m, int n, const int *ex, uint8_t *img, cudaStream_t s)
{
    const i64 total = (m + kBK - 1) / kBK * (kBK / 8) * gram_npad(n);
    ProfScope ps_("oz_gram_image", s);
    oz_gram_image_kernel<T><<<grid_cap(total, 16), 256, 0, s>>>(X, ldx, m, n, ex, img);
    return cudaGetLastError();
}

cudaError_t oz_tn_run(const uint8_t *aimg, const int *exa, int M, const uint8_t *bimg,
                      const int *exb, int N, bool upper, i64 m, int splits, double *P,
                      DevStatus *st, cudaStream_t s)
{
    // whole 32-row blocks per split
    const i64 kbs = ((m + kBK - 1) / kBK + splits - 1) / splits;
    const size_t smem = kTNSmem;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(oz_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const int tiles = upper ? oz_gram_tiles(M) : ((M + 127) / 128) * ((N + kNT - 1) / kNT);
    ProfScope ps_(upper ? "oz_gram" : "oz_tn", s);
    oz_tn_kernel<<<dim3(tiles, splits), kOzThreads, smem, s>>>(aimg, exa, M, bimg, exb, N,
                                                              upper ? 1 : 0, m, kbs * kBK, P, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oz_gram(const T *X, i64 ldx, i64 m, int n, const int *ex, int splits,
                           uint8_t *gimg, double *P, DevStatus *st, cudaStream_t s)
{
    cudaError_t e = oz_col_image<T>(X, ldx, m, n, ex, gimg, s);
    if (e != cudaSuccess) return e;
    return oz_tn_run(gimg, ex, n, gimg, ex, n, true, m, splits, P, st, s);
}

int oz_tn_splits(i64 m, int M, int N)
{
    return balanced_splits(m, ((M + 127) / 128) * ((N + kNT - 1) / kNT));
}

cudaError_t launch_oz_col_image(const double *X, i64 ldx, i64 m, int n, const int *ex,
                                uint8_t *img, cudaStream_t s)
{
    return oz_col_image<double>(X, ldx, m, n, ex, img, s);
}

cudaError_t launch_oz_tn(const uint8_t *aimg, const int *exa, int M, const uint8_t *bimg,
                         const int *exb, int N, i64 m, int splits, double *P, DevStatus *st,
                         cudaStream_t s)
{
    return oz_tn_run(aimg, exa, M, bimg, exb, N, false, m, splits, P, st, s);
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
                             cudaStream_t s, int per_sm)
{
    ProfScope ps_("oz_rowexp", s);
    oz_rowexp_kernel<T><<<grid_cap(m * 32, per_sm), 256, 0, s>>>(A, lda, m, K, pk, er);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_oz_row_image(const T *A, i64 lda, i64 m, int K, const int *pk, const int *er,
                                uint8_t *aimg, cudaStream_t s, int per_sm)
{
    const int KP = (K + 15) / 16 * 16;
    const i64 total = (m + 127) / 128 * 128 * ((KP + kBK - 1) / kBK) * (kBK / 8);
    ProfScope ps_("oz_row_image", s);
    oz_row_image_kernel<T><<<grid_cap(total, per_sm), 256, 0, s>>>(A, lda, m, K, pk, er, aimg);
    return cudaGetLastError();
}

int oz_nn_grid(i64 m, int N)
{
    const i64 ntiles = (m + 127) / 128 * ((N + kNT - 1) / kNT);
    return (int)(ntiles < num_sms() ? ntiles : num_sms());
}

bool oz_nn_fuses(int N) { return N <= kFuseMaxN; }

template <typename TC>
cudaError_t launch_oz_nn_run(const uint8_t *aimg, i64 m, int K, const int *er, const uint8_t *bimg,
                             const int *em, int N, TC *C, i64 ldc, DevStatus *st, cudaStream_t s,
                             unsigned long long *colmax_out, double *colsq_out)
{
    const size_t smem = kNNSmemTotal;
    auto k = oz_nn_kernel<TC>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const i64 ntiles = (m + 127) / 128 * ((N + kNT - 1) / kNT);
    const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
    ProfScope ps_("oz_nn", s);
    k<<<grid, kOzThreads, smem, s>>>(aimg, m, K, er, bimg, em, N, C, ldc, st, colmax_out,
                                     colsq_out);
    return cudaGetLastError();
}

template <typename T, typename TC>
cudaError_t launch_oz_nn(const T *A, i64 lda, i64 m, int K, const int *pk, const int *er,
                         uint8_t *aimg, const uint8_t *bimg, const int *em, int N, TC *C, i64 ldc,
                         DevStatus *st, cudaStream_t s)
{
    cudaError_t e = launch_oz_row_image<T>(A, lda, m, K, pk, er, aimg, s, 16);
    if (e != cudaSuccess) return e;
    return launch_oz_nn_run<TC>(aimg, m, K, er, bimg, em, N, C, ldc, st, s, nullptr, nullptr);
}

template cudaError_t launch_oz_row_image<double>(const double *, i64, i64, int, const int *,
                                                 const int *, uint8_t *, cudaStream_t, int);
template cudaError_t launch_oz_nn_run<double>(const uint8_t *, i64, int, const int *,
                                              const uint8_t *, const int *, int, double *, i64,
                                              DevStatus *, cudaStream_t, unsigned long long *,
                                              double *);
template cudaError_t launch_oz_nn_run<float>(const uint8_t *, i64, int, const int *,
                                             const uint8_t *, const int *, int, float *, i64,
                                             DevStatus *, cudaStream_t, unsigned long long *,
                                             double *);
template cudaError_t launch_oz_row_image<float>(const float *, i64, i64, int, const int *,
                                                const int *, uint8_t *, cudaStream_t, int);

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
                                            uint8_t *, double *, DevStatus *, cudaStream_t);
template cudaError_t launch_oz_gram<float>(const float *, i64, i64, int, const int *, int,
                                           uint8_t *, double *, DevStatus *, cudaStream_t);
template cudaError_t launch_oz_rowexp<double>(const double *, i64, i64, int, const int *, int *,
                                              cudaStream_t, int);
template cudaError_t launch_oz_rowexp<float>(const float *, i64, i64, int, const int *, int *,
                                             cudaStream_t, int);
template cudaError_t launch_oz_nn<double, double>(const double *, i64, i64, int, const int *,
                                                  const int *, uint8_t *, const uint8_t *,
                                                  const int *, int, double *, i64, DevStatus *,
                                                  cudaStream_t);
template cudaError_t launch_oz_nn<float, double>(const float *, i64, i64, int, const int *,
                                                 const int *, uint8_t *, const uint8_t *,
                                                 const int *, int, double *, i64, DevStatus *,
                                                 cudaStream_t);
template cudaError_t launch_oz_nn<double, float>(const double *, i64, i64, int, const int *,
                                                 const int *, uint8_t *, const uint8_t *,
                                                 const int *, int, float *, i64, DevStatus *,
                                                 cudaStream_t);

}  // namespace tssvd
