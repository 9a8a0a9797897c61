// Tall products on the tcgen05 tensor cores with BF16-split operands.
//
// Mixed-precision form of the first orthonormalisation pass of Algorithm 4
// (the Gram matrix of A and Y~ = A V~): every FP64 (or FP32) input value x
// is split into S bfloat16 terms x ~ x_0 + x_1 + ... + x_{S-1}
// (x_0 = bf16(x), x_1 = bf16(x - x_0), ...), and a product a*b is formed as
// the sum of the S(S+1)/2 term products a_s*b_t with s + t < S.  S = 2
// ("BF16x3", 3 products, about 16 significant bits) or S = 3 ("BF16x6",
// 6 products, about 24 bits).  Each term product is exact in the FP32
// accumulator of the tensor core; sums are accumulated in FP32 in tensor
// memory (TMEM) and drained to FP64.
//
// Kernel structure (one CTA per SM, persistent):
//   warps 0-3  producers: load FP64/FP32 rows of A with plain coalesced
//              loads, split them, and store the bf16 terms into shared
//              memory in the tcgen05 K-major no-swizzle layout;
//   warps 4-7  epilogue: tcgen05.ld the FP32 accumulators, convert to FP64
//              and store (Gram partials / product rows);
//   warp  8    allocates TMEM and one elected lane issues tcgen05.mma.
// Stages are handed over with mbarriers (full: producers -> MMA; empty:
// MMA commit -> producers; acc_full / acc_empty between MMA and epilogue).
// The small right-hand operand of A*M is split once into its shared-memory
// image in global memory and staged with cp.async.bulk (TMA bulk copies).
//
// Shared-memory operand layout (K-major, no swizzle): the operand block for
// one 16-deep MMA step is a sequence of 8-row groups, 256 bytes apart (SBO),
// each holding two 8 x 8 bf16 core matrices (k 0-7, then k 8-15, 128 bytes
// apart: LBO); inside a core matrix row r occupies bytes 16r..16r+15.
//
// Every mbarrier wait is bounded (about two seconds of %globaltimer); on
// expiry the kernel records TSSVD_ETIMEOUT in the status block, every role
// leaves its loop, and the allocating warp still frees TMEM.
#include <cuda_bf16.h>

#include "tc_ptx.cuh"

namespace tssvd {

namespace {

using namespace tc;

// Split 8 values into S packed bf16x8 vectors (one uint4 per term).
template <int S>
__device__ __forceinline__ void split8(const double (&x)[8], uint4 (&out)[S])
{
    double r[8];
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = x[i];
#pragma unroll
    for (int s = 0; s < S; s++) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const __nv_bfloat16 lo = __double2bfloat16(r[2 * i]);
            const __nv_bfloat16 hi = __double2bfloat16(r[2 * i + 1]);
            r[2 * i] -= (double)__bfloat162float(lo);
            r[2 * i + 1] -= (double)__bfloat162float(hi);
            w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        out[s] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <typename T>
__device__ __forceinline__ double ldg_d(const T *p)
{
    return (double)__ldg(p);
}

// ------------------------------------------------------------------ Gram
//
// P[split][i][j] = sum over the split's rows k of A[k][i] A[k][j], all
// i, j < n (n <= 256).  The operand image of a stage is W = 128*MT rows
// (the columns of A, zero beyond n) by 64 k (rows of A), per term.
struct GramSmem {
    static constexpr int BK = 64;
};

template <typename T, int S, int MT, int NSTAGE>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gram_kernel(const T *__restrict__ A, i64 lda, i64 m, int n, int NP, i64 rows_per_split,
                   int chunk_stages, double *__restrict__ P, DevStatus *st)
{
    constexpr int BK = GramSmem::BK;
    constexpr int W = 128 * MT;
    constexpr uint32_t kTermBytes = (uint32_t)W * BK * 2;  // one term of one stage
    constexpr uint32_t kStageBytes = kTermBytes * S;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *tiles = smem_raw;
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = &st->err;
    const i64 r0 = (i64)blockIdx.x * rows_per_split;
    const i64 r1 = r0 + rows_per_split < m ? r0 + rows_per_split : m;
    const int nkb = r1 > r0 ? (int)((r1 - r0 + BK - 1) / BK) : 0;
    const int nchunks = (nkb + chunk_stages - 1) / chunk_stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; s++) {
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
        // ---------------- producers
        const int tid = threadIdx.x;
        for (int kb = 0; kb < nkb; kb++) {
            const int s = kb % NSTAGE;
            if (!mbar_wait(&empty_bar[s], ((kb / NSTAGE) & 1) ^ 1, err)) break;
            uint8_t *stage = tiles + (size_t)s * kStageBytes;
            const i64 k0 = r0 + (i64)kb * BK;
            // items: (column c, 8-row chunk q); W * BK/8 items
            for (int it = tid; it < W * (BK / 8); it += kProducers) {
                const int c = it % W, q = it / W;
                double x[8];
#pragma unroll
                for (int r = 0; r < 8; r++) {
                    const i64 k = k0 + 8 * q + r;
                    x[r] = (c < n && k < r1) ? ldg_d(A + k * lda + c) : 0.0;
                }
                uint4 v[S];
                split8<S>(x, v);
                const uint32_t off = (uint32_t)(q >> 1) * (W * 32) + (uint32_t)(c >> 3) * 256 +
                                     (uint32_t)(q & 1) * 128 + (uint32_t)(c & 7) * 16;
#pragma unroll
                for (int t = 0; t < S; t++)
                    *reinterpret_cast<uint4 *>(stage + (size_t)t * kTermBytes + off) = v[t];
            }
            fence_proxy_async();
            mbar_arrive(&full_bar[s]);
        }
    } else if (warp < 8) {
        // ---------------- epilogue: drain FP32 accumulators to FP64 partials
        const int ew = warp - 4;  // TMEM lanes 32*ew .. 32*ew+31
        double *Ps = P + (i64)blockIdx.x * n * n;
        for (int ch = 0; ch < nchunks; ch++) {
            if (!mbar_wait(&acc_full, ch & 1, err)) break;
            tc_fence_after();
            for (int t = 0; t < MT; t++) {
                const int i = t * 128 + ew * 32 + lane;
                for (int j0 = 0; j0 < NP; j0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(t * 256 + j0), v);
                    if (i < n) {
#pragma unroll
                        for (int u = 0; u < 16; u++) {
                            const int j = j0 + u;
                            if (j < n) {
                                double *p = Ps + (i64)i * n + j;
                                *p = (ch == 0 ? 0.0 : *p) + (double)v[u];
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty);
        }
        if (nchunks == 0) {
            // empty split: its partial is zero
            for (int e = threadIdx.x - kProducers; e < n * n; e += kEpilogue) Ps[e] = 0.0;
        }
    } else {
        // ---------------- MMA issuer (one lane)
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, NP);
            int kb = 0;
            bool ok = true;
            for (int ch = 0; ch < nchunks && ok; ch++) {
                if (ch > 0) {
                    if (!mbar_wait(&acc_empty, (ch - 1) & 1, err)) break;
                    tc_fence_after();
                }
                const int kb_end = (ch + 1) * chunk_stages < nkb ? (ch + 1) * chunk_stages : nkb;
                bool first = true;
                for (; kb < kb_end; kb++) {
                    const int s = kb % NSTAGE;
                    if (!mbar_wait(&full_bar[s], (kb / NSTAGE) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = saddr(tiles + (size_t)s * kStageBytes);
#pragma unroll
                    for (int h = 0; h < BK / 16; h++) {
#pragma unroll
                        for (int a = 0; a < S; a++) {
#pragma unroll
                            for (int b = 0; b < S - a; b++) {
                                const uint32_t ab = base + a * kTermBytes + h * (W * 32);
                                const uint32_t bb = base + b * kTermBytes + h * (W * 32);
                                const uint64_t bd = sdesc(bb, 128, 256);
#pragma unroll
                                for (int t = 0; t < MT; t++) {
                                    const uint64_t ad = sdesc(ab + t * 16 * 256, 128, 256);
                                    mma_bf16(tmem + t * 256, ad, bd, idesc, first ? 0u : 1u);
                                }
                                first = false;
                            }
                        }
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full);
            }
            // every MMA issued above has finished before TMEM is freed
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

// ------------------------------------------------------------ A * M
//
// C[r][j] = sum_k A[r][k] M[k][j] for r < m, j < N (N <= 256), K = n.
// Bimg holds M split into S terms in its shared-memory image, one block of
// S * NP * 64 bytes per 32-deep k step (see tc_split_b_kernel).
template <typename T, int S, int NSTAGE>
__global__ void __launch_bounds__(kThreads, 1)
    tc_nn_kernel(const T *__restrict__ A, i64 lda, i64 m, int K, const uint8_t *__restrict__ Bimg,
                 int N, int NP, double *__restrict__ C, i64 ldc, DevStatus *st)
{
    constexpr int BK = 32;
    constexpr uint32_t kATerm = 128 * BK * 2;  // 8 KB
    const uint32_t kBTerm = (uint32_t)NP * BK * 2;
    const uint32_t kStageBytes = S * (kATerm + kBTerm);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], done_bar;
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = &st->err;
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + BK - 1) / BK;
    const i64 nrt = (m + 127) / 128;
    const int my_tiles = blockIdx.x < nrt ? (int)((nrt - 1 - blockIdx.x) / gridDim.x + 1) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; s++) {
            mbar_init(&full_bar[s], kProducers);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpilogue);
        }
        mbar_init(&done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) tmem_alloc(&tmem_base_s, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp < 4) {
        // ---------------- producers: A rows (split in registers), M via bulk copy
        const int tid = threadIdx.x;
        int f = 0;
        int last_copy = -1;  // fill index of the last bulk copy thread 0 issued
        for (int ti = 0; ti < my_tiles; ti++) {
            const i64 rbase = ((i64)blockIdx.x + (i64)ti * gridDim.x) * 128;
            bool ok = true;
            for (int kb = 0; kb < nkb; kb++, f++) {
                const int s = f % NSTAGE;
                if (!mbar_wait(&empty_bar[s], ((f / NSTAGE) & 1) ^ 1, err)) {
                    ok = false;
                    break;
                }
                uint8_t *stage = smem_raw + (size_t)s * kStageBytes;
                if (tid == 0) {
                    const uint32_t bytes = S * kBTerm;
                    mbar_expect_tx(&full_bar[s], bytes);
                    bulk_g2s(stage + S * kATerm, Bimg + (size_t)kb * bytes, bytes, &full_bar[s]);
                    last_copy = f;
                }
                const int k0 = kb * BK;
                // items: (row r, 8-column chunk q): 128 * 4
                for (int it = tid; it < 128 * (BK / 8); it += kProducers) {
                    const int r = it >> 2, q = it & 3;
                    const i64 row = rbase + r;
                    double x[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int k = k0 + 8 * q + u;
                        x[u] = (row < m && k < K) ? ldg_d(A + row * lda + k) : 0.0;
                    }
                    uint4 v[S];
                    split8<S>(x, v);
                    const uint32_t off = (uint32_t)(q >> 1) * (128 * 32) + (uint32_t)(r >> 3) * 256 +
                                         (uint32_t)(q & 1) * 128 + (uint32_t)(r & 7) * 16;
#pragma unroll
                    for (int t = 0; t < S; t++)
                        *reinterpret_cast<uint4 *>(stage + (size_t)t * kATerm + off) = v[t];
                }
                fence_proxy_async();
                mbar_arrive(&full_bar[s]);
            }
            if (!ok) break;
        }
        // the last bulk copy has landed before this CTA can exit
        if (tid == 0 && last_copy >= 0)
            mbar_wait_drain(&full_bar[last_copy % NSTAGE], (last_copy / NSTAGE) & 1);
    } else if (warp < 8) {
        // ---------------- epilogue
        const int ew = warp - 4;
        for (int ti = 0; ti < my_tiles; ti++) {
            const int b = ti & 1;
            if (!mbar_wait(&acc_full[b], (ti >> 1) & 1, err)) break;
            tc_fence_after();
            const i64 row = ((i64)blockIdx.x + (i64)ti * gridDim.x) * 128 + ew * 32 + lane;
            for (int j0 = 0; j0 < NP; j0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(b * 256 + j0), v);
                if (row < m) {
#pragma unroll
                    for (int u = 0; u < 16; u++)
                        if (j0 + u < N) C[row * ldc + j0 + u] = (double)v[u];
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[b]);
        }
    } else {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, NP);
            int f = 0;
            bool ok = true;
            for (int ti = 0; ti < my_tiles && ok; ti++) {
                const int b = ti & 1;
                if (ti >= 2) {
                    if (!mbar_wait(&acc_empty[b], ((ti >> 1) - 1) & 1, err)) break;
                    tc_fence_after();
                }
                bool first = true;
                for (int kb = 0; kb < nkb; kb++, f++) {
                    const int s = f % NSTAGE;
                    if (!mbar_wait(&full_bar[s], (f / NSTAGE) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t abase = saddr(smem_raw + (size_t)s * kStageBytes);
                    const uint32_t bbase = abase + S * kATerm;
#pragma unroll
                    for (int h = 0; h < BK / 16; h++) {
                        if (kb * BK + h * 16 >= KP) break;
#pragma unroll
                        for (int a = 0; a < S; a++) {
#pragma unroll
                            for (int bt = 0; bt < S - a; bt++) {
                                const uint64_t ad =
                                    sdesc(abase + a * kATerm + h * (128 * 32), 128, 256);
                                const uint64_t bd =
                                    sdesc(bbase + bt * kBTerm + h * (NP * 32), 128, 256);
                                mma_bf16(tmem + b * 256, ad, bd, idesc, first ? 0u : 1u);
                                first = false;
                            }
                        }
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full[b]);
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

// M (K x N, row-major FP64, ldm) -> its split shared-memory image:
// for each 32-deep k step kb and term s, NP rows (j) by 32 k in the
// no-swizzle K-major layout (two 16-deep halves of NP*32 bytes).
template <int S>
__global__ void tc_split_b_kernel(const double *__restrict__ M, i64 ldm, int K, int N, int NP,
                                  uint8_t *__restrict__ img)
{
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + 31) / 32;
    const i64 total = (i64)nkb * 4 * NP;  // items: (kb, q = 8-k chunk of 4, j)
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const int j = (int)(e % NP);
        const int q = (int)((e / NP) % 4);
        const int kb = (int)(e / (4 * NP));
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = kb * 32 + 8 * q + u;
            x[u] = (k < K && j < N) ? M[(i64)k * ldm + j] : 0.0;
        }
        uint4 v[S];
        split8<S>(x, v);
        const size_t blk = (size_t)kb * S * NP * 64;
        const uint32_t off = (uint32_t)(q >> 1) * (NP * 32) + (uint32_t)(j >> 3) * 256 +
                             (uint32_t)(q & 1) * 128 + (uint32_t)(j & 7) * 16;
#pragma unroll
        for (int t = 0; t < S; t++)
            *reinterpret_cast<uint4 *>(img + blk + (size_t)t * NP * 64 + off) = v[t];
    }
}

template <typename T, int S>
cudaError_t gram_launch(const T *A, i64 lda, i64 m, int n, int splits, double *P, DevStatus *st,
                        cudaStream_t s)
{
    constexpr int BK = GramSmem::BK;
    const int NP = (n + 15) / 16 * 16;
    i64 rows = (m + splits - 1) / splits;
    rows = (rows + BK - 1) / BK * BK;
    const int chunk_stages = 16;  // 1024 rows per FP32 accumulation chunk
    cudaError_t e;
    if (n <= 128) {
        constexpr int MT = 1, NS = (S == 2) ? 4 : 3;
        size_t smem = (size_t)NS * S * 128 * MT * BK * 2;
        if (smem < kMinSmem) smem = kMinSmem;
        auto k = tc_gram_kernel<T, S, MT, NS>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        ProfScope ps_("tc_gram", s);
        k<<<splits, kThreads, smem, s>>>(A, lda, m, n, NP, rows, chunk_stages, P, st);
    } else {
        constexpr int MT = 2, NS = 2;
        size_t smem = (size_t)NS * S * 128 * MT * BK * 2;
        if (smem < kMinSmem) smem = kMinSmem;
        auto k = tc_gram_kernel<T, S, MT, NS>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        ProfScope ps_("tc_gram", s);
        k<<<splits, kThreads, smem, s>>>(A, lda, m, n, NP, rows, chunk_stages, P, st);
    }
    return cudaGetLastError();
}

template <typename T, int S>
cudaError_t nn_launch(const T *A, i64 lda, i64 m, int K, const uint8_t *img, int N, double *C,
                      i64 ldc, DevStatus *st, cudaStream_t s)
{
    const int NP = (N + 15) / 16 * 16;
    constexpr int NS = 3;
    size_t smem = (size_t)NS * S * (128 * 32 * 2 + (size_t)NP * 32 * 2);
    if (smem < kMinSmem) smem = kMinSmem;
    auto k = tc_nn_kernel<T, S, NS>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const i64 nrt = (m + 127) / 128;
    const int grid = (int)(nrt < num_sms() ? nrt : num_sms());
    ProfScope ps_("tc_nn", s);
    k<<<grid, kThreads, smem, s>>>(A, lda, m, K, img, N, NP, C, ldc, st);
    return cudaGetLastError();
}

}  // namespace

int tc_gram_splits(i64 m)
{
    i64 sp = num_sms();
    const i64 max_sp = (m + 255) / 256;
    if (sp > max_sp) sp = max_sp;
    return sp < 1 ? 1 : (int)sp;
}

size_t tc_split_b_bytes(int K, int N, int S)
{
    const int NP = (N + 15) / 16 * 16;
    const int KP = (K + 15) / 16 * 16;
    const int nkb = (KP + 31) / 32;
    return (size_t)nkb * S * NP * 64;
}

template <typename T>
cudaError_t launch_tc_gram(const T *A, i64 lda, i64 m, int n, int S, int splits, double *P,
                           DevStatus *st, cudaStream_t s)
{
    if (n < 1 || n > 256) return cudaErrorInvalidValue;
    return S == 3 ? gram_launch<T, 3>(A, lda, m, n, splits, P, st, s)
                  : gram_launch<T, 2>(A, lda, m, n, splits, P, st, s);
}

cudaError_t launch_tc_split_b(const double *M, i64 ldm, int K, int N, int S, uint8_t *img,
                              cudaStream_t s)
{
    const int NP = (N + 15) / 16 * 16;
    const int KP = (K + 15) / 16 * 16;
    const i64 total = (i64)((KP + 31) / 32) * 4 * NP;
    i64 blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    ProfScope ps_("tc_split_b", s);
    if (S == 3)
        tc_split_b_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(M, ldm, K, N, NP, img);
    else
        tc_split_b_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(M, ldm, K, N, NP, img);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tc_nn(const T *A, i64 lda, i64 m, int K, const uint8_t *img, int N, int S,
                         double *C, i64 ldc, DevStatus *st, cudaStream_t s)
{
    if (N < 1 || N > 256) return cudaErrorInvalidValue;
    return S == 3 ? nn_launch<T, 3>(A, lda, m, K, img, N, C, ldc, st, s)
                  : nn_launch<T, 2>(A, lda, m, K, img, N, C, ldc, st, s);
}

template cudaError_t launch_tc_gram<double>(const double *, i64, i64, int, int, int, double *,
                                            DevStatus *, cudaStream_t);
template cudaError_t launch_tc_gram<float>(const float *, i64, i64, int, int, int, double *,
                                           DevStatus *, cudaStream_t);
template cudaError_t launch_tc_nn<double>(const double *, i64, i64, int, const uint8_t *, int, int,
                                          double *, i64, DevStatus *, cudaStream_t);
template cudaError_t launch_tc_nn<float>(const float *, i64, i64, int, const uint8_t *, int, int,
                                         double *, i64, DevStatus *, cudaStream_t);

}  // namespace tssvd
