// ts_gram_noalloc: the Gram matrix B = A^T A without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host framework that
// owns every byte of device memory through its own pool (a cudaMalloc from
// underneath it can fail or fragment the pool), or latency-sensitive code
// that cannot afford the implicit device-wide synchronisation a
// cudaMalloc/cudaFree may perform.  For them this entry point runs the same
// split-K Gram kernels as ts_gram, but keeps the split-K partial sums in a
// fixed scratch array that is part of the library's device image instead
// of in a caller-provided or library-allocated workspace.
//
// The scratch array is 4 MiB (2^19 doubles).  Every GPU on which the
// library is loaded holds it until the process exits.  It bounds the
// problem size: the partials take splits * n * n doubles with at least one
// split, so n is limited to 724 (724^2 <= 2^19).
#include <stdio.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr long long kScratchDoubles = 1LL << 19;  // 4 MiB
constexpr long long kMaxN = 724;                   // largest n with n * n <= kScratchDoubles
static_assert(kMaxN * kMaxN <= kScratchDoubles && (kMaxN + 1) * (kMaxN + 1) > kScratchDoubles,
              "kMaxN must be the largest n whose n x n partial fits the scratch");
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol, never a usable address: its device address is obtained
// per device with cudaGetSymbolAddress below.
static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).  Returns nullptr on failure.
double *scratch_on_current_device(int *dev_out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    *dev_out = dev;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess || !p) {
            fprintf(stderr, "ts_gram_noalloc: cudaGetSymbolAddress failed on device %d: %s\n",
                    dev, cudaGetErrorString(e));
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = (double *)p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

using namespace tssvd;

extern "C" int ts_gram_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, double *B,
                               void *stream)
{
    if (!A) return -1;
    if (m < 1) return -2;
    if (n < 1) return -3;
    if (n > kMaxN) {  // (compared directly: n * n could overflow for absurd n)
        fprintf(stderr,
                "ts_gram_noalloc: n = %lld is too large; the fixed 4 MiB scratch holds the "
                "partial Gram matrices only for n <= 724 (use ts_gram instead)\n",
                (long long)n);
        return -3;
    }
    if (lda < n) return -4;
    if (!B) return -5;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = -1;
    double *P = scratch_on_current_device(&dev);
    if (!P) return TSSVD_ECUDA;
    // As many row splits as ts_gram would use, capped by the scratch size.
    long long sp = tn_splits(m, n, n, true);
    const long long cap = kScratchDoubles / (n * n);
    if (sp > cap) sp = cap;
    if (sp < 1) sp = 1;
    // Nothing needs clearing: every partial entry the reduction reads (the
    // upper tiles of every split) is written by the partial kernel first.
    cudaError_t e = launch_tn_partial<double, double>(A, lda, A, lda, m, n, n, (int)sp, true, P, s);
    if (e == cudaSuccess) e = launch_tn_reduce(P, (int)sp, n, n, nullptr, nullptr, true, B, n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        fprintf(stderr, "ts_gram_noalloc: %s\n", cudaGetErrorString(e));
        cudaGetLastError();
        return TSSVD_ECUDA;
    }
    return TSSVD_OK;
}
