// Device helpers shared by the Jacobi kernels (jacobi.cu, jacobi_mixed.cu):
// the bounded grid barrier of the cooperative launches and the
// round-robin (circle) pair schedule.
#pragma once

#include "common.cuh"

namespace tssvd {
namespace {

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier with a bounded wait.  The arrival counter only grows: the
// e-th barrier of the launch (epoch e, counted by every CTA) completes when
// it reaches e * gridDim.x.  One release-add per CTA to arrive, acquire
// loads to wait.  Returns false when the call must be abandoned (this CTA
// or another timed out).
__device__ bool grid_barrier(unsigned long long *count, int &epoch, int *err)
{
    __shared__ int s_ok;
    __syncthreads();
    epoch++;
    if (threadIdx.x == 0) {
        int ok = 1;
        red_release_add64(count, 1ull);
        const unsigned long long target = (unsigned long long)epoch * gridDim.x;
        int spins = 0;
        unsigned long long t0 = 0;
        while (ld_acquire64(count) < target) {
            if (++spins < 256) continue;
            if (t0 == 0) t0 = global_ns();
            if (ld_volatile(err) != 0) {
                ok = 0;
                break;
            }
            if (global_ns() - t0 > kBarrierTimeoutNs) {
                atomicCAS(err, 0, TSSVD_ETIMEOUT);
                ok = 0;
                break;
            }
            spins = 200;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The same barrier in two halves, so that work no other CTA waits for can
// run while the barrier completes: grid_arrive publishes this CTA's writes
// (release) and counts it in; grid_wait returns once every CTA has arrived
// (acquire), or false when the call must be abandoned.
__device__ __forceinline__ void grid_arrive(unsigned long long *count, int &epoch)
{
    __syncthreads();
    epoch++;
    if (threadIdx.x == 0) red_release_add64(count, 1ull);
}

__device__ bool grid_wait(unsigned long long *count, int epoch, int *err)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long target = (unsigned long long)epoch * gridDim.x;
        int spins = 0;
        unsigned long long t0 = 0;
        while (ld_acquire64(count) < target) {
            if (++spins < 256) continue;
            if (t0 == 0) t0 = global_ns();
            if (ld_volatile(err) != 0) {
                ok = 0;
                break;
            }
            if (global_ns() - t0 > kBarrierTimeoutNs) {
                atomicCAS(err, 0, TSSVD_ETIMEOUT);
                ok = 0;
                break;
            }
            spins = 200;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void circle_pair(int pr, int t, int npad, int &P, int &Q)
{
    // positions a - 1 + t and b - 1 + t stay below 2 * rounds, so one
    // conditional subtraction reduces them (no integer division)
    const int rounds = npad - 1;
    const int a = pr, b = npad - 1 - pr;
    int x = a - 1 + t, y = b - 1 + t;
    if (x >= rounds) x -= rounds;
    if (y >= rounds) y -= rounds;
    P = (a == 0) ? 0 : 1 + x;
    Q = (b == 0) ? 0 : 1 + y;
    if (P > Q) {
        int tmp = P;
        P = Q;
        Q = tmp;
    }
}

}  // namespace
}  // namespace tssvd
