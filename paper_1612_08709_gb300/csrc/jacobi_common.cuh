// Device helpers shared by the Jacobi kernels (jacobi.cu, jacobi_mixed.cu,
// jacobi_batch.cu): the bounded grid barrier of the cooperative launches,
// the plane-rotation parameters and the round-robin (circle) pair
// schedule.
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

// Plane rotation for the 2 x 2 symmetric block [a g; g b] (a Gram block:
// a = |x_P|^2, b = |x_Q|^2, g = x_P . x_Q).  Returns (c, s, t, 1) with
// t = s / c the tangent of the angle that annihilates g, or (1, 0, 0, 0)
// when |g| <= tol * sqrt(|a b|).
//
// FP64 on this part has a dependent latency of about 60 cycles per
// add/multiply and about 600 per division or square root, while FP32 and
// integer operations are an order of magnitude faster; a rotation sits on
// the critical path of every round, so it is built from cheap parts:
//  - the skip test in the log2 domain, 2 log2|g| > 2 log2 tol + log2|a| +
//    log2|b|, from the exponent fields and an FP32 log2 of the mantissas
//    (a threshold accurate to about 1e-4 relative);
//  - the angle in FP32: d = b - a in FP64 (no cancellation loss), then d
//    and g reduced to FP32 with a common power-of-two scale by integer
//    operations on their bit patterns, and t = sign(d) g / (|d|/2 +
//    sqrt(d^2/4 + g^2)), the smaller root of t^2 + 2 (d / 2g) t - 1 = 0;
//  - c = 1/sqrt(1 + t^2) and s = c t in FP64 from that one t, so the
//    rotation is orthogonal to working precision whatever t is.  A t with
//    a relative error near 2^-24 leaves |g'| ~ 2^-24 |g|, which the next
//    sweep removes.
// Zeros, subnormals, infinities and angles below FP32's range go through
// the plain FP64 formula instead.
__device__ __forceinline__ int exp_field(double x)
{
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// log2|x| for a normal x: exponent plus an FP32 log2 of the top 23
// mantissa bits.
__device__ __forceinline__ float log2_abs(double x)
{
    const long long bits = __double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7ff);
    const float m = __int_as_float(0x3f800000 | (int)((bits >> 29) & 0x7fffff));
    return (float)(E - 1023) + __log2f(m);
}

// x * 2^(-e) as an FP32, by moving x's exponent; 0 below FP32's normal
// range.  x normal or 0, exp_field(x) <= e.
__device__ __forceinline__ float scaled_f32(double x, int e)
{
    const long long bits = __double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7ff);
    const int fe = E - e + 127;
    if (E == 0 || fe < 1) return 0.0f;
    const unsigned sign = (unsigned)((unsigned long long)bits >> 63) << 31;
    return __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((bits >> 29) & 0x7fffff));
}

// FP64 rotation for the pairs the FP32-angle form cannot take (subnormal or
// non-finite inputs, or g far below |b - a|).  The test is taken against
// sqrt|a| sqrt|b| and the angle as tan = r / (1 + sqrt(1 + r^2)),
// r = |2g| / |b - a| (when |b - a| > |2g|; else from z = 1 / r), so that
// neither overflows or underflows when a and b are hundreds of orders of
// magnitude apart.  An angle that underflows to 0 is no rotation (it would
// be the identity, and counting it would keep the sweep loop going).
__device__ __noinline__ double4 jac_rotation_slow(double a, double b, double g, double tol)
{
    if (g != 0.0 && fabs(g) > tol * (sqrt(fabs(a)) * sqrt(fabs(b)))) {
        const double d = b - a, ad = fabs(d), ag2 = fabs(2.0 * g);
        double tt;
        if (ad > ag2) {
            const double r = ag2 / ad;
            tt = r / (1.0 + sqrt(fma(r, r, 1.0)));
        } else {
            const double z = ad / ag2;
            tt = 1.0 / (z + sqrt(fma(z, z, 1.0)));
        }
        if (tt == 0.0) return make_double4(1.0, 0.0, 0.0, 0.0);
        if (!(d == 0.0 || ((d > 0.0) == (g > 0.0)))) tt = -tt;
        const double c = 1.0 / sqrt(1.0 + tt * tt);
        return make_double4(c, c * tt, tt, 1.0);
    }
    return make_double4(1.0, 0.0, 0.0, 0.0);
}

// gmin > 0 adds a normwise floor: pairs with |g| <= gmin are left alone.
__device__ __forceinline__ double4 jac_rotation(double a, double b, double g, double tol,
                                                float log2tol, double gmin = 0.0)
{
    if (!(fabs(g) > gmin)) return make_double4(1.0, 0.0, 0.0, 0.0);
    const int Ea = exp_field(a), Eb = exp_field(b), Eg = exp_field(g);
    if (Ea == 0 || Eb == 0 || Eg == 0 || Ea == 0x7ff || Eb == 0x7ff || Eg == 0x7ff)
        return jac_rotation_slow(a, b, g, tol);
    if (!(2.0f * log2_abs(g) > 2.0f * log2tol + log2_abs(a) + log2_abs(b)))
        return make_double4(1.0, 0.0, 0.0, 0.0);
    const double d = b - a;
    const int Ed = exp_field(d);
    const int e = Ed > Eg ? Ed : Eg;
    if (Eg - e < -100) return jac_rotation_slow(a, b, g, tol);
    const float hf = 0.5f * scaled_f32(d, e), gf = scaled_f32(g, e);
    float tf = gf / (fabsf(hf) + sqrtf(fmaf(hf, hf, gf * gf)));
    if (hf < 0.0f) tf = -tf;
    const double t = (double)tf;
    const double c = rsqrt(fma(t, t, 1.0));
    return make_double4(c, c * t, t, 1.0);
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
