// One-sided Jacobi in two precisions for the wide n x n problems (n above
// a few hundred), where the FP64 solver is bound by GB300's FP64 rate (2
// FP64 fused multiply-adds per clock per SM, against 128 in FP32).
//
//  1. FP32 phase: X (scaled by a power of two into FP32's range) is
//     orthogonalised in FP32 by the same round-robin one-sided Jacobi,
//     accumulating the rotations K32 (relative threshold 2^-20; its sweep
//     count is added to st->sweeps[3]).
//  2. K = K32 in FP64, made orthogonal to working precision by two
//     Newton-Schulz steps K <- K (3 I - K^T K) / 2 (each squares the
//     departure from orthogonality, about 1e-6 after the FP32 phase).
//  3. X0 = X K in FP64 (an orthogonal change of basis: X0 has the same
//     column space and Gram spectrum as X), whose columns are orthogonal
//     to FP32 accuracy.
//  4. FP64 phase: the FP64 one-sided Jacobi on X0 with the caller's
//     threshold, usually 3 sweeps instead of 14-18.  When the rotations
//     are wanted, J = K J0 (J0 the FP64 phase's).
// The result is the FP64 solver's: the FP32 phase only chooses a better
// starting basis; every convergence decision that the output depends on
// is the FP64 phase's.  Products are FP64 (nn_kernel / tn_partial).
#include "common.cuh"
#include "jacobi_common.cuh"

namespace tssvd {

namespace {

struct Jacobi32Args {
    float *X;
    float *J;
    i64 ld;  // both n x n column-major with this leading dimension
    int n, npad, max_sweeps;
    float tol;
    int *rot;  // [max_sweeps] rotation counts
    DevStatus *st;
};

// Rotation for the 2 x 2 Gram block [a g; g b] in FP32: (c, s) with
// t = s / c the tangent of the smaller angle that annihilates g, computed
// in the overflow-free form; (1, 0) when |g| <= tol sqrt(a) sqrt(b).
__device__ __forceinline__ bool rot32(float a, float b, float g, float tol, float &c, float &s)
{
    if (!(fabsf(g) > tol * (sqrtf(a) * sqrtf(b)))) return false;
    const float d = b - a, ad = fabsf(d), ag2 = fabsf(2.0f * g);
    float t;
    if (ad > ag2) {
        const float r = ag2 / ad;
        t = r / (1.0f + sqrtf(fmaf(r, r, 1.0f)));
    } else {
        const float z = ad / ag2;
        t = 1.0f / (z + sqrtf(fmaf(z, z, 1.0f)));
    }
    if (t == 0.0f) return false;
    if (!(d == 0.0f || ((d > 0.0f) == (g > 0.0f)))) t = -t;
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = c * t;
    return true;
}

// One CTA per pair of the round (a grid of npairs CTAs when they fit,
// else CTAs take several pairs); columns P, Q of X and of J in registers
// (CH values per thread, n <= CH * NT); one grid barrier per round.
template <int NT, int CH>
__global__ void __launch_bounds__(NT) jacobi32_kernel(Jacobi32Args p)
{
    __shared__ float red[3][NT / 32];
    __shared__ float rs[2];
    __shared__ int rflag;
    const int npairs = p.npad / 2, rounds = p.npad - 1, n = p.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0, local_rot = 0, done = -1;
    for (int sweep = 0; sweep < p.max_sweeps; sweep++) {
        for (int t = 0; t < rounds; t++) {
            for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
                int P, Q;
                circle_pair(pr, t, p.npad, P, Q);
                if (Q >= n) continue;  // the padding column of an odd n
                float *xp = p.X + (i64)P * p.ld, *xq = p.X + (i64)Q * p.ld;
                float *jp = p.J + (i64)P * p.ld, *jq = p.J + (i64)Q * p.ld;
                // J's columns are loaded with X's, so that the rotation's
                // update waits on no second round trip to L2
                float u[CH], v[CH], ju[CH], jv[CH];
                float a = 0.0f, b = 0.0f, g = 0.0f;
#pragma unroll
                for (int j = 0; j < CH; j++) {
                    const int i = tid + j * NT;
                    u[j] = i < n ? __ldcg(xp + i) : 0.0f;
                    v[j] = i < n ? __ldcg(xq + i) : 0.0f;
                    ju[j] = i < n ? __ldcg(jp + i) : 0.0f;
                    jv[j] = i < n ? __ldcg(jq + i) : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < CH; j++) {
                    a = fmaf(u[j], u[j], a);
                    b = fmaf(v[j], v[j], b);
                    g = fmaf(u[j], v[j], g);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (lane == 0) {
                    red[0][warp] = a;
                    red[1][warp] = b;
                    red[2][warp] = g;
                }
                __syncthreads();
                if (tid == 0) {
                    float A = 0.0f, B = 0.0f, Gs = 0.0f;
#pragma unroll
                    for (int w = 0; w < NT / 32; w++) {
                        A += red[0][w];
                        B += red[1][w];
                        Gs += red[2][w];
                    }
                    float c = 1.0f, s = 0.0f;
                    const bool r = rot32(A, B, Gs, p.tol, c, s);
                    rs[0] = c;
                    rs[1] = s;
                    rflag = r ? 1 : 0;
                    if (r) local_rot++;
                }
                __syncthreads();
                const float c = rs[0], s = rs[1];
                const int r = rflag;
                __syncthreads();  // rs, rflag and red are rewritten by the next pair
                if (!r) continue;
#pragma unroll
                for (int j = 0; j < CH; j++) {
                    const int i = tid + j * NT;
                    if (i < n) {
                        __stcg(xp + i, c * u[j] - s * v[j]);
                        __stcg(xq + i, s * u[j] + c * v[j]);
                        __stcg(jp + i, c * ju[j] - s * jv[j]);
                        __stcg(jq + i, s * ju[j] + c * jv[j]);
                    }
                }
            }
            if (t == rounds - 1 && tid == 0 && local_rot != 0) {
                atomicAdd(p.rot + sweep, local_rot);
                local_rot = 0;
            }
            grid_arrive(bar, epoch);
            if (!grid_wait(bar, epoch, &p.st->err)) return;
        }
        if (ld_acquire(p.rot + sweep) == 0) {
            done = sweep + 1;
            break;
        }
    }
    // FP32 sweeps of the call's mixed solves, summed (the cap when it was reached)
    if (blockIdx.x == 0 && tid == 0) atomicAdd(&p.st->sweeps[3], done > 0 ? done : p.max_sweeps);
}

// Largest |x| of an n x n array as an ordered bit pattern (x != 0 finite).
__global__ void maxabs_bits_kernel(const double *X, i64 total, unsigned long long *out)
{
    unsigned long long m = 0;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(X[e]) & ~(1ull << 63);
        if (b < 0x7ff0000000000000ull && b > m) m = b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// X32 = X 2^-e (e from the largest |x|, so that it maps below 2; entries
// below FP32's range become 0) and J32 = I.
__global__ void to_f32_kernel(const double *X, i64 n, const unsigned long long *mx, float *X32,
                              float *J32)
{
    const int ex = (int)((*mx >> 52) & 0x7ff) - 1023;  // exponent of the largest entry
    const i64 total = n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        X32[e] = (float)ldexp(X[e], -ex);
        J32[e] = (e / n == e % n) ? 1.0f : 0.0f;
    }
}

__global__ void to_f64_kernel(const float *a, i64 total, double *b)
{
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x)
        b[e] = (double)a[e];
}

// M = (3 I - H) / 2 (n x n row-major).
__global__ void ns_matrix_kernel(const double *H, i64 n, double *M)
{
    const i64 total = n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x)
        M[e] = ((e / n == e % n) ? 1.5 : 0.0) - 0.5 * H[e];
}

unsigned grid_for(i64 total)
{
    i64 b = (total + 255) / 256;
    const i64 cap = (i64)num_sms() * 8;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

bool jacobi_mixed_applies(i64 n) { return n >= kJacobiMixedMinN && n <= kJacobiMixedMaxN; }

cudaError_t launch_jacobi_mixed(double *X, i64 n, double *Jout, const JacobiMixedScratch &w,
                                int max_sweeps, int *ctr, double *prm, DevStatus *st, int which,
                                cudaStream_t s, double tol)
{
    if (!jacobi_mixed_applies(n)) return cudaErrorInvalidValue;
    cudaError_t e;
    const i64 nn = n * n;
    float *X32 = reinterpret_cast<float *>(w.f32);
    float *J32 = X32 + nn;
    unsigned long long *mx = reinterpret_cast<unsigned long long *>(prm);
    // ---- FP32 phase
    if ((e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    {
        ProfScope ps_("jacobi_mixed_cvt", s);
        maxabs_bits_kernel<<<grid_for(nn), 256, 0, s>>>(X, nn, mx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        ProfScope ps_("jacobi_mixed_cvt", s);
        to_f32_kernel<<<grid_for(nn), 256, 0, s>>>(X, n, mx, X32, J32);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(int) * (size_t)(max_sweeps + 4), s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(&st->bar[0], 0, sizeof(int) * 4, s)) != cudaSuccess) return e;
    {
        Jacobi32Args a;
        a.X = X32;
        a.J = J32;
        a.ld = n;
        a.n = (int)n;
        a.npad = (int)(n + (n & 1));
        a.max_sweeps = max_sweeps < kJacobiMixedF32Sweeps ? max_sweeps : kJacobiMixedF32Sweeps;
        a.tol = 0x1p-20f;
        a.rot = ctr;
        a.st = st;
        constexpr int NT = 128;
        const void *kern = n <= 4 * NT   ? (const void *)jacobi32_kernel<NT, 4>
                           : n <= 8 * NT ? (const void *)jacobi32_kernel<NT, 8>
                                         : (const void *)jacobi32_kernel<NT, 16>;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        const int npairs = a.npad / 2;
        int blocks = num_sms() * per_sm;
        if (blocks > npairs) blocks = npairs;
        void *args[] = {&a};
        ProfScope ps_("jacobi_svd32", s);
        if ((e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(NT), args, 0, s)) !=
            cudaSuccess)
            return e;
    }
    // ---- K = J32 in FP64, two Newton-Schulz steps.  The column-major K
    // read as row-major is G = K^T; G <- G (3 I - G^T G) / 2 orthogonalises
    // G and therefore K.
    {
        ProfScope ps_("jacobi_mixed_cvt", s);
        to_f64_kernel<<<grid_for(nn), 256, 0, s>>>(J32, nn, w.K);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    double *G = w.K, *G2 = w.T;
    const int sp = tn_splits(n, n, n, false);
    for (int it = 0; it < 2; it++) {
        if ((e = launch_tn_partial<double, double>(G, n, G, n, n, n, n, sp, false, w.P, s)) !=
            cudaSuccess)
            return e;
        if ((e = launch_tn_reduce(w.P, sp, n, n, nullptr, nullptr, false, w.H, n, s)) !=
            cudaSuccess)
            return e;
        {
            ProfScope ps_("jacobi_mixed_ns", s);
            ns_matrix_kernel<<<grid_for(nn), 256, 0, s>>>(w.H, n, w.H);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if ((e = launch_nn<double, double>(G, n, w.H, n, n, n, n, G2, n, w.NP, s)) != cudaSuccess)
            return e;
        double *tt = G;
        G = G2;
        G2 = tt;
    }
    // ---- X0 = X K (column-major): as row-major buffers, X0^T = K^T X^T = G X^T
    if ((e = launch_nn<double, double>(G, n, X, n, n, n, n, w.X0, n, w.NP, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(X, w.X0, sizeof(double) * (size_t)nn, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return e;
    // ---- FP64 phase on X0; J = K J0 (as row-major buffers J^T = J0^T K^T = J0buf G)
    double *J0 = Jout ? w.X0 : nullptr;
    if ((e = launch_jacobi(X, n, J0, n, (int)n, (int)n, max_sweeps, ctr, prm, st, which, s, tol)) !=
        cudaSuccess)
        return e;
    if (Jout) {
        if ((e = launch_nn<double, double>(J0, n, G, n, n, n, n, Jout, n, w.NP, s)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace tssvd
