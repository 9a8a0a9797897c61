// Batched one-sided (Hestenes) Jacobi: many independent small solves in one
// launch, a cluster of two CTAs per problem, optionally started by an FP32
// phase (see the kernel).
//
// The grid solver (jacobi.cu) spreads one problem over the GPU, one CTA per
// rotation pair and a grid barrier per round, which minimises one solve's
// latency.  A batch of hundreds of problems wants throughput instead: on
// this GPU the FP64 pipe (two lanes per clock per SM) bounds the rotations,
// so each problem's rounds run inside a small cluster (a hardware cluster
// barrier per round, no grid barrier and no spin-wait), and the problems
// fill the SMs side by side.  Tasks are given largest first so that the
// long solves start first.
//
// The cluster's warps take the n/2 pairs of a round, one warp per pair at a
// time: each lane holds up to 8 entries of the two columns in registers,
// the inner product is a warp reduction (an xor butterfly, so every lane
// holds the same bits and takes the same decision), the rotation comes
// from the same parameter function as the grid solver (jac_rotation), and
// the squared column norms are tracked in shared memory in closed form
// (recomputed at every sweep start, and for a column whose update cancels
// below 2^-16 of its inputs).  Rounds follow the circle schedule, so a
// sweep visits every pair once, in the grid solver's order.
#include <cooperative_groups.h>

#include "jacobi_common.cuh"

namespace tssvd {

namespace {

constexpr int kBatchJacobiThreads = 256;
constexpr int kBatchJacobiWarps = kBatchJacobiThreads / 32;
// CTAs per task.  Measured on 512 members (n 16..256): one CTA 1,965 ms a
// step, two 1,550, four 1,631 -- two halve the largest members' solves,
// which set each launch's length, for one cluster barrier a round.
constexpr int kBatchCluster = 2;
constexpr int kBatchF32Sweeps = 40;  // cap of the FP32 phase

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_maxi(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// C = op(A) B for n x n column-major matrices (op(A) = A^T when trans),
// the cluster's threads (tid of NTC) sharing 4 x 4 output blocks.  FP64
// FMAs from L1/L2-resident operands: n^3 FMAs, about two FP64 sweeps'
// worth of work at n = 256.
__device__ void cluster_gemm(const double *A, const double *B, double *Cm, int n, bool trans,
                             int tid, int NTC)
{
    const int nb = (n + 3) / 4;
    for (int blk = tid; blk < nb * nb; blk += NTC) {
        const int i0 = (blk % nb) * 4, j0 = (blk / nb) * 4;
        double acc[4][4];
#pragma unroll
        for (int ii = 0; ii < 4; ii++)
#pragma unroll
            for (int jj = 0; jj < 4; jj++) acc[ii][jj] = 0.0;
        for (int k = 0; k < n; k++) {
            double a[4], b[4];
#pragma unroll
            for (int ii = 0; ii < 4; ii++) {
                const int i = i0 + ii;
                a[ii] = i < n ? (trans ? A[(size_t)i * n + k] : A[(size_t)k * n + i]) : 0.0;
            }
#pragma unroll
            for (int jj = 0; jj < 4; jj++) {
                const int j = j0 + jj;
                b[jj] = j < n ? B[(size_t)j * n + k] : 0.0;
            }
#pragma unroll
            for (int ii = 0; ii < 4; ii++)
#pragma unroll
                for (int jj = 0; jj < 4; jj++) acc[ii][jj] = fma(a[ii], b[jj], acc[ii][jj]);
        }
#pragma unroll
        for (int jj = 0; jj < 4; jj++)
#pragma unroll
            for (int ii = 0; ii < 4; ii++)
                if (i0 + ii < n && j0 + jj < n) Cm[(size_t)(j0 + jj) * n + i0 + ii] = acc[ii][jj];
    }
}

// One solve spread over a cluster of C CTAs (C x 8 warps take the pairs of
// a round).  The round boundary is the cluster barrier (a
// hardware barrier with release / acquire ordering at cluster scope, so the
// columns one CTA rotated are seen by the others in the next round); each
// CTA keeps a copy of the tracked norms in its shared memory and a warp
// that updates a norm writes it into every copy (distributed shared
// memory); the sweep's rotation count is summed in rank 0's shared memory.
// Control flow is uniform over the cluster (the sweep loop ends on the
// summed count), so every CTA reaches every barrier.
template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kBatchJacobiThreads)
    jacobi_batch_cluster_kernel(const JacobiTask *tasks, int max_sweeps)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double nrm[kJacobiBatchMaxN];
    __shared__ int rot_count;
    __shared__ int emax_s;
    const int rank = (int)cl.block_rank();
    const JacobiTask tk = tasks[blockIdx.x / C];
    const int n = tk.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (n < 2 || n > kJacobiBatchMaxN) {
        if (threadIdx.x == 0 && rank == 0) tk.st->sweeps[tk.which] = n < 2 ? 0 : -1;
        return;
    }
    double *nrm_r[C];
#pragma unroll
    for (int r = 0; r < C; r++) nrm_r[r] = cl.map_shared_rank(nrm, r);
    int *cnt0 = cl.map_shared_rank(&rot_count, 0);
    cl.sync();  // every CTA of the cluster runs before its shared memory is written
    const int gw = rank * kBatchJacobiWarps + warp, GW = C * kBatchJacobiWarps;
    double *X = tk.X, *J = tk.J;
    const int npad = n + (n & 1), rounds = npad - 1;
    const double tol = tk.tol;
    const float log2tol = log2f((float)tol);
    if (tk.w32) {
        // Two-precision start: the same one-sided sweeps in FP32 on X
        // scaled by a power of two (threshold 2^-20, at most
        // kBatchF32Sweeps sweeps) accumulate J32; K = J32 in FP64 made
        // orthogonal by two Newton-Schulz steps K <- K (3I - K^T K) / 2;
        // X <- X K, and J starts as K.  The FP64 sweeps below then decide
        // the result.
        const int nn = n * n;
        const int tid = rank * kBatchJacobiThreads + (int)threadIdx.x;
        const int NTC = C * kBatchJacobiThreads;
        float *X32 = tk.w32, *J32 = tk.w32 + (size_t)nn;
        double *K = tk.wk, *H = tk.wk + (size_t)nn, *Kn = reinterpret_cast<double *>(tk.w32);
        int *emax0 = cl.map_shared_rank(&emax_s, 0);
        if (threadIdx.x == 0 && rank == 0) emax_s = -2000;
        cl.sync();
        int em = -2000;
        for (int e = tid; e < nn; e += NTC) {
            const double v = fabs(X[e]);
            if (v > 0.0) em = max(em, ilogb(v));
        }
        em = warp_maxi(em);
        if (lane == 0) atomicMax(emax0, em);
        cl.sync();
        const int E = *emax0;
        for (int e = tid; e < nn; e += NTC) {
            X32[e] = (float)ldexp(X[e], -E);
            J32[e] = (e / n == e % n) ? 1.0f : 0.0f;
        }
        cl.sync();
        int f32_sweeps = kBatchF32Sweeps;
        for (int sweep = 1; sweep <= kBatchF32Sweeps; sweep++) {
            if (threadIdx.x == 0 && rank == 0) rot_count = 0;
            cl.sync();
            int my_rot = 0;
            for (int t = 0; t < rounds; t++) {
                for (int k = gw; k < npad / 2; k += GW) {
                    int P, Q;
                    circle_pair(k, t, npad, P, Q);
                    if (Q >= n) continue;
                    float *xp = X32 + (size_t)P * n, *xq = X32 + (size_t)Q * n;
                    float *jp = J32 + (size_t)P * n, *jq = J32 + (size_t)Q * n;
                    float u[8], v[8], ju[8], jv[8];
                    float a = 0.0f, b = 0.0f, g = 0.0f;
#pragma unroll
                    for (int c = 0; c < 8; c++) {
                        const int i = lane + 32 * c;
                        u[c] = i < n ? xp[i] : 0.0f;
                        v[c] = i < n ? xq[i] : 0.0f;
                        ju[c] = i < n ? jp[i] : 0.0f;
                        jv[c] = i < n ? jq[i] : 0.0f;
                        a = fmaf(u[c], u[c], a);
                        b = fmaf(v[c], v[c], b);
                        g = fmaf(u[c], v[c], g);
                    }
                    a = warp_sumf(a);
                    b = warp_sumf(b);
                    g = warp_sumf(g);
                    if (!(a > 0.0f && b > 0.0f && fabsf(g) > 0x1p-20f * sqrtf(a) * sqrtf(b)))
                        continue;
                    const float zeta = (b - a) / (2.0f * g);
                    const float tt = fabsf(zeta) > 1e18f
                                         ? 0.5f / zeta
                                         : copysignf(1.0f, zeta) /
                                               (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
                    const float c = rsqrtf(fmaf(tt, tt, 1.0f)), sn = c * tt;
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const int i = lane + 32 * e;
                        if (i < n) {
                            xp[i] = c * u[e] - sn * v[e];
                            xq[i] = sn * u[e] + c * v[e];
                            jp[i] = c * ju[e] - sn * jv[e];
                            jq[i] = sn * ju[e] + c * jv[e];
                        }
                    }
                    my_rot++;
                }
                cl.sync();
            }
            if (lane == 0 && my_rot != 0) atomicAdd(cnt0, my_rot);
            cl.sync();
            const int total = *cnt0;
            cl.sync();
            if (total == 0) {
                f32_sweeps = sweep;
                break;
            }
        }
        if (threadIdx.x == 0 && rank == 0) atomicAdd(&tk.st->sweeps[3], f32_sweeps);
        for (int e = tid; e < nn; e += NTC) K[e] = (double)J32[e];
        cl.sync();
        for (int it = 0; it < 2; it++) {
            cluster_gemm(K, K, H, n, true, tid, NTC);  // H = K^T K
            cl.sync();
            for (int e = tid; e < nn; e += NTC)
                H[e] = ((e / n == e % n) ? 1.5 : 0.0) - 0.5 * H[e];
            cl.sync();
            cluster_gemm(K, H, Kn, n, false, tid, NTC);  // Kn = K (3I - K^T K) / 2
            cl.sync();
            for (int e = tid; e < nn; e += NTC) K[e] = Kn[e];
            cl.sync();
        }
        cluster_gemm(X, K, H, n, false, tid, NTC);  // H = X K
        cl.sync();
        for (int e = tid; e < nn; e += NTC) {
            X[e] = H[e];
            if (J) J[e] = K[e];
        }
        cl.sync();
    }
    int done = -1;
    for (int sweep = 1; sweep <= max_sweeps; sweep++) {
        for (int j = gw; j < n; j += GW) {
            const double *x = X + (size_t)j * n;
            double acc = 0.0;
            for (int i = lane; i < n; i += 32) acc = fma(x[i], x[i], acc);
            acc = warp_sum(acc);
            if (lane == 0)
#pragma unroll
                for (int r = 0; r < C; r++) nrm_r[r][j] = acc;
        }
        if (threadIdx.x == 0 && rank == 0) rot_count = 0;
        cl.sync();
        int my_rot = 0;
        for (int t = 0; t < rounds; t++) {
            for (int k = gw; k < npad / 2; k += GW) {
                int P, Q;
                circle_pair(k, t, npad, P, Q);
                if (Q >= n) continue;
                double *xp = X + (size_t)P * n, *xq = X + (size_t)Q * n;
                double u[8], v[8];
                double g = 0.0;
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    const int i = lane + 32 * c;
                    u[c] = i < n ? xp[i] : 0.0;
                    v[c] = i < n ? xq[i] : 0.0;
                    g = fma(u[c], v[c], g);
                }
                g = warp_sum(g);
                double a = nrm[P], b = nrm[Q];
                if (a < 0.0 || b < 0.0) {
                    double sa = 0.0, sb = 0.0;
#pragma unroll
                    for (int c = 0; c < 8; c++) {
                        sa = fma(u[c], u[c], sa);
                        sb = fma(v[c], v[c], sb);
                    }
                    sa = warp_sum(sa);
                    sb = warp_sum(sb);
                    if (a < 0.0) a = sa;
                    if (b < 0.0) b = sb;
                }
                const double4 r = jac_rotation(a, b, g, tol, log2tol);
                double a1 = a, b1 = b;
                if (r.w != 0.0) {
                    const double c = r.x, sn = r.y;
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const int i = lane + 32 * e;
                        if (i < n) {
                            xp[i] = c * u[e] - sn * v[e];
                            xq[i] = sn * u[e] + c * v[e];
                        }
                    }
                    if (J) {
                        double *jp = J + (size_t)P * n, *jq = J + (size_t)Q * n;
#pragma unroll
                        for (int e = 0; e < 8; e++) {
                            const int i = lane + 32 * e;
                            if (i < n) {
                                const double x = jp[i], y = jq[i];
                                jp[i] = c * x - sn * y;
                                jq[i] = sn * x + c * y;
                            }
                        }
                    }
                    const double cc = c * c, ss = sn * sn, cs2 = 2.0 * c * sn;
                    a1 = fma(cc, a, fma(-cs2, g, ss * b));
                    b1 = fma(ss, a, fma(cs2, g, cc * b));
                    const double floor = 0x1p-16 * (a + b);
                    if (!(a1 >= floor)) a1 = -1.0;
                    if (!(b1 >= floor)) b1 = -1.0;
                    my_rot++;
                }
                if (lane == 0)
#pragma unroll
                    for (int q = 0; q < C; q++) {
                        nrm_r[q][P] = a1;
                        nrm_r[q][Q] = b1;
                    }
            }
            cl.sync();  // this round's columns and norms seen by the whole cluster
        }
        if (lane == 0 && my_rot != 0) atomicAdd(cnt0, my_rot);
        cl.sync();
        const int total = *cnt0;
        cl.sync();  // every CTA has read the count before rank 0 resets it
        if (total == 0) {
            done = sweep;
            break;
        }
    }
    if (threadIdx.x == 0 && rank == 0) tk.st->sweeps[tk.which] = done;
}

__global__ void init_identity_batch_kernel(const JacobiTask *tasks)
{
    const JacobiTask tk = tasks[blockIdx.x];
    if (!tk.J || tk.n < 1 || tk.n > kJacobiBatchMaxN) return;
    const int n = tk.n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        tk.J[e] = (e / n == e % n) ? 1.0 : 0.0;
}

}  // namespace

cudaError_t launch_jacobi_batch(const JacobiTask *tasks, int ntasks, int max_sweeps,
                                cudaStream_t s)
{
    if (ntasks < 1) return cudaSuccess;
    {
        ProfScope ps_("init_identity", s);
        init_identity_batch_kernel<<<ntasks, 256, 0, s>>>(tasks);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ProfScope ps_("jacobi_batch", s);
    jacobi_batch_cluster_kernel<kBatchCluster>
        <<<kBatchCluster * ntasks, kBatchJacobiThreads, 0, s>>>(tasks, max_sweeps);
    return cudaGetLastError();
}

}  // namespace tssvd
