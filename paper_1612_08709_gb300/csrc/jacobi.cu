// One-sided (Hestenes) Jacobi for the n x n eigenproblems and the small
// SVD of Algorithm 4, in FP64 on the GPU.
//
// The paper leaves the small eigensolver open (Algorithms 3 and 4 only ask
// for "the eigendecomposition" and "the singular value decomposition").
// Hestenes' method orthogonalises the columns of X by plane rotations
// J: X J has orthogonal columns.  For a symmetric positive semi-definite X
// (a Gram matrix) the columns of J are its eigenvectors and the column
// norms its eigenvalues; for a general X it is an SVD.
//
// Parallel order: the round-robin ("circle") schedule pairs all columns in
// n-1 rounds of n/2 disjoint pairs, so every round's rotations are
// independent.  One CTA handles one pair at a time (dot products reduced
// in a fixed order, then the two-column update of X and J); rounds are
// separated by a grid-wide barrier.  The kernel is launched cooperatively
// so all CTAs are co-resident, and every wait in the barrier is bounded
// (about two seconds of %globaltimer); on expiry the kernel sets the error
// word of the status block and all CTAs return.  The 64-bit arrival counter
// grows by gridDim.x per barrier and is zeroed before every launch.
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

struct JacobiArgs {
    double *X;
    i64 ldx;
    double *J;
    i64 ldj;
    int nr, nc, npad;
    int max_sweeps;
    double tol;
    int *rot;  // [max_sweeps] rotation counts
    DevStatus *st;
    int which;
};

// Block sums of three per-thread partials; the totals are valid in
// thread 0 only.  A halving shuffle tree in which only the receiving lanes
// add, then thread 0 adds the warp partials in a fixed order (FP64
// arithmetic is scarce on this part, so no lane does redundant adds).
template <int NT>
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double (*red)[NT / 32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ta = __shfl_down_sync(0xffffffffu, a, o);
        const double tb = __shfl_down_sync(0xffffffffu, b, o);
        const double tc = __shfl_down_sync(0xffffffffu, c, o);
        if (lane < o) {
            a += ta;
            b += tb;
            c += tc;
        }
    }
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
        red[2][warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = red[0][0];
        b = red[1][0];
        c = red[2][0];
#pragma unroll
        for (int w = 1; w < NT / 32; w++) {
            a += red[0][w];
            b += red[1][w];
            c += red[2][w];
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) jacobi_kernel(JacobiArgs p)
{
    __shared__ double red[3][NT / 32];
    __shared__ double rot_s[3];
    const int npairs = p.npad / 2;
    const int rounds = p.npad - 1;
    const double tol = p.tol;
    int local_rot = 0;
    int done = -1;
    unsigned long long *bar_count = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0;
    for (int sweep = 0; sweep < p.max_sweeps; sweep++) {
        for (int t = 0; t < rounds; t++) {
            for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
                const int a = pr, b = p.npad - 1 - pr;
                int P = (a == 0) ? 0 : 1 + (a - 1 + t) % rounds;
                int Q = (b == 0) ? 0 : 1 + (b - 1 + t) % rounds;
                if (P > Q) {
                    int tmp = P;
                    P = Q;
                    Q = tmp;
                }
                if (Q >= p.nc) continue;  // the padding column of an odd nc
                double *xp = p.X + (i64)P * p.ldx;
                double *xq = p.X + (i64)Q * p.ldx;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = threadIdx.x; i < p.nr; i += NT) {
                    const double u = __ldcg(xp + i), v = __ldcg(xq + i);
                    al = fma(u, u, al);
                    be = fma(v, v, be);
                    ga = fma(u, v, ga);
                }
                block_sum3<NT>(al, be, ga, red);
                // one thread computes the rotation (FP64 division and square
                // root are slow on this part), the block reads it from smem
                if (threadIdx.x == 0) {
                    double c = 1.0, sn = 0.0, rot = 0.0;
                    if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
                        // tan(theta) is the smaller root of t^2 + 2 zeta t - 1 = 0,
                        // which annihilates the (P,Q) inner product.
                        const double zeta = (be - al) / (2.0 * ga);
                        double tt;
                        if (fabs(zeta) > 1e150)
                            tt = 0.5 / zeta;
                        else
                            tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        sn = c * tt;
                        rot = 1.0;
                    }
                    rot_s[0] = c;
                    rot_s[1] = sn;
                    rot_s[2] = rot;
                }
                __syncthreads();  // rotation visible; red free for the next pair
                const double c = rot_s[0], s = rot_s[1];
                const bool do_rot = rot_s[2] != 0.0;
                __syncthreads();  // rot_s is rewritten by the next pair
                if (!do_rot) continue;
                if (threadIdx.x == 0) local_rot++;
                for (int i = threadIdx.x; i < p.nr; i += NT) {
                    const double u = __ldcg(xp + i), v = __ldcg(xq + i);
                    __stcg(xp + i, c * u - s * v);
                    __stcg(xq + i, s * u + c * v);
                }
                double *jp = p.J + (i64)P * p.ldj;
                double *jq = p.J + (i64)Q * p.ldj;
                for (int i = threadIdx.x; i < p.nc; i += NT) {
                    const double u = __ldcg(jp + i), v = __ldcg(jq + i);
                    __stcg(jp + i, c * u - s * v);
                    __stcg(jq + i, s * u + c * v);
                }
            }
            if (t == rounds - 1 && threadIdx.x == 0 && local_rot != 0) {
                atomicAdd(p.rot + sweep, local_rot);
                local_rot = 0;
            }
            if (!grid_barrier(bar_count, epoch, &p.st->err)) return;
        }
        if (ld_acquire(p.rot + sweep) == 0) {
            done = sweep + 1;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) p.st->sweeps[p.which] = done;
}

// ------------------------------------------------------------------
// Gram-form Jacobi for the symmetric eigenproblems (Gram matrices).
//
// B (n x n, row-major, symmetric) is the Gram matrix of an implicit X; the
// rotation of pair (P,Q) orthogonalises columns P and Q of X and is
// computed from b_PP, b_QQ, b_PQ alone.  A round of the circle schedule
// applies all n/2 rotations at once as B <- J^T B J:
//   phase A: the CTA of each pair computes (c, s, t) from its own 2 x 2
//            block and publishes them;            -- grid barrier --
//   phase B: the CTA of pair (P,Q) rewrites rows P and Q of B (each
//            2 x 2 block B[{P,Q},{K,K'}] becomes G_PQ^T B G_KK') and
//            columns P and Q of V;                 -- grid barrier --
// Rows P and Q of the new B depend only on rows P and Q of the old B, so
// the update is in place and race-free.
struct EigArgs {
    double *B;
    i64 ldb;
    double *V;  // column-major n x n
    i64 ldv;
    double4 *prm;  // [npairs] (c, s, t, rotate)
    int n, npad;
    int max_sweeps;
    double tol;
    int *rot;
    DevStatus *st;
    int which;
};

__device__ __forceinline__ double4 ld4cg(const double4 *p)
{
    const double2 a = __ldcg((const double2 *)p), b = __ldcg((const double2 *)p + 1);
    return make_double4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ void st4cg(double4 *p, double4 v)
{
    __stcg((double2 *)p, make_double2(v.x, v.y));
    __stcg((double2 *)p + 1, make_double2(v.z, v.w));
}

__device__ __forceinline__ void circle_pair(int pr, int t, int npad, int &P, int &Q)
{
    const int rounds = npad - 1;
    const int a = pr, b = npad - 1 - pr;
    P = (a == 0) ? 0 : 1 + (a - 1 + t) % rounds;
    Q = (b == 0) ? 0 : 1 + (b - 1 + t) % rounds;
    if (P > Q) {
        int tmp = P;
        P = Q;
        Q = tmp;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) jacobi_eig_kernel(EigArgs p)
{
    const int npairs = p.npad / 2;
    const int rounds = p.npad - 1;
    const int n = p.n;
    int local_rot = 0;
    int done = -1;
    unsigned long long *bar_count = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0;
    for (int sweep = 0; sweep < p.max_sweeps; sweep++) {
        for (int t = 0; t < rounds; t++) {
            // ---- phase A: rotation of each pair from its 2 x 2 block
            if (threadIdx.x == 0) {
                for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
                    int P, Q;
                    circle_pair(pr, t, p.npad, P, Q);
                    double4 r = make_double4(1.0, 0.0, 0.0, 0.0);
                    if (Q < n) {
                        const double a = __ldcg(p.B + (i64)P * p.ldb + P);
                        const double b = __ldcg(p.B + (i64)Q * p.ldb + Q);
                        const double g = __ldcg(p.B + (i64)P * p.ldb + Q);
                        if (g != 0.0 && fabs(g) > p.tol * sqrt(fabs(a * b))) {
                            const double zeta = (b - a) / (2.0 * g);
                            double tt;
                            if (fabs(zeta) > 1e150)
                                tt = 0.5 / zeta;
                            else
                                tt = (zeta >= 0.0 ? 1.0 : -1.0) /
                                     (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                            const double c = 1.0 / sqrt(1.0 + tt * tt);
                            r = make_double4(c, c * tt, tt, 1.0);
                            local_rot++;
                        }
                    }
                    st4cg(p.prm + pr, r);
                }
            }
            if (t == rounds - 1 && threadIdx.x == 0 && local_rot != 0) {
                atomicAdd(p.rot + sweep, local_rot);
                local_rot = 0;
            }
            if (!grid_barrier(bar_count, epoch, &p.st->err)) return;
            // ---- phase B: rows P, Q of J^T B J and columns P, Q of V J
            for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
                int P, Q;
                circle_pair(pr, t, p.npad, P, Q);
                const double4 me = ld4cg(p.prm + pr);
                const bool hasQ = Q < n;
                double *rP = p.B + (i64)P * p.ldb;
                double *rQ = hasQ ? p.B + (i64)Q * p.ldb : nullptr;
                const double c = me.x, s = me.y;
                for (int k = threadIdx.x; k < npairs; k += NT) {
                    int K, K2;
                    circle_pair(k, t, p.npad, K, K2);
                    const bool hasK2 = K2 < n;
                    if (k == pr) {
                        if (me.w != 0.0) {
                            const double a = __ldcg(rP + P), b = __ldcg(rQ + Q);
                            const double g = __ldcg(rP + Q);
                            __stcg(rP + P, a - me.z * g);
                            __stcg(rQ + Q, b + me.z * g);
                            __stcg(rP + Q, 0.0);
                            __stcg(rQ + P, 0.0);
                        }
                        continue;
                    }
                    const double4 o = ld4cg(p.prm + k);
                    double x = __ldcg(rP + K), y = hasK2 ? __ldcg(rP + K2) : 0.0;
                    double z = hasQ ? __ldcg(rQ + K) : 0.0;
                    double w = (hasQ && hasK2) ? __ldcg(rQ + K2) : 0.0;
                    // rows (own rotation), then columns (the other pair's)
                    const double x1 = c * x - s * z, y1 = c * y - s * w;
                    const double z1 = s * x + c * z, w1 = s * y + c * w;
                    const double ck = o.x, sk = o.y;
                    __stcg(rP + K, ck * x1 - sk * y1);
                    if (hasK2) __stcg(rP + K2, sk * x1 + ck * y1);
                    if (hasQ) {
                        __stcg(rQ + K, ck * z1 - sk * w1);
                        if (hasK2) __stcg(rQ + K2, sk * z1 + ck * w1);
                    }
                }
                if (me.w != 0.0) {
                    double *vp = p.V + (i64)P * p.ldv;
                    double *vq = p.V + (i64)Q * p.ldv;
                    for (int i = threadIdx.x; i < n; i += NT) {
                        const double u = __ldcg(vp + i), v = __ldcg(vq + i);
                        __stcg(vp + i, c * u - s * v);
                        __stcg(vq + i, s * u + c * v);
                    }
                }
            }
            if (!grid_barrier(bar_count, epoch, &p.st->err)) return;
        }
        if (ld_acquire(p.rot + sweep) == 0) {
            done = sweep + 1;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) p.st->sweeps[p.which] = done;
}

__global__ void diag_kernel(const double *B, i64 ldb, int n, double *d)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) d[j] = B[(i64)j * ldb + j];
}

__global__ void init_identity_kernel(double *J, i64 ldj, int nc)
{
    const i64 total = (i64)nc * nc;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        const i64 c = e / nc, r = e % nc;
        J[c * ldj + r] = (r == c) ? 1.0 : 0.0;
    }
}

// One warp per column: norm of column j of the column-major X.
__global__ void colnorm_cm_kernel(const double *X, i64 ldx, int nr, int nc, double *norms)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nc) return;
    const double *x = X + (i64)warp * ldx;
    double s = 0.0;
    for (int i = lane; i < nr; i += 32) s = fma(x[i], x[i], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (lane == 0) norms[warp] = sqrt(s);
}

// perm[rank] = j with rank = #{i : n_i > n_j or (n_i == n_j and i < j)}:
// a stable sort into decreasing order.
__global__ void rank_sort_kernel(const double *norms, int nc, int *perm)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nc; j += gridDim.x * blockDim.x) {
        // NaN sorts last (norms are otherwise >= 0), so the order is total
        // and perm is a permutation.
        const double v = isnan(norms[j]) ? -1.0 : norms[j];
        int r = 0;
        for (int i = 0; i < nc; i++) {
            const double w = isnan(norms[i]) ? -1.0 : norms[i];
            r += (w > v) || (w == v && i < j);
        }
        perm[r] = j;
    }
}

__global__ void permute_out_kernel(const double *X, i64 ldx, const double *J, i64 ldj, int nr,
                                   int nc, const double *norms, const int *perm, double *Jout,
                                   i64 ldjo, double *lam, double *Xout, i64 ldxo)
{
    const i64 tj = (i64)nc * nc;
    const i64 tx = Xout ? (i64)nr * nc : 0;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < tj + tx;
         e += (i64)gridDim.x * blockDim.x) {
        if (e < tj) {
            const i64 i = e / nc, r = e % nc;  // row i, output column r
            int src = perm[r];
            if (src < 0 || src >= nc) src = (int)r;
            Jout[i * ldjo + r] = J[(i64)src * ldj + i];
            if (i == 0 && lam) lam[r] = norms[src];
        } else {
            const i64 f = e - tj;
            const i64 i = f / nc, r = f % nc;
            int src = perm[r];
            if (src < 0 || src >= nc) src = (int)r;
            const double s = norms[src];
            Xout[i * ldxo + r] = (s > 0.0) ? X[(i64)src * ldx + i] / s : 0.0;
        }
    }
}

}  // namespace

cudaError_t launch_jacobi(double *X, i64 ldx, double *J, i64 ldj, int nr, int nc, int max_sweeps,
                          int *ctr, DevStatus *st, int which, cudaStream_t s)
{
    cudaError_t e;
    {
        i64 total = (i64)nc * nc;
        i64 blocks = (total + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        if (blocks < 1) blocks = 1;
        ProfScope ps_("init_identity", s);
        init_identity_kernel<<<(unsigned)blocks, 256, 0, s>>>(J, ldj, nc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(int) * (size_t)(max_sweeps + 4), s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(&st->bar[0], 0, sizeof(int) * 4, s)) != cudaSuccess) return e;
    if (nc < 2) {
        // nothing to rotate: a single column is already "orthogonal"
        return cudaMemsetAsync(&st->sweeps[which], 0, sizeof(int), s);
    }

    JacobiArgs a;
    a.X = X;
    a.ldx = ldx;
    a.J = J;
    a.ldj = ldj;
    a.nr = nr;
    a.nc = nc;
    a.npad = nc + (nc & 1);
    a.max_sweeps = max_sweeps;
    a.tol = (double)nr * 0x1p-53;
    a.rot = ctr;
    a.st = st;
    a.which = which;

    constexpr int NT = 128;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel<NT>, NT, 0)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int npairs = a.npad / 2;
    int blocks = num_sms() * per_sm;
    if (blocks > npairs) blocks = npairs;
    void *args[] = {&a};
    ProfScope ps_("jacobi_svd", s);
    return cudaLaunchCooperativeKernel((const void *)jacobi_kernel<NT>, dim3(blocks), dim3(NT),
                                       args, 0, s);
}

cudaError_t launch_jacobi_eig(double *B, i64 ldb, double *V, i64 ldv, double *lam, double *Vout,
                              i64 ldvo, int n, int max_sweeps, int *ctr, double *prm,
                              int *perm, DevStatus *st, int which, cudaStream_t s)
{
    cudaError_t e;
    {
        i64 total = (i64)n * n;
        i64 blocks = (total + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        if (blocks < 1) blocks = 1;
        ProfScope ps_("init_identity", s);
        init_identity_kernel<<<(unsigned)blocks, 256, 0, s>>>(V, ldv, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemsetAsync(ctr, 0, sizeof(int) * (size_t)(max_sweeps + 4), s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(&st->bar[0], 0, sizeof(int) * 4, s)) != cudaSuccess) return e;
    if (n >= 2) {
        EigArgs a;
        a.B = B;
        a.ldb = ldb;
        a.V = V;
        a.ldv = ldv;
        a.prm = (double4 *)prm;
        a.n = n;
        a.npad = n + (n & 1);
        a.max_sweeps = max_sweeps;
        a.tol = (double)n * 0x1p-53;
        a.rot = ctr;
        a.st = st;
        a.which = which;
        constexpr int NT = 128;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_eig_kernel<NT>, NT,
                                                                0)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        int npairs = a.npad / 2;
        int blocks = num_sms() * per_sm;
        if (blocks > npairs) blocks = npairs;
        void *args[] = {&a};
        ProfScope ps_("jacobi_eig", s);
        if ((e = cudaLaunchCooperativeKernel((const void *)jacobi_eig_kernel<NT>, dim3(blocks),
                                             dim3(NT), args, 0, s)) != cudaSuccess)
            return e;
    } else {
        if ((e = cudaMemsetAsync(&st->sweeps[which], 0, sizeof(int), s)) != cudaSuccess) return e;
    }
    // the rotation-parameter scratch (>= 2n doubles) now holds the diagonal
    double *dg = prm;
    {
    ProfScope ps_("diag", s);
    diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(B, ldb, n, dg);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
    ProfScope ps_("rank_sort", s);
    rank_sort_kernel<<<(n + 255) / 256, 256, 0, s>>>(dg, n, perm);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        i64 total = (i64)n * n;
        i64 blocks = (total + 255) / 256;
        if (blocks > (i64)num_sms() * 8) blocks = (i64)num_sms() * 8;
        if (blocks < 1) blocks = 1;
        ProfScope ps_("permute", s);
        permute_out_kernel<<<(unsigned)blocks, 256, 0, s>>>(nullptr, 0, V, ldv, 0, n, dg, perm,
                                                            Vout, ldvo, lam, nullptr, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_jacobi_finalize(const double *X, i64 ldx, const double *J, i64 ldj, int nr,
                                   int nc, double *norms, int *perm, double *Jout, i64 ldjo,
                                   double *lam, double *Xout, i64 ldxo, cudaStream_t s)
{
    cudaError_t e;
    {
        const int warps_per_block = 8;
        const int blocks = (nc + warps_per_block - 1) / warps_per_block;
        ProfScope ps_("colnorm", s);
        colnorm_cm_kernel<<<blocks, 32 * warps_per_block, 0, s>>>(X, ldx, nr, nc, norms);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
    ProfScope ps_("rank_sort", s);
    rank_sort_kernel<<<(nc + 255) / 256, 256, 0, s>>>(norms, nc, perm);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        i64 total = (i64)nc * nc + (Xout ? (i64)nr * nc : 0);
        i64 blocks = (total + 255) / 256;
        if (blocks > (i64)num_sms() * 8) blocks = (i64)num_sms() * 8;
        if (blocks < 1) blocks = 1;
        ProfScope ps_("permute", s);
        permute_out_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, J, ldj, nr, nc, norms, perm,
                                                            Jout, ldjo, lam, Xout, ldxo);
    }
    return cudaGetLastError();
}

}  // namespace tssvd
