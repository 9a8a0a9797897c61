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
#include "jacobi_common.cuh"

namespace tssvd {

namespace {

struct JacobiArgs {
    double *X;
    i64 ldx;
    double *J;
    i64 ldj;
    double4 *prm;  // [2][npairs] published (c, s, 0, rotate) of the last two rounds
    double *nrm;   // [nc] tracked squared column norms (negative: recompute)
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

// Block sum of one per-thread partial (valid in thread 0), as block_sum3.
template <int NT>
__device__ __forceinline__ void block_sum1(double &a, double (*red)[NT / 32])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ta = __shfl_down_sync(0xffffffffu, a, o);
        if (lane < o) a += ta;
    }
    if (lane == 0) red[2][warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        a = red[2][0];
#pragma unroll
        for (int w = 1; w < NT / 32; w++) a += red[2][w];
    }
}

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

// Rows of an accumulated rotation matrix held in shared memory (rows x nc,
// row-major; the CTA's own rows) take all rotations of round t: columns
// K and K' of pair k turn by (c, s) = (prm[k].x, prm[k].y).
__device__ __forceinline__ void rotate_rows_s(double *R, int rows, int nc, const double4 *prm,
                                              int npad, int t)
{
    for (int k = threadIdx.x; k < npad / 2; k += blockDim.x) {
        const double4 o = prm[k];
        if (o.w == 0.0) continue;
        int K, K2;
        circle_pair(k, t, npad, K, K2);
        for (int li = 0; li < rows; li++) {
            const double u = R[li * nc + K], v = R[li * nc + K2];
            R[li * nc + K] = o.x * u - o.y * v;
            R[li * nc + K2] = o.y * u + o.x * v;
        }
    }
}

// One round per grid barrier: the CTA of pair (P,Q) reduces the three inner
// products of columns P and Q of X, and rotates those columns of X and J.
// CH > 0: nr, nc <= CH * NT and each thread keeps its CH entries of the
// four columns in registers (one read per round); CH = 0: no cache.  FP64
// issue is scarce (two lanes per clock per SM), so CH is sized to the
// problem rather than padded.
template <int NT, int CH, bool JS>
__global__ void __launch_bounds__(NT) jacobi_kernel(JacobiArgs p)
{
    constexpr int C = CH > 0 ? CH : 1;
    // Norm tracking saves two of the three inner products per pair; it pays
    // where the FP64 pipe bounds a round (n > 256, CH >= 4 or uncached;
    // n = 1000: 12.8 -> 10.5 us), not where latency does (n <= 256, where
    // this kernel keeps the plain form)
    constexpr bool kTrack = CH == 0 || CH >= 4;
    __shared__ double red[3][NT / 32];
    __shared__ double rot_s[3];
    // JS: this CTA's rows of J (row i for i = blockIdx.x mod gridDim.x) live
    // in shared memory after the round's rotations; the rotations of round
    // t reach them in round t + 1 between arrival and wait.
    extern __shared__ double js_raw[];
    double4 *prev_s = reinterpret_cast<double4 *>(js_raw);
    double *J_s = js_raw + 4 * (size_t)(p.npad / 2);
    const int jrows = JS ? (p.nc - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    if (JS) {
        for (int e = threadIdx.x; e < jrows * p.nc; e += NT) {
            const int li = e / p.nc, c = e % p.nc;
            J_s[e] = (blockIdx.x + li * gridDim.x == c) ? 1.0 : 0.0;
        }
    }
    const int npairs = p.npad / 2;
    const int rounds = p.npad - 1;
    const double tol = p.tol;
    const float log2tol = log2f((float)p.tol);
    const bool hasJ = p.J != nullptr;  // J == null: no accumulation (X_out alone is wanted)
    int local_rot = 0;
    int done = -1;
    unsigned long long *bar_count = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0;
    int gr = 0;  // rounds completed
    for (int sweep = 0; sweep < p.max_sweeps; sweep++) {
        for (int t = 0; t < rounds; t++, gr++) {
            double4 *pub = p.prm + (size_t)(gr & 1) * npairs;
            // the previous round's rotations (for J's rows), loaded after
            // this round's columns and parked in shared memory before the
            // arrival, so that no wait on them sits in the critical path
            const double4 *prev_g = p.prm + (size_t)((gr - 1) & 1) * npairs;
            const bool want_prev = JS && gr > 0 && (int)threadIdx.x < npairs;
            double4 pv = make_double4(1.0, 0.0, 0.0, 0.0);
            bool pv_loaded = false;
            for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
                int P, Q;
                circle_pair(pr, t, p.npad, P, Q);
                if (Q >= p.nc) {  // the padding column of an odd nc
                    if (JS && threadIdx.x == 0) st4cg(pub + pr, make_double4(1.0, 0.0, 0.0, 0.0));
                    continue;
                }
                double *xp = p.X + (i64)P * p.ldx, *xq = p.X + (i64)Q * p.ldx;
                double *jp = hasJ ? p.J + (i64)P * p.ldj : nullptr;
                double *jq = hasJ ? p.J + (i64)Q * p.ldj : nullptr;
                // Squared norms: tracked through the rotations (each rotation
                // gives its two columns' new norms in closed form), so only the
                // inner product is summed; recomputed in the first two rounds
                // of every sweep (every column is in a real pair in one of
                // them, whatever the padding) and after a cancelling update
                // (flag < 0).
                double na = -1.0, nb = -1.0;
                if (kTrack && t >= 2) {
                    na = __ldcg(p.nrm + P);
                    nb = __ldcg(p.nrm + Q);
                }
                const bool need_a = !(na >= 0.0), need_b = !(nb >= 0.0);
                double u[C], v[C], ju[C], jv[C];
                double al = 0.0, be = 0.0, ga = 0.0;
                if (CH > 0) {
#pragma unroll
                    for (int j = 0; j < C; j++) {
                        const int i = threadIdx.x + j * NT;
                        u[j] = i < p.nr ? __ldcg(xp + i) : 0.0;
                        v[j] = i < p.nr ? __ldcg(xq + i) : 0.0;
                        ju[j] = (!JS && hasJ && i < p.nc) ? __ldcg(jp + i) : 0.0;
                        jv[j] = (!JS && hasJ && i < p.nc) ? __ldcg(jq + i) : 0.0;
                    }
                    if (want_prev && !pv_loaded) {
                        pv = ld4cg(prev_g + threadIdx.x);
                        pv_loaded = true;
                    }
                    if (need_a || need_b) {
#pragma unroll
                        for (int j = 0; j < C; j++) {
                            al = fma(u[j], u[j], al);
                            be = fma(v[j], v[j], be);
                            ga = fma(u[j], v[j], ga);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < C; j++) ga = fma(u[j], v[j], ga);
                    }
                } else {
                    for (int i = threadIdx.x; i < p.nr; i += NT) {
                        const double x = __ldcg(xp + i), y = __ldcg(xq + i);
                        al = fma(x, x, al);
                        be = fma(y, y, be);
                        ga = fma(x, y, ga);
                    }
                }
                if (need_a || need_b || CH == 0)
                    block_sum3<NT>(al, be, ga, red);
                else
                    block_sum1<NT>(ga, red);
                if (threadIdx.x == 0) {
                    const double a = (need_a || CH == 0) ? al : na;
                    const double b = (need_b || CH == 0) ? be : nb;
                    const double4 r = jac_rotation(a, b, ga, tol, log2tol);
                    rot_s[0] = r.x;
                    rot_s[1] = r.y;
                    rot_s[2] = r.w;
                    double a1 = a, b1 = b;
                    if (kTrack && r.w != 0.0) {
                        // ||c x_P - s x_Q||^2 and ||s x_P + c x_Q||^2; an update
                        // that cancels below 2^-16 of the inputs is recomputed
                        const double cc = r.x * r.x, ss = r.y * r.y, cs2 = 2.0 * r.x * r.y;
                        a1 = fma(cc, a, fma(-cs2, ga, ss * b));
                        b1 = fma(ss, a, fma(cs2, ga, cc * b));
                        const double floor = 0x1p-16 * (a + b);
                        if (!(a1 >= floor)) a1 = -1.0;
                        if (!(b1 >= floor)) b1 = -1.0;
                    }
                    if (kTrack && (r.w != 0.0 || need_a || need_b)) {
                        __stcg(p.nrm + P, a1);
                        __stcg(p.nrm + Q, b1);
                    }
                }
                __syncthreads();  // rotation visible; red free for the next pair
                const double c = rot_s[0], sn = rot_s[1];
                const bool do_rot = rot_s[2] != 0.0;
                __syncthreads();  // rot_s is rewritten by the next pair
                if (JS && threadIdx.x == 0)
                    st4cg(pub + pr, make_double4(c, sn, 0.0, do_rot ? 1.0 : 0.0));
                if (!do_rot) continue;
                if (threadIdx.x == 0) local_rot++;
                if (CH > 0) {
#pragma unroll
                    for (int j = 0; j < C; j++) {
                        const int i = threadIdx.x + j * NT;
                        if (i < p.nr) {
                            __stcg(xp + i, c * u[j] - sn * v[j]);
                            __stcg(xq + i, sn * u[j] + c * v[j]);
                        }
                        if (!JS && hasJ && i < p.nc) {
                            __stcg(jp + i, c * ju[j] - sn * jv[j]);
                            __stcg(jq + i, sn * ju[j] + c * jv[j]);
                        }
                    }
                } else {
                    for (int i = threadIdx.x; i < p.nr; i += NT) {
                        const double x = __ldcg(xp + i), y = __ldcg(xq + i);
                        __stcg(xp + i, c * x - sn * y);
                        __stcg(xq + i, sn * x + c * y);
                    }
                    if (!JS && hasJ)
                        for (int i = threadIdx.x; i < p.nc; i += NT) {
                            const double x = __ldcg(jp + i), y = __ldcg(jq + i);
                            __stcg(jp + i, c * x - sn * y);
                            __stcg(jq + i, sn * x + c * y);
                        }
                }
            }
            if (t == rounds - 1 && threadIdx.x == 0 && local_rot != 0) {
                atomicAdd(p.rot + sweep, local_rot);
                local_rot = 0;
            }
            if (want_prev) prev_s[threadIdx.x] = pv_loaded ? pv : ld4cg(prev_g + threadIdx.x);
            if (JS && gr > 0)
                for (int k = threadIdx.x + NT; k < npairs; k += NT) prev_s[k] = ld4cg(prev_g + k);
            grid_arrive(bar_count, epoch);
            if (JS && gr > 0) rotate_rows_s(J_s, jrows, p.nc, prev_s, p.npad, (t + rounds - 1) % rounds);
            if (!grid_wait(bar_count, epoch, &p.st->err)) return;
        }
        if (ld_acquire(p.rot + sweep) == 0) {
            done = sweep + 1;
            break;
        }
    }
    if (JS) {
        // the last round's rotations, then J's rows to global memory
        if (gr > 0) {
            for (int k = threadIdx.x; k < npairs; k += NT)
                prev_s[k] = ld4cg(p.prm + (size_t)((gr - 1) & 1) * npairs + k);
            __syncthreads();
            rotate_rows_s(J_s, jrows, p.nc, prev_s, p.npad, rounds - 1);
            __syncthreads();
        }
        for (int e = threadIdx.x; e < jrows * p.nc; e += NT) {
            const int li = e / p.nc, c = e % p.nc;
            p.J[(i64)c * p.ldj + blockIdx.x + li * gridDim.x] = J_s[e];
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
    double *B2;  // second copy of B (single-barrier form)
    i64 ldb;
    double *V;  // column-major n x n
    i64 ldv;
    double4 *prm;  // [npairs] (c, s, t, rotate)
    double *diag;  // [n] diagonal of the final B (single-barrier form)
    int n, npad;
    int normwise;  // 1: rotate only when also |b_PQ| > 2^-52 max_k b_kk
    int max_sweeps;
    double tol;
    int *rot;
    DevStatus *st;
    int which;
};

// Gram-form Jacobi with one grid barrier per round (npad <= 2 * kEigSmemPairs).
// B is double-buffered: round t reads Bc and writes every entry of Bn, so a
// CTA may start round t + 1 while others still read Bc.  Every CTA derives
// all n/2 rotations of the round from Bc's 2 x 2 diagonal blocks (the same
// arithmetic on the same values, so all CTAs agree bit for bit) into shared
// memory; the CTA of pair (P,Q) then writes rows P and Q of J^T B J into Bn.
// V's rotations are applied by rows (see VS) or, for large n, to columns P
// and Q by the pair's CTA.
// Block {pr, pr + d mod npairs} of the symmetric B is formed by pair pr
// when 1 <= d <= npairs / 2, except that for an even count the opposite
// pair (d = npairs / 2) is taken by the smaller index only: every unordered
// pair of pairs exactly once.
__device__ __forceinline__ bool block_mine(int pr, int d, int npairs)
{
    if (d < 1 || d > npairs / 2) return false;
    if (2 * d == npairs) return pr < d;
    return true;
}

constexpr int kEigSmemPairs = 1024;
// Largest shared-memory footprint for rotation rows held by a CTA.
constexpr size_t kRowsSmemMax = 96 * 1024;

template <int NT, bool VS>
__global__ void __launch_bounds__(NT) jacobi_eig1_kernel(EigArgs p)
{
    extern __shared__ double4 prm_s[];
    const int npairs = p.npad / 2;
    const int rounds = p.npad - 1;
    const int n = p.n;
    const i64 ldb = p.ldb, ldv = p.ldv;
    // VS: this CTA's rows of V (row i for i = blockIdx.x mod gridDim.x) live
    // in shared memory and take each round's rotations while the barrier
    // completes; they are written out at the end.
    double *V_s = reinterpret_cast<double *>(prm_s + npairs);
    const int vrows = VS ? (n - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    if (VS) {
        for (int e = threadIdx.x; e < vrows * n; e += NT) {
            const int li = e / n, c = e % n;
            V_s[e] = (blockIdx.x + li * gridDim.x == c) ? 1.0 : 0.0;
        }
    }
    int done = -1;
    unsigned long long *bar_count = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0;
    const double *Bc = p.B;
    double *Bn = p.B2;
    const int tid = threadIdx.x;
    const float log2tol = log2f((float)p.tol);
    // Normwise floor: one unit of FP64 rounding (2^-52) of the largest
    // diagonal entry, the level below which B's entries carry no
    // information (they were formed with rounding errors of at least that
    // size).  Taken from the diagonals every CTA loads as rotation inputs
    // (the same values in every CTA, so all agree on the floor), refreshed
    // once per sweep.
    __shared__ double dmax_s[NT / 32];
    double dmx = 0.0, gmin = 0.0;
    if (p.normwise) {
        for (int i = tid; i < n; i += NT) dmx = fmax(dmx, __ldcg(Bc + (i64)i * ldb + i));
    }
    for (int sweep = 0; sweep < p.max_sweeps; sweep++) {
        if (p.normwise) {
            for (int o = 16; o > 0; o >>= 1) dmx = fmax(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
            if ((tid & 31) == 0) dmax_s[tid >> 5] = dmx;
            __syncthreads();
            double m = 0.0;
            for (int w = 0; w < NT / 32; w++) m = fmax(m, dmax_s[w]);
            gmin = 0x1p-52 * m;
            dmx = 0.0;
            __syncthreads();  // dmax_s is rewritten next sweep
        }
        int sweep_rot = 0;
        for (int t = 0; t < rounds; t++) {
            // ---- issue the loads first: the 2 x 2 block of pair k = tid
            // (for the rotations) and the first off-diagonal block this
            // thread updates, so both wait on memory together
            int K0 = 0, K20 = 0;
            double a0 = 0.0, b0 = 0.0, g0 = 0.0;
            if (tid < npairs) {
                circle_pair(tid, t, p.npad, K0, K20);
                if (K20 < n) {
                    a0 = __ldcg(Bc + (i64)K0 * ldb + K0);
                    b0 = __ldcg(Bc + (i64)K20 * ldb + K20);
                    g0 = __ldcg(Bc + (i64)K0 * ldb + K20);
                }
            }
            const int pr0 = blockIdx.x;
            int P0, Q0;
            circle_pair(pr0, t, p.npad, P0, Q0);
            int k0 = pr0 + 1 + tid;
            if (k0 >= npairs) k0 -= npairs;
            const bool pf = block_mine(pr0, 1 + tid, npairs);
            int KB0 = 0, KB20 = 0;
            double x0 = 0.0, y0 = 0.0, z0 = 0.0, w0 = 0.0;
            if (pf) {
                circle_pair(k0, t, p.npad, KB0, KB20);
                const double *cP = Bc + (i64)P0 * ldb, *cQ = Bc + (i64)Q0 * ldb;
                x0 = __ldcg(cP + KB0);
                if (KB20 < n) y0 = __ldcg(cP + KB20);
                if (Q0 < n) {
                    z0 = __ldcg(cQ + KB0);
                    if (KB20 < n) w0 = __ldcg(cQ + KB20);
                }
            }
            // ---- all rotations of the round
            int rot_here = 0;
            if (tid < npairs) {
                double4 r = make_double4(1.0, 0.0, 0.0, 0.0);
                if (K20 < n) {
                    r = jac_rotation(a0, b0, g0, p.tol, log2tol, gmin);
                    rot_here |= r.w != 0.0;
                    if (t == rounds - 1) dmx = fmax(dmx, fmax(a0, b0));
                }
                prm_s[tid] = r;
            }
            for (int k = tid + NT; k < npairs; k += NT) {
                int K, K2;
                circle_pair(k, t, p.npad, K, K2);
                double4 r = make_double4(1.0, 0.0, 0.0, 0.0);
                if (K2 < n) {
                    const double a = __ldcg(Bc + (i64)K * ldb + K);
                    const double b = __ldcg(Bc + (i64)K2 * ldb + K2);
                    const double g = __ldcg(Bc + (i64)K * ldb + K2);
                    r = jac_rotation(a, b, g, p.tol, log2tol, gmin);
                    rot_here |= r.w != 0.0;
                    if (t == rounds - 1) dmx = fmax(dmx, fmax(a, b));
                }
                prm_s[k] = r;
            }
            // A round in which no pair rotates leaves B and V as they are:
            // every CTA sees the same rotations, so all skip its update and
            // its barrier together (Bc stays the current copy).
            if (!__syncthreads_or(rot_here)) continue;
            sweep_rot = 1;
            for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
                const bool first = pr == pr0;
                int P, Q;
                circle_pair(pr, t, p.npad, P, Q);
                const double4 me = prm_s[pr];
                const bool hasQ = Q < n;
                const double c = me.x, s = me.y;
                // ---- columns P and Q of V J (when V is not held by rows)
                if (!VS && hasQ && me.w != 0.0) {
                    double *vp = p.V + (i64)P * ldv, *vq = p.V + (i64)Q * ldv;
                    for (int i = tid; i < n; i += NT) {
                        const double u = __ldcg(vp + i), v = __ldcg(vq + i);
                        __stcg(vp + i, c * u - s * v);
                        __stcg(vq + i, s * u + c * v);
                    }
                }
                const double *cP = Bc + (i64)P * ldb;
                const double *cQ = hasQ ? Bc + (i64)Q * ldb : nullptr;
                double *nP = Bn + (i64)P * ldb;
                double *nQ = hasQ ? Bn + (i64)Q * ldb : nullptr;
                // ---- the pair's own 2 x 2 block G^T [a g; g b] G, by the
                // thread that loaded it as rotation input (pair index mod NT)
                if (tid == pr % NT) {
                    double a, b = 0.0, g = 0.0;
                    if (first && pr < NT && K20 < n) {
                        a = a0;
                        b = b0;
                        g = g0;
                    } else {
                        a = __ldcg(cP + P);
                        if (hasQ) {
                            b = __ldcg(cQ + Q);
                            g = __ldcg(cP + Q);
                        }
                    }
                    if (hasQ) {
                        if (me.w != 0.0) {
                            const double cc = c * c, ss = s * s, cs = c * s;
                            const double a1 = fma(cc, a, fma(-2.0 * cs, g, ss * b));
                            const double b1 = fma(ss, a, fma(2.0 * cs, g, cc * b));
                            const double g1 = fma(cs, a - b, (cc - ss) * g);
                            __stcg(nP + P, a1);
                            __stcg(nQ + Q, b1);
                            __stcg(nP + Q, g1);
                            __stcg(nQ + P, g1);
                        } else {
                            __stcg(nP + P, a);
                            __stcg(nQ + Q, b);
                            __stcg(nP + Q, g);
                            __stcg(nQ + P, g);
                        }
                    } else {
                        __stcg(nP + P, a);
                    }
                }
                // ---- off-diagonal blocks of rows P, Q: B is symmetric, so
                // each block {pr, k} is formed once, by the CTA for which k
                // lies in the next half of the pair circle, and written
                // together with its transpose (rows K, K' of the new B)
                for (int d = 1 + tid; d <= npairs / 2; d += NT) {
                    if (!block_mine(pr, d, npairs)) continue;
                    int k = pr + d;
                    if (k >= npairs) k -= npairs;
                    int K, K2;
                    double x, y, z, w;
                    if (first && d == 1 + tid) {
                        K = KB0;
                        K2 = KB20;
                        x = x0;
                        y = y0;
                        z = z0;
                        w = w0;
                    } else {
                        circle_pair(k, t, p.npad, K, K2);
                        x = __ldcg(cP + K);
                        y = K2 < n ? __ldcg(cP + K2) : 0.0;
                        z = hasQ ? __ldcg(cQ + K) : 0.0;
                        w = (hasQ && K2 < n) ? __ldcg(cQ + K2) : 0.0;
                    }
                    const bool hasK2 = K2 < n;
                    const double4 o = prm_s[k];
                    // rows (own rotation), then columns (the other pair's)
                    const double x1 = c * x - s * z, y1 = c * y - s * w;
                    const double z1 = s * x + c * z, w1 = s * y + c * w;
                    const double ck = o.x, sk = o.y;
                    const double pk = ck * x1 - sk * y1, pk2 = sk * x1 + ck * y1;
                    __stcg(nP + K, pk);
                    __stcg(Bn + (i64)K * ldb + P, pk);
                    if (hasK2) {
                        __stcg(nP + K2, pk2);
                        __stcg(Bn + (i64)K2 * ldb + P, pk2);
                    }
                    if (hasQ) {
                        const double qk = ck * z1 - sk * w1, qk2 = sk * z1 + ck * w1;
                        __stcg(nQ + K, qk);
                        __stcg(Bn + (i64)K * ldb + Q, qk);
                        if (hasK2) {
                            __stcg(nQ + K2, qk2);
                            __stcg(Bn + (i64)K2 * ldb + Q, qk2);
                        }
                    }
                }
            }
            grid_arrive(bar_count, epoch);
            if (VS) rotate_rows_s(V_s, vrows, n, prm_s, p.npad, t);
            if (!grid_wait(bar_count, epoch, &p.st->err)) return;
            double *tmp = Bn;
            Bn = const_cast<double *>(Bc);
            Bc = tmp;
        }
        if (!sweep_rot) {
            done = sweep + 1;
            break;
        }
    }
    if (VS) {
        for (int e = tid; e < vrows * n; e += NT) {
            const int li = e / n, c = e % n;
            p.V[(i64)c * ldv + blockIdx.x + li * gridDim.x] = V_s[e];
        }
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < n; i += NT) p.diag[i] = __ldcg(Bc + (i64)i * ldb + i);
        if (tid == 0) p.st->sweeps[p.which] = done;
    }
}

// Circle-schedule inverse: the pair index that holds column i in round t.
__device__ __forceinline__ int circle_slot(int i, int t, int npad)
{
    const int rounds = npad - 1;
    int pos = 0;
    if (i != 0) {
        int x = i - 1 - t;
        if (x < 0) x += rounds;
        pos = x + 1;
    }
    return pos < npad / 2 ? pos : npad - 1 - pos;
}

// Column i of a round's rotation matrix J restricted to its pair (ra, rb):
// J e_i = ua e_ra + ub e_rb (ra < rb; rb may be the padding column).
struct JCol {
    int ra, rb;
    double ua, ub;
};

__device__ __forceinline__ JCol jcol_idx(int i, int t, int npad)
{
    JCol u;
    const int pr = circle_slot(i, t, npad);
    circle_pair(pr, t, npad, u.ra, u.rb);
    u.ua = 0.0;
    u.ub = 0.0;
    return u;
}

__device__ __forceinline__ void jcol_coef(JCol &u, int i, double4 r)
{
    // new column P = c e_P - s e_Q, new column Q = s e_P + c e_Q
    if (i == u.ra) {
        u.ua = r.x;
        u.ub = -r.y;
    } else {
        u.ua = r.y;
        u.ub = r.x;
    }
}

// The four entries of the 2 x 2 block B[{ra_i, rb_i}][{ra_j, rb_j}] (zero
// where an index is the padding column).
struct Blk4 {
    double aa, ab, ba, bb;
};

__device__ __forceinline__ Blk4 load_blk4(const double *Bc, i64 ldb, int n, const JCol &ri,
                                          const JCol &cj)
{
    Blk4 m;
    const double *ra = Bc + (i64)ri.ra * ldb;
    m.aa = __ldcg(ra + cj.ra);
    m.ab = cj.rb < n ? __ldcg(ra + cj.rb) : 0.0;
    if (ri.rb < n) {
        const double *rb = Bc + (i64)ri.rb * ldb;
        m.ba = __ldcg(rb + cj.ra);
        m.bb = cj.rb < n ? __ldcg(rb + cj.rb) : 0.0;
    } else {
        m.ba = 0.0;
        m.bb = 0.0;
    }
    return m;
}

// u_i^T M u_j: entry (i, j) of J^T B J from the 2 x 2 block M.
__device__ __forceinline__ double bilin(const JCol &ui, const Blk4 &m, const JCol &uj)
{
    const double ta = fma(m.ab, uj.ub, m.aa * uj.ua);
    const double tb = fma(m.bb, uj.ub, m.ba * uj.ua);
    return fma(ui.ub, tb, ui.ua * ta);
}

// Two rounds of the circle schedule per grid barrier (V held by rows in
// shared memory).  With J = J_t J_t2 (rounds t and t2 = t + 1), every entry
// of J^T B J depends on one 2 x 2 block of B in each of round t's pairs of
// its row and column indices, so both rounds are formed from the current
// copy Bc alone:
//  - round t's rotations from Bc's diagonal 2 x 2 blocks (as one round);
//  - round t2's rotation inputs (B'[P][P], B'[Q][Q], B'[P][Q] of
//    B' = J_t^T B J_t) from those blocks and one more 2 x 2 block per pair;
//  - rows P, Q of J^T B J for the CTA's round-t2 pair from 4 x 4 blocks of
//    Bc (16 loads and 40 FP64 operations per output 2 x 2 block, against
//    two rounds of 4 loads and 16 operations).
// All loads depend only on the schedule and are issued before any rotation
// is known.  For an odd round count the last round is taken alone by
// letting round t2 repeat round t's pairing with identity rotations.
template <int NT>
__global__ void __launch_bounds__(NT) jacobi_eig2r_kernel(EigArgs p)
{
    extern __shared__ double4 prm_s[];  // [npairs] round t, then [npairs] round t2
    const int npairs = p.npad / 2;
    const int rounds = p.npad - 1;
    const int n = p.n, npad = p.npad;
    const i64 ldb = p.ldb, ldv = p.ldv;
    double4 *prm2_s = prm_s + npairs;
    double *d1_s = reinterpret_cast<double *>(prm_s + 2 * npairs);  // [npad] diag of B'
    double *g1_s = d1_s + npad;                                     // [npairs] B'[P2][Q2]
    double *V_s = g1_s + npairs;
    const int vrows = (n - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int tid = threadIdx.x;
    for (int e = tid; e < vrows * n; e += NT) {
        const int li = e / n, c = e % n;
        V_s[e] = (blockIdx.x + li * gridDim.x == c) ? 1.0 : 0.0;
    }
    int done = -1;
    unsigned long long *bar_count = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0;
    const double *Bc = p.B;
    double *Bn = p.B2;
    const float log2tol = log2f((float)p.tol);
    __shared__ double dmax_s[NT / 32];
    double dmx = 0.0, gmin = 0.0;
    if (p.normwise) {
        for (int i = tid; i < n; i += NT) dmx = fmax(dmx, __ldcg(Bc + (i64)i * ldb + i));
    }
    for (int sweep = 0; sweep < p.max_sweeps; sweep++) {
        if (p.normwise) {
            for (int o = 16; o > 0; o >>= 1) dmx = fmax(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
            if ((tid & 31) == 0) dmax_s[tid >> 5] = dmx;
            __syncthreads();
            double m = 0.0;
            for (int w = 0; w < NT / 32; w++) m = fmax(m, dmax_s[w]);
            gmin = 0x1p-52 * m;
            dmx = 0.0;
            __syncthreads();
        }
        int sweep_rot = 0;
        for (int t = 0; t < rounds; t += 2) {
            const bool has2 = t + 1 < rounds;
            const int t2 = has2 ? t + 1 : t;
            const bool last_t = t == rounds - 1, last_t2 = has2 && t2 == rounds - 1;
            // ---- loads: round t's 2 x 2 block of pair tid, round t2's cross
            // block of pair tid, and the first output block of this CTA
            int P0 = 0, Q0 = 0;
            double a0 = 0.0, b0 = 0.0, g0 = 0.0;
            JCol xp = {0, 0, 0.0, 0.0}, xq = xp;
            Blk4 xm = {0.0, 0.0, 0.0, 0.0};
            int P1 = 0, Q1 = 0;
            if (tid < npairs) {
                circle_pair(tid, t, npad, P0, Q0);
                a0 = __ldcg(Bc + (i64)P0 * ldb + P0);
                if (Q0 < n) {
                    b0 = __ldcg(Bc + (i64)Q0 * ldb + Q0);
                    g0 = __ldcg(Bc + (i64)P0 * ldb + Q0);
                }
                if (has2) {
                    circle_pair(tid, t2, npad, P1, Q1);
                    if (Q1 < n) {
                        xp = jcol_idx(P1, t, npad);
                        xq = jcol_idx(Q1, t, npad);
                        xm = load_blk4(Bc, ldb, n, xp, xq);
                    }
                }
            }
            const int prB = blockIdx.x;  // one round-t2 pair per CTA (gridDim == npairs)
            int PB, QB;
            circle_pair(prB, t2, npad, PB, QB);
            const bool hasQB = QB < n;
            const JCol up0 = jcol_idx(PB, t, npad);
            const JCol uq0 = hasQB ? jcol_idx(QB, t, npad) : up0;
            const int d0 = 1 + tid;
            const bool pf = block_mine(prB, d0, npairs);
            int KB = 0, K2B = 0;
            JCol uk0 = up0, uk20 = up0;
            Blk4 mpk = {0.0, 0.0, 0.0, 0.0}, mpk2 = mpk, mqk = mpk, mqk2 = mpk;
            if (pf) {
                int k = prB + d0;
                if (k >= npairs) k -= npairs;
                circle_pair(k, t2, npad, KB, K2B);
                uk0 = jcol_idx(KB, t, npad);
                mpk = load_blk4(Bc, ldb, n, up0, uk0);
                if (hasQB) mqk = load_blk4(Bc, ldb, n, uq0, uk0);
                if (K2B < n) {
                    uk20 = jcol_idx(K2B, t, npad);
                    mpk2 = load_blk4(Bc, ldb, n, up0, uk20);
                    if (hasQB) mqk2 = load_blk4(Bc, ldb, n, uq0, uk20);
                }
            }
            // ---- round t: all rotations, and B''s diagonal
            int rot_here = 0;
            for (int k = tid; k < npairs; k += NT) {
                int P = P0, Q = Q0;
                double a = a0, b = b0, g = g0;
                if (k != tid) {
                    circle_pair(k, t, npad, P, Q);
                    a = __ldcg(Bc + (i64)P * ldb + P);
                    b = Q < n ? __ldcg(Bc + (i64)Q * ldb + Q) : 0.0;
                    g = Q < n ? __ldcg(Bc + (i64)P * ldb + Q) : 0.0;
                }
                double4 r = make_double4(1.0, 0.0, 0.0, 0.0);
                if (Q < n) {
                    r = jac_rotation(a, b, g, p.tol, log2tol, gmin);
                    rot_here |= r.w != 0.0;
                    if (last_t) dmx = fmax(dmx, fmax(a, b));
                    double a1 = a, b1 = b, g1 = g;
                    if (r.w != 0.0) {
                        const double c = r.x, s = r.y;
                        const double cc = c * c, ss = s * s, cs = c * s;
                        a1 = fma(cc, a, fma(-2.0 * cs, g, ss * b));
                        b1 = fma(ss, a, fma(2.0 * cs, g, cc * b));
                        g1 = fma(cs, a - b, (cc - ss) * g);
                    }
                    d1_s[P] = a1;
                    d1_s[Q] = b1;
                    if (!has2) g1_s[k] = g1;
                } else {
                    if (last_t) dmx = fmax(dmx, a);
                    d1_s[P] = a;
                }
                prm_s[k] = r;
            }
            __syncthreads();
            // ---- round t2: rotations from B' = J_t^T B J_t
            if (has2) {
                for (int k = tid; k < npairs; k += NT) {
                    int P = P1, Q = Q1;
                    JCol up = xp, uq = xq;
                    Blk4 m = xm;
                    if (k != tid) {
                        circle_pair(k, t2, npad, P, Q);
                        if (Q < n) {
                            up = jcol_idx(P, t, npad);
                            uq = jcol_idx(Q, t, npad);
                            m = load_blk4(Bc, ldb, n, up, uq);
                        }
                    }
                    double4 r = make_double4(1.0, 0.0, 0.0, 0.0);
                    if (Q < n) {
                        jcol_coef(up, P, prm_s[circle_slot(P, t, npad)]);
                        jcol_coef(uq, Q, prm_s[circle_slot(Q, t, npad)]);
                        const double a = d1_s[P], b = d1_s[Q], g = bilin(up, m, uq);
                        g1_s[k] = g;
                        r = jac_rotation(a, b, g, p.tol, log2tol, gmin);
                        rot_here |= r.w != 0.0;
                        if (last_t2) dmx = fmax(dmx, fmax(a, b));
                    } else if (last_t2) {
                        dmx = fmax(dmx, d1_s[P]);
                    }
                    prm2_s[k] = r;
                }
            } else {
                for (int k = tid; k < npairs; k += NT) prm2_s[k] = make_double4(1.0, 0.0, 0.0, 0.0);
            }
            // A double round in which no pair rotates leaves B and V as they
            // are; every CTA sees the same rotations, so all skip together.
            if (!__syncthreads_or(rot_here)) continue;
            sweep_rot = 1;
            // ---- rows PB, QB of J^T B J
            {
                const double4 me = prm2_s[prB];
                const double c = me.x, s = me.y;
                double *nP = Bn + (i64)PB * ldb;
                double *nQ = hasQB ? Bn + (i64)QB * ldb : nullptr;
                // the pair's own 2 x 2 block, by the last thread: with
                // npairs <= 152 it has no off-diagonal block (those go to
                // threads 0 .. npairs/2 - 1), so this work is off their path
                if (tid == NT - 1) {
                    const double a = d1_s[PB];
                    if (hasQB) {
                        const double b = d1_s[QB], g = g1_s[prB];
                        double a1 = a, b1 = b, g1 = g;
                        if (me.w != 0.0) {
                            const double cc = c * c, ss = s * s, cs = c * s;
                            a1 = fma(cc, a, fma(-2.0 * cs, g, ss * b));
                            b1 = fma(ss, a, fma(2.0 * cs, g, cc * b));
                            g1 = fma(cs, a - b, (cc - ss) * g);
                        }
                        __stcg(nP + PB, a1);
                        __stcg(nQ + QB, b1);
                        __stcg(nP + QB, g1);
                        __stcg(nQ + PB, g1);
                    } else {
                        __stcg(nP + PB, a);
                    }
                }
                JCol up = up0, uq = uq0;
                jcol_coef(up, PB, prm_s[circle_slot(PB, t, npad)]);
                if (hasQB) jcol_coef(uq, QB, prm_s[circle_slot(QB, t, npad)]);
                for (int d = d0; d <= npairs / 2; d += NT) {
                    if (!block_mine(prB, d, npairs)) continue;
                    int k = prB + d;
                    if (k >= npairs) k -= npairs;
                    int K, K2;
                    JCol uk, uk2;
                    Blk4 m1, m2, m3, m4;
                    if (d == d0) {
                        K = KB;
                        K2 = K2B;
                        uk = uk0;
                        uk2 = uk20;
                        m1 = mpk;
                        m2 = mpk2;
                        m3 = mqk;
                        m4 = mqk2;
                    } else {
                        circle_pair(k, t2, npad, K, K2);
                        uk = jcol_idx(K, t, npad);
                        uk2 = uk;
                        m1 = load_blk4(Bc, ldb, n, up, uk);
                        m3 = hasQB ? load_blk4(Bc, ldb, n, uq, uk) : m1;
                        if (K2 < n) {
                            uk2 = jcol_idx(K2, t, npad);
                            m2 = load_blk4(Bc, ldb, n, up, uk2);
                            m4 = hasQB ? load_blk4(Bc, ldb, n, uq, uk2) : m2;
                        } else {
                            m2 = m1;
                            m4 = m3;
                        }
                    }
                    const bool hasK2 = K2 < n;
                    jcol_coef(uk, K, prm_s[circle_slot(K, t, npad)]);
                    if (hasK2) jcol_coef(uk2, K2, prm_s[circle_slot(K2, t, npad)]);
                    // B' entries, then round t2's rotations: rows (own), columns (pair k)
                    const double x = bilin(up, m1, uk);
                    const double y = hasK2 ? bilin(up, m2, uk2) : 0.0;
                    const double z = hasQB ? bilin(uq, m3, uk) : 0.0;
                    const double w = (hasQB && hasK2) ? bilin(uq, m4, uk2) : 0.0;
                    const double4 o = prm2_s[k];
                    const double x1 = c * x - s * z, y1 = c * y - s * w;
                    const double z1 = s * x + c * z, w1 = s * y + c * w;
                    const double ck = o.x, sk = o.y;
                    const double pk = ck * x1 - sk * y1, pk2 = sk * x1 + ck * y1;
                    __stcg(nP + K, pk);
                    __stcg(Bn + (i64)K * ldb + PB, pk);
                    if (hasK2) {
                        __stcg(nP + K2, pk2);
                        __stcg(Bn + (i64)K2 * ldb + PB, pk2);
                    }
                    if (hasQB) {
                        const double qk = ck * z1 - sk * w1, qk2 = sk * z1 + ck * w1;
                        __stcg(nQ + K, qk);
                        __stcg(Bn + (i64)K * ldb + QB, qk);
                        if (hasK2) {
                            __stcg(nQ + K2, qk2);
                            __stcg(Bn + (i64)K2 * ldb + QB, qk2);
                        }
                    }
                }
            }
            grid_arrive(bar_count, epoch);
            rotate_rows_s(V_s, vrows, n, prm_s, npad, t);
            if (has2) {
                __syncthreads();
                rotate_rows_s(V_s, vrows, n, prm2_s, npad, t2);
            }
            if (!grid_wait(bar_count, epoch, &p.st->err)) return;
            double *tmp = Bn;
            Bn = const_cast<double *>(Bc);
            Bc = tmp;
        }
        if (!sweep_rot) {
            done = sweep + 1;
            break;
        }
    }
    for (int e = tid; e < vrows * n; e += NT) {
        const int li = e / n, c = e % n;
        p.V[(i64)c * ldv + blockIdx.x + li * gridDim.x] = V_s[e];
    }
    if (blockIdx.x == 0) {
        for (int i = tid; i < n; i += NT) p.diag[i] = __ldcg(Bc + (i64)i * ldb + i);
        if (tid == 0) p.st->sweeps[p.which] = done;
    }
}

// Two-barrier in-place form for npad > 2 * kEigSmemPairs (the rotations
// of a round do not fit in shared memory).
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
                        r = jac_rotation_slow(a, b, g, p.tol);
                        if (r.w != 0.0) local_rot++;
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

// Jout column r = J column perm[r] divided by its norm jnorm[perm[r]]
// (jnorm may be null: no division).  A product of plane rotations has unit
// columns in exact arithmetic; in FP64 each rotation with c = 1/sqrt(1 +
// t^2) and s = c t has c^2 + s^2 = 1 + O(eps) with a positive bias once
// t^2 falls below the rounding unit, so over thousands of rotations a
// column's norm drifts upward (1e-13 at n = 300), and that drift, not the
// convergence test, set the orthonormality of U = Q P.  Dividing by the
// recomputed norms removes it.
__global__ void permute_out_kernel(const double *X, i64 ldx, const double *J, i64 ldj, int nr,
                                   int nc, const double *norms, const int *perm, double *Jout,
                                   i64 ldjo, double *lam, double *Xout, i64 ldxo,
                                   const int *orient, const double *jnorm)
{
    if (orient && Xout && nr == nc && *orient != 0) {
        double *tp = Jout;
        Jout = Xout;
        Xout = tp;
        const i64 tl = ldjo;
        ldjo = ldxo;
        ldxo = tl;
    }
    const i64 tj = J ? (i64)nc * nc : 0;
    const i64 tx = Xout ? (i64)nr * nc : 0;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < tj + tx;
         e += (i64)gridDim.x * blockDim.x) {
        if (e < tj) {
            const i64 i = e / nc, r = e % nc;  // row i, output column r
            int src = perm[r];
            if (src < 0 || src >= nc) src = (int)r;
            const double jn = jnorm ? jnorm[src] : 1.0;
            Jout[i * ldjo + r] = jn > 0.0 ? J[(i64)src * ldj + i] / jn : J[(i64)src * ldj + i];
            if (i == 0 && lam) lam[r] = norms[src];
        } else {
            const i64 f = e - tj;
            const i64 i = f / nc, r = f % nc;
            int src = perm[r];
            if (src < 0 || src >= nc) src = (int)r;
            const double s = norms[src];
            Xout[i * ldxo + r] = (s > 0.0) ? X[(i64)src * ldx + i] / s : 0.0;
            if (i == 0 && lam && !J) lam[r] = s;
        }
    }
}

// Pivoted Cholesky with a floor, one CTA: P^T W P = R^T R with the pivot
// the largest remaining diagonal entry at each step.  Once every remaining
// diagonal entry is <= delta = 2^-52 max_i W_ii (the rounding already in a
// Gram matrix of that size), the trailing block of R is set to sqrt(delta) I
// (W perturbed by at most 2 delta in norm); W = 0 gives R = I.  W (n x n,
// row-major, symmetric) is consumed: rows and columns of its trailing
// block are swapped physically so the rank-one updates stay contiguous.
// Output: X = R^T column-major (X[k ldx + i] = R[k][i]) and piv (logical
// index i is original index piv[i]).
constexpr int kPcholThreads = 1024;

__device__ __forceinline__ void pchol_body(double *__restrict__ W, int n, double *__restrict__ X,
                                           i64 ldx, int *__restrict__ piv)
{
    extern __shared__ double pc_s[];
    double *rk = pc_s;                               // row k of R (n)
    double *rv = rk + n;                             // reduction values (32)
    int *ri = (int *)(rv + 32);                      // reduction indices (32)
    int *pm = ri + 32;                               // permutation (n)
    __shared__ double sdelta, spiv, sinv;
    __shared__ int sj, sstop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = kPcholThreads / 32;
    for (int i = tid; i < n; i += kPcholThreads) pm[i] = i;
    for (i64 e = tid; e < (i64)n * n; e += kPcholThreads) {
        const i64 k = e / n, i = e - k * n;
        X[k * ldx + i] = 0.0;
    }
    // delta = 2^-52 max diag
    {
        double v = 0.0;
        for (int i = tid; i < n; i += kPcholThreads) v = fmax(v, W[(i64)i * n + i]);
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) rv[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nw; w++) t = fmax(t, rv[w]);
            sdelta = 0x1p-52 * t;
        }
        __syncthreads();
    }
    const double delta = sdelta;
    int k = 0;
    for (; k < n; k++) {
        // pivot: the largest remaining diagonal entry (lowest index on ties)
        double bv = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += kPcholThreads) {
            const double v = W[(i64)i * n + i];
            if (v > bv) {
                bv = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            rv[warp] = bv;
            ri[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double t = rv[0];
            int j = ri[0];
            for (int w = 1; w < nw; w++)
                if (rv[w] > t || (rv[w] == t && ri[w] < j)) {
                    t = rv[w];
                    j = ri[w];
                }
            sj = j;
            sstop = (delta > 0.0 && t > delta) ? 0 : 1;
            // (one thread: FP64 sqrt and divide are long FP64-pipe sequences)
            spiv = sstop ? 0.0 : sqrt(t);
            sinv = sstop ? 0.0 : 1.0 / spiv;
        }
        __syncthreads();
        if (sstop) break;
        const int j = sj;
        if (j != k) {
            // swap rows k and j of the trailing block, then columns k and j
            for (int c = k + tid; c < n; c += kPcholThreads) {
                const double a = W[(i64)k * n + c], b = W[(i64)j * n + c];
                W[(i64)k * n + c] = b;
                W[(i64)j * n + c] = a;
            }
            // the finished rows of R: entries at logical columns k and j
            for (int r = tid; r < k; r += kPcholThreads) {
                const double a = X[(i64)r * ldx + k], b = X[(i64)r * ldx + j];
                X[(i64)r * ldx + k] = b;
                X[(i64)r * ldx + j] = a;
            }
            __syncthreads();
            for (int r = k + tid; r < n; r += kPcholThreads) {
                const double a = W[(i64)r * n + k], b = W[(i64)r * n + j];
                W[(i64)r * n + k] = b;
                W[(i64)r * n + j] = a;
            }
            if (tid == 0) {
                const int t = pm[k];
                pm[k] = pm[j];
                pm[j] = t;
            }
            __syncthreads();
        }
        // row k of R
        const double pv = spiv, inv = sinv;
        for (int c = k + tid; c < n; c += kPcholThreads) {
            const double r = (c == k) ? pv : W[(i64)k * n + c] * inv;
            rk[c] = r;
            X[(i64)k * ldx + c] = r;
        }
        __syncthreads();
        // rank-one update of the trailing block (rows and columns > k): a
        // warp per row, each lane's columns loaded together (n <= 256: at
        // most 8 per lane), so a row costs one memory round trip
        for (int i = k + 1 + warp; i < n; i += nw) {
            double *row = W + (i64)i * n;
            const double ri_ = rk[i];
            double w[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int c = k + 1 + lane + 32 * q;
                w[q] = c < n ? row[c] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int c = k + 1 + lane + 32 * q;
                if (c < n) row[c] = fma(-ri_, rk[c], w[q]);
            }
        }
        __syncthreads();
    }
    // the trailing block below the floor (or all of R when W = 0)
    const double tail = delta > 0.0 ? sqrt(delta) : 1.0;
    for (int i = k + tid; i < n; i += kPcholThreads) X[(i64)i * ldx + i] = tail;
    for (int i = tid; i < n; i += kPcholThreads) piv[i] = pm[i];
}

__global__ void __launch_bounds__(kPcholThreads, 1)
    pchol_kernel(double *__restrict__ W, int n, double *__restrict__ X, i64 ldx,
                 int *__restrict__ piv)
{
    pchol_body(W, n, X, ldx, piv);
}

// Many factorizations in one launch, one CTA each (the batched TS-SVD).
__global__ void __launch_bounds__(kPcholThreads, 1) pchol_batch_kernel(const PcholTask *tasks)
{
    const PcholTask t = tasks[blockIdx.x];
    pchol_body(t.W, t.n, t.X, t.n, t.piv);
}

// Pivoted Cholesky over the whole grid, for n above one CTA's reach:
// W = R~^T R~ with R~ = R P^T, R the upper-triangular factor of the
// diagonally pivoted P^T W P (pivot: the largest remaining diagonal entry,
// lowest index on ties), stopped with the floor of pchol_kernel: once
// every remaining diagonal entry is <= delta = 2^-52 max_i W_ii, the
// remaining rows of R~ are sqrt(delta) times unit vectors on the remaining
// indices in increasing order (W = 0: R~ = I).
// The pivoting is logical: W stays in the original order, and row k of
// R~ (the k-th pivot's row, in original column order) is written as
// column k of X (X[k ldx + c]), so X's rows are in the original order and
// the eigenvectors found from X need no un-pivoting.
// Rows of W belong to CTAs round-robin (row i to CTA i mod gridDim.x).
// Step k: every CTA reads the pivot j (published by an atomic maximum of a
// packed key) and row j of W, forms row k of R~ in shared memory, and
// updates its own remaining rows by the rank-one term over the remaining
// columns (a sorted list, so the loads stay nearly coalesced); then it
// publishes the largest remaining diagonal entry of its rows for step
// k + 1 and the grid barrier ends the step.  The key packs the diagonal
// value's bit pattern (non-negative, so ordered as an unsigned integer)
// above 11 bits of (2047 - index): ties within the dropped low bits of the
// value go to the lower index; the pivot value itself is re-read exactly.
__device__ __forceinline__ unsigned long long pivot_key(double v, int i)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v > 0.0 ? v : 0.0);
    return (b & ~0x7ffull) | (unsigned long long)(2047 - i);
}

struct PcholArgs {
    double *W;  // n x n row-major, consumed
    double *X;  // column-major: column k = row k of R~
    i64 ldx;
    unsigned long long *key;  // [3] pivot keys, zeroed before the launch
    DevStatus *st;
    int n;
};

template <int NT>
__global__ void __launch_bounds__(NT) pchol_grid_kernel(PcholArgs p)
{
    extern __shared__ double pg_s[];
    const int n = p.n;
    double *r = pg_s;                              // [n] row k of R~
    int *act = reinterpret_cast<int *>(r + n);     // [n] remaining columns, increasing
    unsigned char *done = reinterpret_cast<unsigned char *>(act + n);  // [n]
    __shared__ unsigned long long s_key[NT / 32];
    __shared__ double s_piv, s_inv, s_delta;
    __shared__ int s_j, s_stop, s_nact;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
    const int G = gridDim.x, b = blockIdx.x;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(&p.st->bar[0]);
    int epoch = 0;
    for (int c = tid; c < n; c += NT) {
        done[c] = 0;
        act[c] = c;
    }
    if (tid == 0) s_nact = n;
    __syncthreads();
    // publishes this CTA's largest remaining diagonal entry into key slot q
    auto publish = [&](int q) {
        unsigned long long k = 0;
        for (int i = b + tid * G; i < n; i += NT * G)
            if (!done[i]) {
                const unsigned long long kk = pivot_key(__ldcg(p.W + (i64)i * n + i), i);
                k = kk > k ? kk : k;
            }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, k, o);
            k = t > k ? t : k;
        }
        if (lane == 0) s_key[warp] = k;
        __syncthreads();
        if (tid == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < NW; w++) t = s_key[w] > t ? s_key[w] : t;
            if (t != 0) atomicMax(p.key + q, t);
        }
    };
    publish(0);
    if (!grid_barrier(bar, epoch, &p.st->err)) return;
    int k = 0;
    for (; k < n; k++) {
        if (tid == 0) {
            const unsigned long long kk = __ldcg(p.key + (k % 3));
            const int j = 2047 - (int)(kk & 0x7ffull);
            const double dj = kk ? __ldcg(p.W + (i64)j * n + j) : 0.0;
            if (k == 0) s_delta = 0x1p-52 * dj;
            const double delta = s_delta;
            const int stop = (kk == 0 || !(delta > 0.0 && dj > delta)) ? 1 : 0;
            s_stop = stop;
            s_j = j;
            // (one thread: FP64 square root and divide are long sequences)
            s_piv = stop ? 0.0 : sqrt(dj);
            s_inv = stop ? 0.0 : 1.0 / s_piv;
            if (b == 0) atomicExch(p.key + (k + 2) % 3, 0ull);  // step k + 2's slot, read in k - 1
        }
        __syncthreads();
        if (s_stop) break;
        const int j = s_j, nact = s_nact;
        const double piv = s_piv, inv = s_inv;
        // row k of R~ over the remaining columns (others stay 0 in r)
        const double *wj = p.W + (i64)j * n;
        for (int t = tid; t < nact; t += NT) {
            const int c = act[t];
            r[c] = (c == j) ? piv : __ldcg(wj + c) * inv;
        }
        __syncthreads();
        if (b == 0)
            for (int c = tid; c < n; c += NT) __stcg(p.X + (i64)k * p.ldx + c, done[c] ? 0.0 : r[c]);
        // rank-one update of this CTA's remaining rows (i != j) over the
        // remaining columns, a warp per row, four loads in flight per lane
        for (int i = b + warp * G; i < n; i += NW * G) {
            if (done[i] || i == j) continue;
            double *wi = p.W + (i64)i * n;
            const double ri = r[i];
            int t = lane;
            for (; t + 96 < nact; t += 128) {
                const int c0 = act[t], c1 = act[t + 32], c2 = act[t + 64], c3 = act[t + 96];
                const double w0 = __ldcg(wi + c0), w1 = __ldcg(wi + c1);
                const double w2 = __ldcg(wi + c2), w3 = __ldcg(wi + c3);
                __stcg(wi + c0, fma(-ri, r[c0], w0));
                __stcg(wi + c1, fma(-ri, r[c1], w1));
                __stcg(wi + c2, fma(-ri, r[c2], w2));
                __stcg(wi + c3, fma(-ri, r[c3], w3));
            }
            for (; t < nact; t += 32) {
                const int c0 = act[t];
                __stcg(wi + c0, fma(-ri, r[c0], __ldcg(wi + c0)));
            }
        }
        __syncthreads();
        // j leaves the remaining columns (the list stays increasing)
        {
            int pos = -1;
            for (int t = tid; t < nact; t += NT)
                if (act[t] == j) pos = t;
            // at most one thread found it; share through s_j's neighbour
            __shared__ int s_pos;
            if (pos >= 0) s_pos = pos;
            __syncthreads();
            const int ps = s_pos;
            int v[(kPcholGridMaxN + NT - 1) / NT];
            int cnt = 0;
            for (int t = ps + 1 + tid; t < nact; t += NT) v[cnt++] = act[t];
            __syncthreads();
            cnt = 0;
            for (int t = ps + 1 + tid; t < nact; t += NT) act[t - 1] = v[cnt++];
            if (tid == 0) {
                done[j] = 1;
                s_nact = nact - 1;
            }
            __syncthreads();
        }
        publish((k + 1) % 3);
        if (!grid_barrier(bar, epoch, &p.st->err)) return;
    }
    // rows k .. n-1 of R~: the floor's square root on the remaining indices
    // in increasing order (act), spread over the CTAs
    const double tail = s_delta > 0.0 ? sqrt(s_delta) : 1.0;
    for (int kk = k + b; kk < n; kk += G) {
        const int c0 = act[kk - k];
        for (int c = tid; c < n; c += NT) __stcg(p.X + (i64)kk * p.ldx + c, c == c0 ? tail : 0.0);
    }
}

// V[piv[i]][j] = Xn[i][j] (n x n row-major): the eigenvectors of the
// pivoted matrix back in the original order.
__global__ void row_scatter_kernel(const double *__restrict__ Xn, const int *__restrict__ piv,
                                   int n, double *__restrict__ V)
{
    const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (i64)n * n) return;
    const i64 i = e / n, j = e - i * n;
    V[(i64)piv[i] * n + j] = Xn[e];
}


}  // namespace

cudaError_t launch_pchol(double *W, int n, double *X, i64 ldx, int *piv, cudaStream_t s)
{
    const size_t smem = sizeof(double) * ((size_t)n + 32) + sizeof(int) * ((size_t)n + 32);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pchol_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (n > 256) return cudaErrorInvalidValue;  // rows held as 8 values per lane
    ProfScope ps_("pchol", s);
    pchol_kernel<<<1, kPcholThreads, smem, s>>>(W, n, X, ldx, piv);
    return cudaGetLastError();
}

cudaError_t launch_pchol_batch(const PcholTask *tasks, int ntasks, int nmax, cudaStream_t s)
{
    if (ntasks < 1) return cudaSuccess;
    if (nmax > 256) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * ((size_t)nmax + 32) + sizeof(int) * ((size_t)nmax + 32);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pchol_batch_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    ProfScope ps_("pchol", s);
    pchol_batch_kernel<<<ntasks, kPcholThreads, smem, s>>>(tasks);
    return cudaGetLastError();
}

cudaError_t launch_pchol_grid(double *W, int n, double *X, i64 ldx, unsigned long long *key,
                              DevStatus *st, cudaStream_t s)
{
    if (n < 1 || n > kPcholGridMaxN) return cudaErrorInvalidValue;
    constexpr int NT = 256;
    cudaError_t e;
    if ((e = cudaMemsetAsync(key, 0, 3 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&st->bar[0], 0, sizeof(int) * 4, s)) != cudaSuccess) return e;
    const size_t smem = sizeof(double) * (size_t)n + sizeof(int) * (size_t)n + (size_t)n;
    const void *kern = (const void *)pchol_grid_kernel<NT>;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // one CTA per SM: every CTA reads the pivot row each step, so more CTAs
    // only add L2 traffic and barrier arrivals
    int blocks = num_sms();
    const int rows_cap = (n + 7) / 8;  // at least 8 rows (a warp each) per CTA
    if (blocks > rows_cap) blocks = rows_cap;
    if (blocks < 1) blocks = 1;
    PcholArgs a;
    a.W = W;
    a.X = X;
    a.ldx = ldx;
    a.key = key;
    a.st = st;
    a.n = n;
    void *args[] = {&a};
    ProfScope ps_("pchol_grid", s);
    return cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(NT), args, smem, s);
}

cudaError_t launch_row_scatter(const double *Xn, const int *piv, int n, double *V, cudaStream_t s)
{
    const i64 total = (i64)n * n;
    row_scatter_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Xn, piv, n, V);
    return cudaGetLastError();
}

cudaError_t launch_jacobi(double *X, i64 ldx, double *J, i64 ldj, int nr, int nc, int max_sweeps,
                          int *ctr, double *prm, DevStatus *st, int which, cudaStream_t s,
                          double tol)
{
    cudaError_t e;
    if (J) {
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
    a.prm = (double4 *)prm;
    a.nrm = prm + 8 * (size_t)((nc + 1) / 2);  // after [2][npairs] double4
    a.nr = nr;
    a.nc = nc;
    a.npad = nc + (nc & 1);
    a.max_sweeps = max_sweeps;
    a.tol = tol > 0.0 ? tol : (double)nr * 0x1p-53;
    a.rot = ctr;
    a.st = st;
    a.which = which;

    constexpr int NT = 128;
    const int npairs = a.npad / 2;
    const int mx = nr > nc ? nr : nc;
    const int ch = mx <= NT ? 1 : mx <= 2 * NT ? 2 : mx <= 4 * NT ? 4 : mx <= 8 * NT ? 8 : 0;
    auto pick = [&](bool js_) -> const void * {
        switch (ch * 2 + (js_ ? 1 : 0)) {
            case 2: return (const void *)jacobi_kernel<NT, 1, false>;
            case 3: return (const void *)jacobi_kernel<NT, 1, true>;
            case 4: return (const void *)jacobi_kernel<NT, 2, false>;
            case 5: return (const void *)jacobi_kernel<NT, 2, true>;
            case 8: return (const void *)jacobi_kernel<NT, 4, false>;
            case 9: return (const void *)jacobi_kernel<NT, 4, true>;
            case 16: return (const void *)jacobi_kernel<NT, 8, false>;
            case 17: return (const void *)jacobi_kernel<NT, 8, true>;
            case 1: return (const void *)jacobi_kernel<NT, 0, true>;
            default: return (const void *)jacobi_kernel<NT, 0, false>;
        }
    };
    // J's rows in shared memory when they fit: a CTA of a grid of g CTAs
    // holds ceil(nc / g) rows.  First choice: one pair per CTA (every CTA
    // one pair a round, nothing serialised), sized for that grid, if that
    // many CTAs fit on the GPU at once; else one CTA per SM (the row count
    // for at most one CTA per SM, an upper bound).
    auto js_bytes_for = [&](int g) {
        return sizeof(double4) * (size_t)npairs + sizeof(double) * (size_t)((nc + g - 1) / g) * nc;
    };
    bool js = false, one_pair = false;
    size_t js_bytes = 0;
    if (J != nullptr && js_bytes_for(npairs) <= kRowsSmemMax) {
        const void *k1 = pick(true);
        const size_t b1 = js_bytes_for(npairs);
        int ps1 = 0;
        if (b1 > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1)) !=
                cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps1, k1, NT, b1)) != cudaSuccess)
            return e;
        if ((i64)ps1 * num_sms() >= npairs) {
            js = true;
            one_pair = true;
            js_bytes = b1;
        }
    }
    if (J != nullptr && !js) {
        const int b0 = npairs < num_sms() ? npairs : num_sms();
        js_bytes = js_bytes_for(b0);
        js = js_bytes <= kRowsSmemMax;
    }
    const void *kern = pick(js);
    const size_t smem = js ? js_bytes : 0;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int blocks = num_sms() * per_sm;
    if (blocks > npairs) blocks = npairs;
    if (one_pair && blocks < npairs) return cudaErrorCooperativeLaunchTooLarge;  // (checked above)
    void *args[] = {&a};
    ProfScope ps_("jacobi_svd", s);
    return cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(NT), args, smem, s);
}

cudaError_t launch_jacobi_eig(double *B, double *B2, i64 ldb, double *V, i64 ldv, double *lam,
                              double *Vout, i64 ldvo, int n, int max_sweeps, int *ctr, double *prm,
                              int *perm, DevStatus *st, int which, cudaStream_t s, bool normwise)
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
    // the rotation-parameter scratch (>= 2n doubles) holds the diagonal after
    double *dg = prm;
    const int npad = n + (n & 1);
    const bool single = B2 != nullptr && npad / 2 <= kEigSmemPairs;
    if (n >= 2) {
        EigArgs a;
        a.B = B;
        a.B2 = B2;
        a.ldb = ldb;
        a.V = V;
        a.ldv = ldv;
        a.prm = (double4 *)prm;
        a.diag = dg;
        a.n = n;
        a.npad = npad;
        a.max_sweeps = max_sweeps;
        a.tol = (double)n * 0x1p-53;
        a.rot = ctr;
        a.st = st;
        a.which = which;
        a.normwise = normwise ? 1 : 0;
        constexpr int NT = 128;
        const int npairs0 = npad / 2;
        // V's rows in shared memory (ceil(n / g) rows for a grid of g CTAs):
        // sized for one pair per CTA when that grid fits on the GPU at once,
        // else for one CTA per SM
        auto vs_bytes_for = [&](int g) {
            return sizeof(double4) * (size_t)npairs0 + sizeof(double) * (size_t)((n + g - 1) / g) * n;
        };
        size_t vs_bytes = vs_bytes_for(npairs0 < num_sms() ? npairs0 : num_sms());
        if (single && vs_bytes_for(npairs0) <= kRowsSmemMax) {
            const void *k1 = (const void *)jacobi_eig1_kernel<NT, true>;
            const size_t b1 = vs_bytes_for(npairs0);
            int ps1 = 0;
            if (b1 > 48 * 1024 &&
                (e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)b1)) != cudaSuccess)
                return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps1, k1, NT, b1)) != cudaSuccess)
                return e;
            if ((i64)ps1 * num_sms() >= npairs0) vs_bytes = b1;
        }
        const bool vs = single && vs_bytes <= kRowsSmemMax;
        // two rounds per barrier: one CTA per pair, each on its own SM (with
        // two CTAs per SM the doubled FP64 work of a round outweighs the
        // saved barrier: measured at n = 512), V by rows
        const size_t two_bytes = sizeof(double4) * 2 * (size_t)npairs0 +
                                 sizeof(double) * (size_t)(npad + npairs0) +
                                 sizeof(double) * (size_t)((n + npairs0 - 1) / npairs0) * n;
        bool two = false;
        if (single && two_bytes <= kRowsSmemMax) {
            const void *k2 = (const void *)jacobi_eig2r_kernel<NT>;
            if (two_bytes > 48 * 1024 &&
                (e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)two_bytes)) != cudaSuccess)
                return e;
            int per_sm2 = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k2, NT, two_bytes)) !=
                cudaSuccess)
                return e;
            two = npairs0 <= num_sms() && (i64)per_sm2 * num_sms() >= npairs0;
        }
        const void *kern = two      ? (const void *)jacobi_eig2r_kernel<NT>
                           : !single ? (const void *)jacobi_eig_kernel<NT>
                           : vs      ? (const void *)jacobi_eig1_kernel<NT, true>
                                     : (const void *)jacobi_eig1_kernel<NT, false>;
        const size_t smem = two ? two_bytes
                            : !single ? 0 : vs ? vs_bytes : sizeof(double4) * (size_t)npairs0;
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) !=
            cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        int npairs = npad / 2;
        int blocks = num_sms() * per_sm;
        if (blocks > npairs || two) blocks = npairs;
        void *args[] = {&a};
        ProfScope ps_("jacobi_eig", s);
        if ((e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(NT), args, smem, s)) !=
            cudaSuccess)
            return e;
    } else {
        if ((e = cudaMemsetAsync(&st->sweeps[which], 0, sizeof(int), s)) != cudaSuccess) return e;
    }
    if (!(single && n >= 2)) {
        ProfScope ps_("diag", s);
        diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(B, ldb, n, dg);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
    ProfScope ps_("rank_sort", s);
    rank_sort_kernel<<<(n + 255) / 256, 256, 0, s>>>(dg, n, perm);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // unit eigenvectors: the norms of V's accumulated columns (prm + n)
    double *vn = prm + n;
    {
        const int warps_per_block = 8;
        ProfScope ps_("colnorm", s);
        colnorm_cm_kernel<<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0,
                            s>>>(V, ldv, n, n, vn);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
        i64 total = (i64)n * n;
        i64 blocks = (total + 255) / 256;
        if (blocks > (i64)num_sms() * 8) blocks = (i64)num_sms() * 8;
        if (blocks < 1) blocks = 1;
        ProfScope ps_("permute", s);
        permute_out_kernel<<<(unsigned)blocks, 256, 0, s>>>(nullptr, 0, V, ldv, 0, n, dg, perm,
                                                            Vout, ldvo, lam, nullptr, 0, nullptr,
                                                            vn);
    }
    return cudaGetLastError();
}

cudaError_t launch_jacobi_finalize(const double *X, i64 ldx, const double *J, i64 ldj, int nr,
                                   int nc, double *norms, int *perm, double *Jout, i64 ldjo,
                                   double *lam, double *Xout, i64 ldxo, cudaStream_t s,
                                   const int *orient, double *jnorm)
{
    cudaError_t e;
    {
        const int warps_per_block = 8;
        const int blocks = (nc + warps_per_block - 1) / warps_per_block;
        ProfScope ps_("colnorm", s);
        colnorm_cm_kernel<<<blocks, 32 * warps_per_block, 0, s>>>(X, ldx, nr, nc, norms);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (jnorm && J) {
            colnorm_cm_kernel<<<blocks, 32 * warps_per_block, 0, s>>>(J, ldj, nc, nc, jnorm);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    {
    ProfScope ps_("rank_sort", s);
    rank_sort_kernel<<<(nc + 255) / 256, 256, 0, s>>>(norms, nc, perm);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        i64 total = (J ? (i64)nc * nc : 0) + (Xout ? (i64)nr * nc : 0);
        i64 blocks = (total + 255) / 256;
        if (blocks > (i64)num_sms() * 8) blocks = (i64)num_sms() * 8;
        if (blocks < 1) blocks = 1;
        ProfScope ps_("permute", s);
        permute_out_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, J, ldj, nr, nc, norms, perm,
                                                            Jout, ldjo, lam, Xout, ldxo, orient,
                                                            J ? jnorm : nullptr);
    }
    return cudaGetLastError();
}

}  // namespace tssvd
