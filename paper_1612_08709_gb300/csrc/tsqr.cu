// Algorithms 1 and 2 (randomized TS-SVD via TSQR): the random mixing of
// Remark "randomness" as an explicit orthogonal matrix, Householder TSQR
// (blocked QRs of row blocks, a reduction tree over the stacked R factors,
// and Q formed explicitly back down the tree) and the discard of R's
// diagonal.  All in FP64 on the CUDA cores: the block QRs are bound by the
// FP64 pipe (2 b n^2 flops to factor a block of b rows, 4 b n^2 to form its
// Q).  Panels of up to 16 columns are factored in shared memory; their
// reflections are applied to the rest of the block in compact WY form
// (I - V T V^T), register-tiled, so that every panel streams the block
// through L2 once.  At the upper levels of the tree, where blocks are
// fewer than SMs, the column tiles of one block are spread over the CTAs
// of a thread-block cluster.
#include "common.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace tssvd {
namespace {

// Columns 2k and 2k+1 of the real form of Omega = D F S D~ F S~ (one block
// per complex column k), written transposed into Mt = O^T (n2 x n2):
// Mt[2k][2j] = Re w, Mt[2k][2j+1] = Im w, Mt[2k+1][2j] = -Im w,
// Mt[2k+1][2j+1] = Re w, w = Omega_jk.  F is the unitary DFT.  A
// permutation entry outside [0, h) sets bad (and is read as the identity),
// so no index leaves the shared arrays.
__global__ void mixing_kernel(int h, const double *__restrict__ th, const i64 *__restrict__ perm,
                              double *__restrict__ Mt, int *bad)
{
    extern __shared__ double mx_s[];
    double *xr = mx_s, *xi = mx_s + h, *yr = mx_s + 2 * h, *yi = mx_s + 3 * h;
    const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const i64 *p1 = perm, *p2 = perm + h;
    const double *t1 = th, *t2 = th + h;
    auto pidx = [&](const i64 *p, int a) -> int {
        const i64 v = p[a];
        if (v < 0 || v >= h) {
            atomicExch(bad, 1);
            return a;
        }
        return (int)v;
    };
    const double sc = rsqrt((double)h);
    // S~ e_k then F: (F S~ e_k)_a = exp(-2 pi i a q / h) / sqrt(h), q = the
    // position a' with p2[a'] = k, i.e. F applied to a unit vector at q
    for (int a = tid; a < h; a += nt) {
        xr[a] = (pidx(p2, a) == k) ? 1.0 : 0.0;
        xi[a] = 0.0;
    }
    __syncthreads();
    for (int pass = 0; pass < 2; pass++) {
        // y = F x
        for (int a = tid; a < h; a += nt) {
            double sr = 0.0, si = 0.0;
            for (int b = 0; b < h; b++) {
                const double xb = xr[b], xib = xi[b];
                if (xb == 0.0 && xib == 0.0) continue;
                const i64 r = ((i64)a * b) % h;
                double s, c;
                sincospi(-2.0 * (double)r / (double)h, &s, &c);
                sr = fma(xb, c, fma(-xib, s, sr));
                si = fma(xb, s, fma(xib, c, si));
            }
            yr[a] = sr * sc;
            yi[a] = si * sc;
        }
        __syncthreads();
        if (pass == 0) {
            // D~ then S: x_a = (D~ y)_{p1[a]}
            for (int a = tid; a < h; a += nt) {
                const int q = pidx(p1, a);
                double s, c;
                sincos(t2[q], &s, &c);
                xr[a] = yr[q] * c - yi[q] * s;
                xi[a] = yr[q] * s + yi[q] * c;
            }
            __syncthreads();
        }
    }
    const int n2 = 2 * h;
    for (int j = tid; j < h; j += nt) {
        double s, c;
        sincos(t1[j], &s, &c);
        const double wr = yr[j] * c - yi[j] * s, wi = yr[j] * s + yi[j] * c;
        Mt[(i64)(2 * k) * n2 + 2 * j] = wr;
        Mt[(i64)(2 * k) * n2 + 2 * j + 1] = wi;
        Mt[(i64)(2 * k + 1) * n2 + 2 * j] = -wi;
        Mt[(i64)(2 * k + 1) * n2 + 2 * j + 1] = wr;
    }
}

constexpr int kQrThreads = 256;
constexpr int kQrWarps = kQrThreads / 32;
// Columns per tile of the trailing updates (lanes: TC columns x 32/TC rows).
constexpr int kQrTC = 16;

// Rows [qr_row0(q), qr_row0(q + 1)) of a tree level form block q of nblk:
// the level's rows / unit units split evenly, unit = 1 at the leaves (every
// block has at least n rows) and unit = n above them (every block holds
// whole stacked R factors).
__host__ __device__ __forceinline__ i64 qr_row0(i64 rows, int unit, int nblk, int q)
{
    return (i64)q * (rows / unit) / nblk * unit;
}

// Block row of the panel's active row a.  Dense blocks: every row from the
// panel's first column j0 down.  Blocks of kR stacked upper triangular R
// factors (n x n each): column c is zero below row c of every factor, and
// stays so, so the panel's reflections touch only rows j0 .. j0 + jb - 1 of
// the first factor and rows 0 .. j0 + jb - 1 of each further factor.
__device__ __forceinline__ int qr_active_rows(bool stacked, int rbk, int n, int j0, int jb)
{
    return stacked ? jb + (rbk / n - 1) * (j0 + jb) : rbk - j0;
}
__device__ __forceinline__ int qr_row_of(bool stacked, int n, int j0, int jb, int a)
{
    if (!stacked || a < jb) return j0 + a;
    const int t = a - jb, h = j0 + jb;
    return (t / h + 1) * n + t % h;
}

// Shared memory of the QR kernels, in doubles: the panel P (rbmax x PS),
// its top NB rows as V with the unit diagonal and zeros made explicit
// (Vt), the per-row-group partials of W = V^T C (Wp), W (Ws), op(T) W
// (Wt), T, V^T V (G), reduction scratch and the panel's row map (ints).
__host__ __device__ constexpr size_t qr_smem_doubles(int nb, int tc, i64 rbmax)
{
    return (size_t)rbmax * (nb + 1) + (size_t)nb * (nb + 1) + (size_t)kQrThreads * nb +
           2 * (size_t)nb * tc + 2 * (size_t)nb * nb + (size_t)kQrWarps * nb + 8 + nb +
           (size_t)(rbmax + 1) / 2;
}

template <int NB, int TC>
struct QrSmem {
    double *P, *Vt, *Wp, *Ws, *Wt, *Tm, *G, *red, *stp;
    int *rmap;
    __device__ QrSmem(double *base, int rbmax)
    {
        P = base;
        Vt = P + (size_t)rbmax * (NB + 1);
        Wp = Vt + NB * (NB + 1);
        Ws = Wp + kQrThreads * NB;
        Wt = Ws + NB * TC;
        Tm = Wt + NB * TC;
        G = Tm + NB * NB;
        red = G + NB * NB;
        stp = red + kQrWarps * NB;
        rmap = (int *)(stp + 8 + NB);
    }
};

// CTA-wide sums of each thread's v[0..K): out[k] (shared) for all threads
// on return.
template <int K>
__device__ __forceinline__ void qr_sum_vec(double (&v)[K], double *red, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) red[warp * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int w = 0; w < kQrWarps; w++) t += red[w * K + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// CTA-wide maximum of one value per thread, returned to every thread.
__device__ __forceinline__ double qr_max(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kQrWarps; w++) t = fmax(t, red[w]);
    __syncthreads();
    return t;
}

// Euclidean norm of P[i][j] over rows lo <= i < rb: the plain sum of
// squares, or, when that leaves [2^-960, 2^960] (underflow or overflow
// possible), the sum of squares of the entries scaled by a power of two
// near 1 / max |entry|.  Uniform across the CTA; all threads get it.
template <int PS>
__device__ double qr_col_norm(const double *P, int lo, int rb, int j, double *red, double *out,
                              bool *in_range)
{
    const int tid = threadIdx.x;
    double ss[1] = {0.0};
    for (int i = lo + tid; i < rb; i += kQrThreads) {
        const double x = P[i * PS + j];
        ss[0] = fma(x, x, ss[0]);
    }
    qr_sum_vec<1>(ss, red, out);
    const double xs = out[0];
    if (xs >= 0x1p-960 && xs <= 0x1p960) {
        *in_range = true;
        // only thread 0 uses the norm: one FP64 square root, not one per thread
        return threadIdx.x == 0 ? sqrt(xs) : 1.0;
    }
    *in_range = false;
    double am = 0.0;
    for (int i = lo + tid; i < rb; i += kQrThreads) am = fmax(am, fabs(P[i * PS + j]));
    am = qr_max(am, red);
    if (am == 0.0 || !(am <= 1.79e308)) return am;  // zero column, or inf / nan propagates
    const int e = ilogb(am);
    ss[0] = 0.0;
    for (int i = lo + tid; i < rb; i += kQrThreads) {
        const double x = ldexp(P[i * PS + j], -e);
        ss[0] = fma(x, x, ss[0]);
    }
    qr_sum_vec<1>(ss, red, out);
    return ldexp(sqrt(out[0]), e);
}

// Vt = the top NB rows of the panel's V: unit diagonal, zeros above it and
// in columns >= jb, P's entries below the diagonal.
template <int NB>
__device__ void qr_build_vt(const double *P, int jb, double *Vt)
{
    constexpr int PS = NB + 1;
    for (int e = threadIdx.x; e < NB * NB; e += kQrThreads) {
        const int i = e / NB, k = e % NB;
        Vt[i * PS + k] = (k >= jb || i < k) ? 0.0 : (i == k ? 1.0 : P[i * PS + k]);
    }
}

// Reflection JJ of the panel applied to the panel's columns JJ + 1 .. NB - 1
// (a compile-time range, so no lane computes a column the reflection does
// not change): w_c = sum_{i >= JJ} v_i P[i][c], P[i][c] -= tau v_i w_c.
template <int NB, int JJ>
__device__ __forceinline__ void qr_panel_update(double *P, int rb, double tau, double *red,
                                                double *stp)
{
    constexpr int PS = NB + 1, K = NB - 1 - JJ;
    if constexpr (K > 0) {
        const int tid = threadIdx.x;
        double w[K];
#pragma unroll
        for (int c = 0; c < K; c++) w[c] = 0.0;
        for (int i = JJ + tid; i < rb; i += kQrThreads) {
            const double v = (i == JJ) ? 1.0 : P[i * PS + JJ];
#pragma unroll
            for (int c = 0; c < K; c++) w[c] = fma(v, P[i * PS + JJ + 1 + c], w[c]);
        }
        qr_sum_vec<K>(w, red, stp + 4);
        for (int i = JJ + tid; i < rb; i += kQrThreads) {
            const double tv = tau * ((i == JJ) ? 1.0 : P[i * PS + JJ]);
#pragma unroll
            for (int c = 0; c < K; c++)
                P[i * PS + JJ + 1 + c] = fma(-tv, stp[4 + c], P[i * PS + JJ + 1 + c]);
        }
    }
    __syncthreads();
}

// qr_panel_update for a run-time column jj (uniform across the CTA).
template <int NB, int JJ = 0>
__device__ __forceinline__ void qr_panel_update_at(int jj, double *P, int rb, double tau,
                                                   double *red, double *stp)
{
    if constexpr (JJ < NB) {
        if (jj == JJ)
            qr_panel_update<NB, JJ>(P, rb, tau, red, stp);
        else
            qr_panel_update_at<NB, JJ + 1>(jj, P, rb, tau, red, stp);
    }
}

// Householder QR of the panel in shared memory: P (rb x NB, row stride
// NB + 1; columns >= jb are zero) becomes R above the diagonal and the
// reflection vectors v_k below it (v_k[k] = 1 implicit), reflection k
// being I - tau_k v_k v_k^T.  Then T (upper triangular, T_kk = tau_k) with
// H_0 H_1 ... H_{jb-1} = I - V T V^T (the compact WY form), and Vt.
// Every thread calls this; it ends with a barrier.
template <int NB>
__device__ void qr_panel(double *P, int rb, int jb, double *Tm, double *G, double *Vt, double *red,
                         double *stp)
{
    constexpr int PS = NB + 1;
    const int tid = threadIdx.x;
    for (int e = tid; e < NB * NB; e += kQrThreads) Tm[e] = 0.0;
    for (int jj = 0; jj < jb; jj++) {
        bool in_range;
        const double xn = qr_col_norm<PS>(P, jj + 1, rb, jj, red, stp, &in_range);
        if (tid == 0) {
            const double alpha = P[jj * PS + jj];
            double tau = 0.0, scv = 0.0;
            if (xn != 0.0) {
                const double nrm = (in_range && fabs(alpha) < 0x1p480)
                                       ? sqrt(fma(alpha, alpha, stp[0]))
                                       : hypot(alpha, xn);
                const double beta = -copysign(nrm, alpha);
                tau = (beta - alpha) / beta;
                scv = 1.0 / (alpha - beta);
                P[jj * PS + jj] = beta;
            }
            Tm[jj * NB + jj] = tau;
            stp[1] = tau;
            stp[2] = scv;
        }
        __syncthreads();
        const double tau = stp[1], scv = stp[2];
        if (tau == 0.0) continue;  // uniform: H_jj = I
        for (int i = jj + 1 + tid; i < rb; i += kQrThreads) P[i * PS + jj] *= scv;
        __syncthreads();
        qr_panel_update_at<NB>(jj, P, rb, tau, red, stp);
    }
    // G[k][l] = v_k . v_l (k < l < jb) = P[l][k] + sum_{i > l} P[i][k] P[i][l];
    // two threads per pair (alternate row pairs), combined by a shuffle
    {
        const int npair = jb * (jb - 1) / 2;
        const int q = tid >> 1, half = tid & 1;
        int k = 0, l = 1;
        double sacc = 0.0;
        if (q < npair) {
            int base = 0;
            while (q >= base + l) {
                base += l;
                ++l;
            }
            k = q - base;
            double a0 = 0.0, a1 = 0.0;
            int i = l + 1 + half;
            for (; i + 2 < rb; i += 4) {
                a0 = fma(P[i * PS + k], P[i * PS + l], a0);
                a1 = fma(P[(i + 2) * PS + k], P[(i + 2) * PS + l], a1);
            }
            if (i < rb) a0 = fma(P[i * PS + k], P[i * PS + l], a0);
            sacc = a0 + a1;
        }
        sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
        if (q < npair && half == 0) G[k * NB + l] = sacc + P[l * PS + k];
    }
    qr_build_vt<NB>(P, jb, Vt);
    __syncthreads();
    // T[0:l, l] = -tau_l T[0:l, 0:l] (V^T v_l)[0:l]
    for (int l = 1; l < jb; l++) {
        if (tid < l) {
            double acc = 0.0;
            for (int k = tid; k < l; k++) acc = fma(Tm[tid * NB + k], G[k * NB + l], acc);
            Tm[tid * NB + l] = -Tm[l * NB + l] * acc;
        }
        __syncthreads();
    }
}

// Applies the panel's block reflection to one tile of C (the panel's active
// row a is row sm.rmap[a] of C, a < rb; columns c0 .. c0 + TC - 1, only
// those in [clo, chi) changed): C <- C - V op(T) V^T C with op(T) = T^T
// (TRANS, the transpose of H_0 ... H_{jb-1}: the factorization's trailing
// update) or T (the product itself: forming Q).  Thread layout: lane = (row group, column),
// warps and row groups stride the rows; W = V^T C is reduced through
// shared memory.  Every thread calls this.
template <int NB, int TC, bool TRANS>
__device__ void qr_apply_tile(double *C, i64 ldc, int rb, int jb, int c0, int clo, int chi,
                              const QrSmem<NB, TC> &sm)
{
    constexpr int PS = NB + 1, RG = 32 / TC, RS = kQrWarps * RG, U = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tc = lane % TC, ro = warp * RG + lane / TC;
    const int c = c0 + tc;
    const bool cok = c >= clo && c < chi;
    double acc[NB];
#pragma unroll
    for (int k = 0; k < NB; k++) acc[k] = 0.0;
    for (int i = ro; i < rb; i += RS * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int r = i + u * RS;
            x[u] = (cok && r < rb) ? __ldcg(C + (i64)sm.rmap[r] * ldc + c) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int r = i + u * RS;
            if (r < rb) {
                const double *v = (r < jb) ? sm.Vt + r * PS : sm.P + r * PS;
#pragma unroll
                for (int k = 0; k < NB; k++) acc[k] = fma(v[k], x[u], acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NB; k++) sm.Wp[(ro * NB + k) * TC + tc] = acc[k];
    __syncthreads();
    for (int e = threadIdx.x; e < NB * TC; e += kQrThreads) {
        const int k = e / TC, t = e % TC;
        double s0 = 0.0, s1 = 0.0;
        for (int r = 0; r < RS; r += 2) {
            s0 += sm.Wp[(r * NB + k) * TC + t];
            s1 += sm.Wp[((r + 1) * NB + k) * TC + t];
        }
        sm.Ws[e] = s0 + s1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * TC; e += kQrThreads) {
        const int k = e / TC, t = e % TC;
        double s = 0.0;
        if (TRANS) {
            for (int q = 0; q <= k; q++) s = fma(sm.Tm[q * NB + k], sm.Ws[q * TC + t], s);
        } else {
            for (int q = k; q < NB; q++) s = fma(sm.Tm[k * NB + q], sm.Ws[q * TC + t], s);
        }
        sm.Wt[e] = s;
    }
    __syncthreads();
    double w[NB];
#pragma unroll
    for (int k = 0; k < NB; k++) w[k] = sm.Wt[k * TC + tc];
    if (!cok) return;
    for (int i = ro; i < rb; i += RS * U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int r = i + u * RS;
            x[u] = (r < rb) ? __ldcg(C + (i64)sm.rmap[r] * ldc + c) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int r = i + u * RS;
            if (r < rb) {
                const double *v = (r < jb) ? sm.Vt + r * PS : sm.P + r * PS;
                double y = x[u];
#pragma unroll
                for (int k = 0; k < NB; k++) y = fma(-v[k], w[k], y);
                __stcg(C + (i64)sm.rmap[r] * ldc + c, y);
            }
        }
    }
}

__device__ __forceinline__ void qr_cluster_sync()
{
    __threadfence();
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Blocked Householder QR of every row block of one tree level (X: rows x
// n, leading dimension ldx, overwritten by R above and V below the
// diagonal of each block).  CTA (blk, part), cs parts per block: part owns
// the column tiles t with t % cs == part and applies every panel's
// reflection to them; every part factors each panel itself (identical
// arithmetic, so identical results) after a cluster barrier has made the
// owner's update of the panel's columns visible.  The factored panel and
// its T are written back by the owner one step later, once no part reads
// the panel's columns any more.  Per block: T blocks to Tg, R (n x n,
// zeros below the diagonal) to rows [blk n, blk n + n) of Rs.
template <int NB, int TC>
__global__ void __launch_bounds__(kQrThreads, 1)
    geqrf_kernel(double *__restrict__ X, i64 ldx, i64 rows, int unit, int n, int nblk, int cs,
                 int rbmax, double *__restrict__ Tg, double *__restrict__ Rs)
{
    constexpr int PS = NB + 1;
    extern __shared__ double qr_smem[];
    const QrSmem<NB, TC> sm(qr_smem, rbmax);
    const int blk = blockIdx.x / cs, part = blockIdx.x % cs, tid = threadIdx.x;
    const i64 r0 = qr_row0(rows, unit, nblk, blk), r1 = qr_row0(rows, unit, nblk, blk + 1);
    const int rbk = (int)(r1 - r0);
    const bool stacked = unit > 1;
    const int kq = rbk < n ? rbk : n;
    const int npan = (kq + NB - 1) / NB, npan_all = (n + NB - 1) / NB;
    const int ntiles = (n + TC - 1) / TC;
    double *Xb = X + r0 * ldx;
    // sm.rmap = the active rows of panel p
    auto map_rows = [&](int j0, int jb, int rb) {
        for (int a = tid; a < rb; a += kQrThreads) sm.rmap[a] = qr_row_of(stacked, n, j0, jb, a);
    };
    // the owner writes panel p (rows in sm.rmap) and its T back
    auto write_back = [&](int p) {
        const int j0 = p * NB, jb = min(NB, kq - j0);
        const int rb = qr_active_rows(stacked, rbk, n, j0, jb);
        if ((j0 / TC) % cs != part) return;
        for (int e = tid; e < rb * NB; e += kQrThreads) {
            const int i = e / NB, k = e % NB;
            if (k < jb) __stcg(Xb + (i64)sm.rmap[i] * ldx + j0 + k, sm.P[i * PS + k]);
        }
        double *T = Tg + ((i64)blk * npan_all + p) * NB * NB;
        for (int e = tid; e < NB * NB; e += kQrThreads) T[e] = sm.Tm[e];
    };
    for (int p = 0; p < npan; p++) {
        const int j0 = p * NB, jb = min(NB, kq - j0);
        const int rb = qr_active_rows(stacked, rbk, n, j0, jb);
        if (p > 0) {
            write_back(p - 1);
            __syncthreads();
        }
        map_rows(j0, jb, rb);
        __syncthreads();
        for (int e = tid; e < rb * NB; e += kQrThreads) {
            const int i = e / NB, k = e % NB;
            sm.P[i * PS + k] = (k < jb) ? __ldcg(Xb + (i64)sm.rmap[i] * ldx + j0 + k) : 0.0;
        }
        __syncthreads();
        qr_panel<NB>(sm.P, rb, jb, sm.Tm, sm.G, sm.Vt, sm.red, sm.stp);
        const int clo = j0 + jb;
        for (int t = clo / TC; t < ntiles; t++)
            if (t % cs == part) qr_apply_tile<NB, TC, true>(Xb, ldx, rb, jb, t * TC, clo, n, sm);
        if (cs > 1)
            qr_cluster_sync();
        else
            __syncthreads();
    }
    if (npan > 0) write_back(npan - 1);
    __syncthreads();
    double *R = Rs + (i64)blk * n * n;
    for (int t = part; t < ntiles; t += cs)
        for (int e = tid; e < n * TC; e += kQrThreads) {
            const int i = e / TC, c = t * TC + e % TC;
            if (c < n) R[(i64)i * n + c] = (i <= c && i < kq) ? __ldcg(Xb + (i64)i * ldx + c) : 0.0;
        }
}

// Q of every row block of one level: Y = H_0 ... H_{kq-1} [C; 0], C = rows
// [blk n, blk n + n) of Cin (the next level's Q), or the identity at the
// top, written to the block's rows of Qout.  Panels are applied last to
// first, each to its active rows (those of the factorization); CTA (blk,
// part) forms the column tiles t % cs == part (no dependence between
// parts).  With C = I, columns below the panel's first column are still
// unit vectors and are skipped.
template <int NB, int TC>
__global__ void __launch_bounds__(kQrThreads, 1)
    orgqr_kernel(const double *__restrict__ X, i64 ldx, i64 rows, int unit, int n, int nblk,
                 int cs, int rbmax, const double *__restrict__ Tg, const double *__restrict__ Cin,
                 double *__restrict__ Qout, i64 ldq)
{
    constexpr int PS = NB + 1;
    extern __shared__ double qr_smem[];
    const QrSmem<NB, TC> sm(qr_smem, rbmax);
    const int blk = blockIdx.x / cs, part = blockIdx.x % cs, tid = threadIdx.x;
    const i64 r0 = qr_row0(rows, unit, nblk, blk), r1 = qr_row0(rows, unit, nblk, blk + 1);
    const int rbk = (int)(r1 - r0);
    const bool stacked = unit > 1;
    const int kq = rbk < n ? rbk : n;
    const int npan = (kq + NB - 1) / NB, npan_all = (n + NB - 1) / NB;
    const int ntiles = (n + TC - 1) / TC;
    const double *Xb = X + r0 * ldx;
    double *Y = Qout + r0 * ldq;
    for (int t = part; t < ntiles; t += cs)
        for (int e = tid; e < rbk * TC; e += kQrThreads) {
            const int i = e / TC, c = t * TC + e % TC;
            if (c >= n) continue;
            double y = 0.0;
            if (i < n) y = Cin ? Cin[((i64)blk * n + i) * n + c] : (i == c ? 1.0 : 0.0);
            __stcg(Y + (i64)i * ldq + c, y);
        }
    for (int p = npan - 1; p >= 0; p--) {
        const int j0 = p * NB, jb = min(NB, kq - j0);
        const int rb = qr_active_rows(stacked, rbk, n, j0, jb);
        __syncthreads();  // the previous panel's readers of sm are done
        for (int a = tid; a < rb; a += kQrThreads) sm.rmap[a] = qr_row_of(stacked, n, j0, jb, a);
        __syncthreads();
        for (int e = tid; e < rb * NB; e += kQrThreads) {
            const int i = e / NB, k = e % NB;
            sm.P[i * PS + k] = (k < jb) ? Xb[(i64)sm.rmap[i] * ldx + j0 + k] : 0.0;
        }
        const double *T = Tg + ((i64)blk * npan_all + p) * NB * NB;
        for (int e = tid; e < NB * NB; e += kQrThreads) sm.Tm[e] = T[e];
        __syncthreads();
        qr_build_vt<NB>(sm.P, jb, sm.Vt);
        __syncthreads();
        const int clo = Cin ? 0 : j0;
        for (int t = part; t < ntiles; t += cs)
            if ((t + 1) * TC > clo)
                qr_apply_tile<NB, TC, false>(Y, ldq, rb, jb, t * TC, clo, n, sm);
    }
}

// Discard of Algorithms 1 and 2: row j of R and column j of Q are zeroed
// when |R_jj| < |R_00| wp or R_jj == 0.  keep[j] receives 0/1.
__global__ void tsqr_keep_kernel(const double *R, int n, double wp, int *keep)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double d = fabs(R[(i64)j * n + j]), thr = fabs(R[0]) * wp;
    keep[j] = (d > 0.0 && !(d < thr)) ? 1 : 0;
}

__global__ void tsqr_mask_kernel(double *R, double *Q, i64 m, int n, const int *keep)
{
    const i64 total = m * n + (i64)n * n;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (i64)gridDim.x * blockDim.x) {
        if (e < m * n) {
            const int c = (int)(e % n);
            if (!keep[c]) Q[e] = 0.0;
        } else {
            const i64 f = e - m * n;
            if (!keep[f / n]) R[f] = 0.0;
        }
    }
}

// The mixing draw for w columns from the draw for l >= w columns (h and hw
// complex entries): the first hw phases of each set and each permutation
// restricted to 0..hw-1 (its entries below hw, in their order).  One
// thread: h is at most a few thousand.  An entry outside [0, h) sets bad.
__global__ void restrict_mix_kernel(const double *th, const i64 *perm, int h, int hw,
                                    double *thw, i64 *permw, int *bad)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int a = 0; a < hw; a++) {
        thw[a] = th[a];
        thw[hw + a] = th[h + a];
    }
    for (int set = 0; set < 2; set++) {
        int c = 0;
        for (int a = 0; a < h; a++) {
            const i64 v = perm[(i64)set * h + a];
            if (v < 0 || v >= h) {
                *bad = 1;
                continue;
            }
            if (v < hw && c < hw) permw[(i64)set * hw + c++] = v;
        }
        for (; c < hw; c++) permw[(i64)set * hw + c] = c;  // only after a bad entry
    }
}

}  // namespace

// ------------------------------------------------------------ launchers

cudaError_t launch_restrict_mix(const double *th, const i64 *perm, int h, int hw, double *thw,
                                i64 *permw, int *bad, cudaStream_t s)
{
    restrict_mix_kernel<<<1, 32, 0, s>>>(th, perm, h, hw, thw, permw, bad);
    return cudaGetLastError();
}

cudaError_t launch_mixing(int h, const double *th, const i64 *perm, double *Mt, int *bad,
                          cudaStream_t s)
{
    ProfScope ps_("mixing", s);
    const size_t smem = sizeof(double) * 4 * (size_t)h;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(mixing_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    mixing_kernel<<<h, 128, smem, s>>>(h, th, perm, Mt, bad);
    return cudaGetLastError();
}

constexpr size_t kQrSmemCap = 220 * 1024;

// Panel width of a level whose blocks have at most rbmax rows: the widest
// of 16, 8, 4, 2 whose shared memory fits (0: none does).
static int tsqr_panel_width(i64 rbmax)
{
    for (int nb = 16; nb >= 2; nb /= 2)
        if (qr_smem_doubles(nb, kQrTC, rbmax) * sizeof(double) <= kQrSmemCap) return nb;
    return 0;
}

// The most rows a block may have with 16-column panels.
static i64 tsqr_rows_cap()
{
    i64 lo = 16, hi = 1 << 16;
    while (lo < hi) {
        const i64 mid = (lo + hi + 1) / 2;
        if (qr_smem_doubles(16, kQrTC, mid) * sizeof(double) <= kQrSmemCap)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The reduction tree.  Level 0 (the leaves): X's m rows in nblk blocks of
// at most max(cap, 2n) rows (cap: the rows a 16-column panel allows),
// rounded up to whole waves over the SMs when there are at least half as
// many blocks as SMs and every block keeps 2n rows.  Level l + 1: the
// nblk(l) stacked n x n R factors of level l, k per block (k = cap / n,
// between 2 and 8), up to one block.
struct TsqrPlan {
    int L;
    i64 rows[64];
    int unit[64], nblk[64], rbmax[64];
};

static void tsqr_plan(i64 m, int n, TsqrPlan &P)
{
    const i64 cap = tsqr_rows_cap();
    const i64 bleaf = cap > 2 * (i64)n ? cap : 2 * (i64)n;
    i64 nb0 = (m + bleaf - 1) / bleaf;
    const int sms = num_sms();
    if (nb0 >= sms / 2) {
        const i64 r = (nb0 + sms - 1) / sms * sms;
        if (m / r >= 2 * (i64)n) nb0 = r;
    }
    if (nb0 < 1) nb0 = 1;
    i64 k = cap / n;
    if (k < 2) k = 2;
    if (k > 8) k = 8;
    P.L = 0;
    i64 rows = m, nb = nb0;
    int unit = 1;
    while (P.L < 64) {
        const int l = P.L++;
        P.rows[l] = rows;
        P.unit[l] = unit;
        P.nblk[l] = (int)nb;
        const i64 units = rows / unit;
        P.rbmax[l] = (int)((units + nb - 1) / nb * unit);
        if (nb == 1) break;
        rows = nb * n;
        unit = n;
        nb = (nb + k - 1) / k;
    }
}

size_t tsqr_workspace_doubles(i64 m, int n)
{
    TsqrPlan P;
    tsqr_plan(m, n, P);
    size_t d = 0;
    for (int l = 0; l < P.L; l++) {
        const int nb = P.nblk[l];
        d += (size_t)nb * ((size_t)n + 16) * 16 + 8;  // T blocks (panel width <= 16)
        d += (size_t)nb * n * n + 8;                 // stacked R (next level's X)
        if (l > 0) d += (size_t)P.rows[l] * n + 8;   // Q of this level
    }
    return d + 64;
}

template <int NB>
static cudaError_t launch_geqrf_nb(double *X, i64 rows, int unit, int n, int nblk, int cs,
                                   int rbmax, double *Tg, double *Rs, cudaStream_t s)
{
    auto kern = geqrf_kernel<NB, kQrTC>;
    const size_t smem = qr_smem_doubles(NB, kQrTC, rbmax) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nblk * cs));
    cfg.blockDim = dim3(kQrThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    // Cluster width: each width's co-resident cluster count gives the waves
    // a level needs; the cost model is waves x (the widest part's share of
    // the tile work + a fixed share for the panel chain every part runs).
    {
        int best = 1;
        double best_cost = 1e300;
        for (int c = cs; c >= 1; c--) {
            int ncl = 0;
            if (c > 1) {
                static std::mutex mu;
                static std::map<std::tuple<int, int, size_t>, int> cache;
                const auto key = std::make_tuple(NB, c, smem);
                std::lock_guard<std::mutex> g(mu);
                auto it = cache.find(key);
                if (it != cache.end()) {
                    ncl = it->second;
                } else {
                    cfg.gridDim = dim3((unsigned)(nblk * c));
                    at[0].val.clusterDim.x = (unsigned)c;
                    cfg.numAttrs = 1;
                    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) {
                        cudaGetLastError();
                        ncl = 0;
                    }
                    cache[key] = ncl;
                }
            } else {
                ncl = num_sms();
            }
            if (ncl <= 0) continue;
            const int waves = (nblk + ncl - 1) / ncl;
            const double cost = waves * (1.0 / c + 0.1);
            if (cost < best_cost) {
                best_cost = cost;
                best = c;
            }
        }
        cs = best;
    }
    at[0].val.clusterDim.x = (unsigned)cs;
    cfg.gridDim = dim3((unsigned)(nblk * cs));
    cfg.numAttrs = cs > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, X, (i64)n, rows, unit, n, nblk, cs, rbmax, Tg, Rs);
}

template <int NB>
static cudaError_t launch_orgqr_nb(const double *X, i64 rows, int unit, int n, int nblk, int cs,
                                   int rbmax, const double *Tg, const double *Cin, double *Q,
                                   cudaStream_t s)
{
    auto kern = orgqr_kernel<NB, kQrTC>;
    const size_t smem = qr_smem_doubles(NB, kQrTC, rbmax) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(nblk * cs), kQrThreads, smem, s>>>(X, (i64)n, rows, unit, n, nblk, cs, rbmax,
                                                         Tg, Cin, Q, (i64)n);
    return cudaGetLastError();
}

// Parts per block of a level with nblk blocks: enough CTAs to cover the
// SMs once, at most one per column tile (and at most 8, a portable
// cluster, for the factorization, whose parts synchronise).
static int tsqr_parts(int nblk, int n, int cap)
{
    const int ntiles = (n + kQrTC - 1) / kQrTC;
    int cs = nblk >= num_sms() ? 1 : num_sms() / nblk;
    if (cs > ntiles) cs = ntiles;
    if (cs > cap) cs = cap;
    return cs < 1 ? 1 : cs;
}

cudaError_t launch_tsqr(double *X, i64 m, int n, double *work, double *R, double *Q,
                        cudaStream_t s)
{
    TsqrPlan P;
    tsqr_plan(m, n, P);
    const int L = P.L;
    double *Tgs[64], *Rst[64], *Qs[64];
    int pw[64];
    double *w = work;
    for (int l = 0; l < L; l++) {
        const int nb = P.nblk[l];
        pw[l] = tsqr_panel_width(P.rbmax[l]);
        if (pw[l] == 0) return cudaErrorInvalidValue;
        Tgs[l] = w;
        w += (size_t)nb * ((size_t)n + 16) * 16 + 8;
        Rst[l] = w;
        w += (size_t)nb * n * n + 8;
        Qs[l] = (l == 0) ? Q : w;
        if (l > 0) w += (size_t)P.rows[l] * n + 8;
    }
    static const char *const kGeqrfNames[] = {"tsqr_geqrf", "tsqr_geqrf_tree1", "tsqr_geqrf_tree2",
                                              "tsqr_geqrf_tree3", "tsqr_geqrf_tree4+"};
    static const char *const kOrgqrNames[] = {"tsqr_orgqr", "tsqr_orgqr_tree1", "tsqr_orgqr_tree2",
                                              "tsqr_orgqr_tree3", "tsqr_orgqr_tree4+"};
    // factorization up the tree
    for (int l = 0; l < L; l++) {
        double *Xl = (l == 0) ? X : Rst[l - 1];
        const int cs = tsqr_parts(P.nblk[l], n, 8);
        ProfScope ps_(kGeqrfNames[l < 4 ? l : 4], s);
        cudaError_t e;
        const i64 rw = P.rows[l];
        const int u = P.unit[l], nb = P.nblk[l], rm = P.rbmax[l];
        switch (pw[l]) {
        case 16: e = launch_geqrf_nb<16>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Rst[l], s); break;
        case 8: e = launch_geqrf_nb<8>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Rst[l], s); break;
        case 4: e = launch_geqrf_nb<4>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Rst[l], s); break;
        default: e = launch_geqrf_nb<2>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Rst[l], s); break;
        }
        if (e != cudaSuccess) return e;
    }
    // R = the top block's R
    cudaError_t e = cudaMemcpyAsync(R, Rst[L - 1], sizeof(double) * (size_t)n * n,
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // Q down the tree
    for (int l = L - 1; l >= 0; l--) {
        const double *Xl = (l == 0) ? X : Rst[l - 1];
        const double *Cin = (l == L - 1) ? nullptr : Qs[l + 1];
        const int cs = tsqr_parts(P.nblk[l], n, 1 << 20);
        ProfScope ps_(kOrgqrNames[l < 4 ? l : 4], s);
        const i64 rw = P.rows[l];
        const int u = P.unit[l], nb = P.nblk[l], rm = P.rbmax[l];
        switch (pw[l]) {
        case 16: e = launch_orgqr_nb<16>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Cin, Qs[l], s); break;
        case 8: e = launch_orgqr_nb<8>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Cin, Qs[l], s); break;
        case 4: e = launch_orgqr_nb<4>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Cin, Qs[l], s); break;
        default: e = launch_orgqr_nb<2>(Xl, rw, u, n, nb, cs, rm, Tgs[l], Cin, Qs[l], s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_tsqr_discard(double *R, double *Q, i64 m, int n, double wp, int *keep,
                                cudaStream_t s)
{
    ProfScope ps_("tsqr_discard", s);
    tsqr_keep_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, n, wp, keep);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    i64 blocks = (m * n + (i64)n * n + 255) / 256;
    if (blocks > (i64)num_sms() * 8) blocks = (i64)num_sms() * 8;
    tsqr_mask_kernel<<<(unsigned)blocks, 256, 0, s>>>(R, Q, m, n, keep);
    return cudaGetLastError();
}

}  // namespace tssvd
