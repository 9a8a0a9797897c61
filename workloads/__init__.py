"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.

This module holds input construction only (random factors, spectra, test
matrices).  It contains none of the method's arithmetic: no Gram matrices,
eigendecompositions or TS-SVD steps.  Orthonormal factors come from a QR
factorisation of a seeded Gaussian matrix (numpy on the host, torch on a
device), with the signs of diag(R) made positive so the factor is unique.

Recipes (sizes and distributions of the workloads the method is run on):
  * known-spectrum tall matrices  A = U diag(sigma) V^T, U (m x n) and V
    (n x n) orthonormal from QR of N(0,1) matrices;
  * the paper's test matrix (eq. "originalmat" with "testS"/"testSl"):
    U, V orthonormal DCT-II bases, sigma_j = 10^(-20 (j-1)/(p-1));
  * the low-rank workload  A = U_r diag(1/j) V_r^T + 1e-4 G / sqrt(m);
  * batches of uneven tall problems with log-uniform spectra;
  * the Devil's-staircase spectrum of the paper's Appendix B (many
    repeated singular values of varying multiplicity, and zeros).
"""
import math

import numpy as np

# --------------------------------------------------------------------------
# Spectra
# --------------------------------------------------------------------------


def sigma_geometric(n, lo, hi=1.0):
    """n values falling geometrically from hi to lo (sigma_1 = hi)."""
    if n == 1:
        return np.array([hi], dtype=np.float64)
    j = np.arange(n, dtype=np.float64)
    return hi * (lo / hi) ** (j / (n - 1))


def sigma_small_tall(n=50):
    """sigma_j = 10^(-6 (j-1)/(n-1)): 1 down to 1e-6 (the 20000 x 50 case)."""
    return sigma_geometric(n, 1e-6)


def sigma_paper(p):
    """The paper's spectrum exp((j-1)/(p-1) ln 1e-20), j = 1..p (eq. testS)."""
    j = np.arange(p, dtype=np.float64)
    return np.exp(j / (p - 1) * np.log(1e-20)) if p > 1 else np.ones(1)


def sigma_distinct_gaps(n):
    """sigma_j = 1 + (n - j)/n, j = 1..n: distinct, gaps 1/n (gradient case)."""
    j = np.arange(1, n + 1, dtype=np.float64)
    return 1.0 + (n - j) / n


# --------------------------------------------------------------------------
# Orthonormal factors
# --------------------------------------------------------------------------


def sigma_devils_staircase(k):
    """The "Devil's staircase" spectrum of the paper's Appendix B: for
    j = 0..k-1, the real number j/k is rounded to six octal digits
    (round(j * 8^6 / k), evaluated in single precision with half-up
    rounding), every nonzero octal digit becomes the binary digit 1, the
    resulting six-bit binary number is divided by 2^6 - 1 = 63, and the k
    values are sorted in decreasing order.  Values lie in [0, 1] with many
    repeats (multiplicities vary) and include zeros."""
    q = np.float32(8.0 ** 6) / np.float32(k)
    out = np.empty(k, dtype=np.float64)
    for j in range(k):
        x = int(np.floor(np.float32(np.float32(j) * q) + np.float32(0.5)))
        bits = 0
        for pos in range(7):  # at most seven octal digits (8^6 itself)
            digit = (x >> (3 * pos)) & 7
            if digit:
                bits |= 1 << pos
        out[j] = bits / 63.0
    return np.sort(out)[::-1].copy()


def orthonormal(rows, cols, rng):
    """rows x cols matrix with orthonormal columns: Q of a Gaussian, diag(R) > 0."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return np.ascontiguousarray(Q * s)


def orthonormal_torch(rows, cols, seed, device, dtype=None):
    """Device-side variant of `orthonormal` (torch QR of a seeded Gaussian).

    Used only to build inputs too large to generate quickly on the host.
    """
    import torch
    dtype = dtype or torch.float64
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    G = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    return (Q * s).to(dtype).contiguous()


def dct2_basis(size, cols):
    """First `cols` columns of the orthonormal DCT-II basis of length `size`.

    Column j is sqrt(2/size) cos(pi (i + 1/2) j / size), with column 0 scaled
    to sqrt(1/size).
    """
    i = np.arange(size, dtype=np.float64)[:, None]
    j = np.arange(cols, dtype=np.float64)[None, :]
    C = np.sqrt(2.0 / size) * np.cos(np.pi * (i + 0.5) * j / size)
    C[:, 0] = np.sqrt(1.0 / size)
    return np.ascontiguousarray(C)


# --------------------------------------------------------------------------
# Test matrices
# --------------------------------------------------------------------------


def known_spectrum(m, n, sigma, seed):
    """A = U diag(sigma) V^T with seeded orthonormal U (m x n), V (n x n).

    Returns (A, U, sigma, V), all float64 numpy arrays.
    """
    rng = np.random.default_rng(seed)
    U = orthonormal(m, n, rng)
    V = orthonormal(n, n, rng)
    sigma = np.asarray(sigma, dtype=np.float64)
    A = (U * sigma) @ V.T
    return np.ascontiguousarray(A), U, sigma, V


def known_spectrum_torch(m, n, sigma, seed, device, dtype=None):
    """Device-built known-spectrum matrix (same recipe, torch RNG and QR)."""
    import torch
    dtype = dtype or torch.float64
    U = orthonormal_torch(m, n, seed, device)
    V = orthonormal_torch(n, n, seed + 1000003, device)
    s = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device)
    A = ((U * s) @ V.T).to(dtype).contiguous()
    return A, U, s, V


def known_spectrum_rowblock_torch(m_local, n, sigma, seed, rank, size, device):
    """Rank `rank`'s block of rows of a row-sharded known-spectrum matrix:
    A_r = (U_r / sqrt(size)) diag(sigma) V^T with U_r (m_local x n) seeded
    per rank and V shared.  The stacked U = [U_0; ...] / sqrt(size) has
    orthonormal columns (U^T U = sum_r U_r^T U_r / size = I), so the whole
    matrix has singular values sigma and right singular vectors V.
    Returns (A_r, sigma tensor, V)."""
    import torch
    Ur = orthonormal_torch(m_local, n, seed + 7919 * (rank + 1), device)
    V = orthonormal_torch(n, n, seed + 1000003, device)
    s = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device)
    A = ((Ur * (s / np.sqrt(size))) @ V.T).contiguous()
    return A, s, V


def paper_dct_matrix(m, n, p):
    """The paper's test matrix: DCT-II U (m x p) and V (n x p), sigma of eq.
    testS (p = n) or testSl (p = l), A = U diag(sigma) V^T (m x n)."""
    U = dct2_basis(m, p)
    V = dct2_basis(n, p)
    s = sigma_paper(p)
    return np.ascontiguousarray((U * s) @ V.T), U, s, V


def lowrank_plus_noise(m, n, r, seed, noise=1e-4):
    """A = U_r diag(1/j) V_r^T + noise * G / sqrt(m), U_r, V_r orthonormal."""
    rng = np.random.default_rng(seed)
    Ur = orthonormal(m, r, rng)
    Vr = orthonormal(n, r, rng)
    s = 1.0 / np.arange(1, r + 1, dtype=np.float64)
    A = (Ur * s) @ Vr.T
    A += (noise / math.sqrt(m)) * rng.standard_normal((m, n))
    return np.ascontiguousarray(A), Ur, s, Vr


def pca_data(m, n, sigma, seed, offset=1e3):
    """Observations with a known centred structure plus large column means:
    A = Q diag(sigma) V^T + 1 c^T, where Q (m x n) is orthonormal and
    orthogonal to the all-ones vector (so A - 1 c^T is exactly the centred
    part and its singular values are sigma) and c_j = offset * N(0, 1).

    Returns (A, c, Q, sigma, V), float64 numpy arrays.
    """
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, n))
    G -= G.mean(axis=0)  # columns orthogonal to the ones vector
    Q, R = np.linalg.qr(G)
    Q *= np.sign(np.diag(R))
    V = orthonormal(n, n, rng)
    sigma = np.asarray(sigma, dtype=np.float64)
    c = offset * rng.standard_normal(n)
    A = (Q * sigma) @ V.T + c
    return np.ascontiguousarray(A), c, Q, sigma, V


def mixing_draws(n, seed):
    """The random inputs of Remark "randomness"'s mixing for n real columns
    (h = ceil(n / 2) complex ones): two sets of phases, uniform on
    [0, 2 pi), and two uniformly random permutations of h (Fisher-Yates
    shuffles by numpy's generator).  Returns (theta1, theta2, perm1, perm2)."""
    h = (n + 1) // 2
    rng = np.random.default_rng(seed)
    t1 = rng.uniform(0.0, 2.0 * math.pi, h)
    t2 = rng.uniform(0.0, 2.0 * math.pi, h)
    p1 = rng.permutation(h).astype(np.int64)
    p2 = rng.permutation(h).astype(np.int64)
    return t1, t2, p1, p2


def gaussian(rows, cols, seed):
    """i.i.d. N(0,1) matrix (the starting matrix Omega of the subspace iteration)."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


def batch_shapes(count, seed, m_range=(1000, 200000), n_range=(16, 256)):
    """(m_b, n_b) pairs uniform in the given ranges."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=count)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(ms, ns)]


def batch_instance(m, n, seed, lo=1e-6):
    """One batch member: sigma i.i.d. log-uniform in [lo, 1], sorted descending."""
    rng = np.random.default_rng(seed)
    s = np.sort(np.exp(rng.uniform(np.log(lo), 0.0, size=n)))[::-1].copy()
    return known_spectrum(m, n, s, seed + 7919)
