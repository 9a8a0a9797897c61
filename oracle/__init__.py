"""ctypes binding of the plain FP64 CPU oracle (oracle/tssvd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg, never by the product package.  It shares no
code with the CUDA library.  Every function takes and returns numpy float64
arrays (row-major, C-contiguous); see the C file for the paper passages
each step follows.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_gram.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64]
        L.or_matmul.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64, _i64, _dp, _i64]
        L.or_matmul_tn.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64, _i64, _dp, _i64]
        L.or_col_norms.argtypes = [_dp, _i64, _i64, _i64, _dp]
        L.or_maxentry_scale.argtypes = [_dp, _i64, _i64, _i64, _dp]
        L.or_jacobi.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64, _dp, ctypes.c_int]
        L.or_jacobi.restype = ctypes.c_int
        L.or_jacobi_eig.argtypes = [_dp, _i64, _i64, _dp, _i64, _dp, ctypes.c_int]
        L.or_jacobi_eig.restype = ctypes.c_int
        L.or_ts_svd1.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_double, ctypes.c_int,
                                 _dp, _i64, _dp, _dp, _i64, _lp]
        L.or_ts_svd1.restype = ctypes.c_int
        L.or_ts_svd2.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, _dp, _i64, _dp, _dp, _i64, _lp, _lp]
        L.or_ts_svd2.restype = ctypes.c_int
        L.or_mixing.argtypes = [_i64, _dp, _dp, _lp, _lp, _dp]
        L.or_householder_qr.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64, _dp, _i64]
        L.or_ts_svd_tsqr.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_double, _dp,
                                     _dp, _lp, _lp, ctypes.c_int, _dp, _i64, _dp, _dp, _i64, _lp]
        L.or_ts_svd_tsqr.restype = ctypes.c_int
        L.or_lowrank_svd_tsqr.argtypes = [_dp, _i64, _i64, _i64, _i64, _i64, ctypes.c_int, _dp,
                                          _dp, _dp, _lp, _lp, ctypes.c_double, ctypes.c_int, _dp,
                                          _i64, _dp, _dp, _i64, _lp]
        L.or_lowrank_svd_tsqr.restype = ctypes.c_int
        L.or_col_means.argtypes = [_dp, _i64, _i64, _i64, _dp]
        L.or_pca.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                             ctypes.c_int, _dp, _dp, _i64, _dp, _dp, _i64, _lp]
        L.or_pca.restype = ctypes.c_int
        L.or_lowrank_svd.argtypes = [_dp, _i64, _i64, _i64, _i64, _i64, ctypes.c_int, _dp,
                                     ctypes.c_double, ctypes.c_int, _dp, _i64, _dp, _dp,
                                     _i64, _lp, _lp]
        L.or_lowrank_svd.restype = ctypes.c_int
        L.or_ts_svd_backward.argtypes = [_dp, _i64, _i64, _i64, _dp, _dp, _i64, _dp, _i64,
                                         _dp, _dp, _i64, _dp, _i64]
        L.or_lowrank_svd_backward.argtypes = [_dp, _i64, _i64, _i64, _dp, _dp, _i64, _i64,
                                              _dp, _i64, _dp, _dp, _i64, _dp, _i64]
        L.or_orth_error.argtypes = [_dp, _i64, _i64, _i64]
        L.or_orth_error.restype = ctypes.c_double
        L.or_spectral_error.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64, _dp, _dp, _i64,
                                        _i64, ctypes.c_int, ctypes.c_uint64]
        L.or_spectral_error.restype = ctypes.c_double
        L.or_num_threads.restype = ctypes.c_int
        L.or_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# Paper default for the discard threshold: square root of a working
# precision of 1e-11 (Remark "working"; Algorithms 3 and 4, discard steps).
PAPER_DROP_TOL = 1e-11 ** 0.5
MAX_SWEEPS = 50


def num_threads():
    return lib().or_num_threads()


def set_num_threads(t):
    lib().or_set_num_threads(int(t))


def gram(A):
    A = _c(A)
    m, n = A.shape
    B = np.zeros((n, n))
    lib().or_gram(_p(A), m, n, n, _p(B), n)
    return B


def matmul(A, X):
    A, X = _c(A), _c(X)
    C = np.zeros((A.shape[0], X.shape[1]))
    lib().or_matmul(_p(A), A.shape[0], A.shape[1], A.shape[1], _p(X), X.shape[1],
                    X.shape[1], _p(C), C.shape[1])
    return C


def matmul_tn(A, X):
    A, X = _c(A), _c(X)
    C = np.zeros((A.shape[1], X.shape[1]))
    lib().or_matmul_tn(_p(A), A.shape[0], A.shape[1], A.shape[1], _p(X), X.shape[1],
                       X.shape[1], _p(C), C.shape[1])
    return C


def col_norms(Y):
    Y = _c(Y)
    s = np.zeros(Y.shape[1])
    lib().or_col_norms(_p(Y), Y.shape[0], Y.shape[1], Y.shape[1], _p(s))
    return s


def maxentry_scale(A):
    A = _c(A)
    d = np.zeros(A.shape[1])
    lib().or_maxentry_scale(_p(A), A.shape[0], A.shape[1], A.shape[1], _p(d))
    return d


def jacobi(X, max_sweeps=MAX_SWEEPS):
    """One-sided Jacobi: returns (X_out, J, s, sweeps) with X_in J = X_out."""
    X = _c(X).copy()
    nr, nc = X.shape
    J = np.zeros((nc, nc))
    s = np.zeros(nc)
    sw = lib().or_jacobi(_p(X), nr, nc, nc, _p(J), nc, _p(s), int(max_sweeps))
    return X, J, s, sw


def jacobi_eig(B, max_sweeps=MAX_SWEEPS):
    """Gram-form Jacobi eigendecomposition: returns (lam, V, B_rot, sweeps)."""
    B = _c(B).copy()
    n = B.shape[0]
    V = np.zeros((n, n))
    lam = np.zeros(n)
    sw = lib().or_jacobi_eig(_p(B), n, n, _p(V), n, _p(lam), int(max_sweeps))
    return lam, V, B, sw


def ts_svd(A, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, max_sweeps=MAX_SWEEPS,
           return_diag=False):
    """Algorithm 3 (passes=1) or Algorithm 4 (passes=2) on A (m x n).

    Returns (U m x n, S n, V n x n, rank, status); columns past `rank` are 0.
    """
    A = _c(A)
    m, n = A.shape
    U = np.zeros((m, n)); S = np.zeros(n); V = np.zeros((n, n))
    r = ctypes.c_int64(0)
    diag = (ctypes.c_int64 * 4)()
    if passes == 1:
        st = lib().or_ts_svd1(_p(A), m, n, n, float(drop_tol), int(max_sweeps),
                              _p(U), n, _p(S), _p(V), n, ctypes.byref(r))
    else:
        st = lib().or_ts_svd2(_p(A), m, n, n, int(bool(scale)), float(drop_tol),
                              int(max_sweeps), _p(U), n, _p(S), _p(V), n,
                              ctypes.byref(r), diag)
    out = (U, S, V, r.value, st)
    if return_diag:
        return out + ((diag[0], diag[1]),)
    return out


def _ip(a):
    return a.ctypes.data_as(_lp)


def mixing(theta1, theta2, perm1, perm2):
    """Real 2h x 2h matrix of Remark "randomness"'s Omega = D F S D~ F S~."""
    t1, t2 = _c(theta1), _c(theta2)
    p1 = np.ascontiguousarray(perm1, dtype=np.int64)
    p2 = np.ascontiguousarray(perm2, dtype=np.int64)
    h = len(t1)
    O = np.zeros((2 * h, 2 * h))
    lib().or_mixing(h, _p(t1), _p(t2), _ip(p1), _ip(p2), _p(O))
    return O


def householder_qr(X):
    X = _c(X)
    m, n = X.shape
    Q = np.zeros((m, n)); R = np.zeros((n, n))
    lib().or_householder_qr(_p(X), m, n, n, _p(Q), n, _p(R), n)
    return Q, R


def ts_svd_tsqr(A, mix, passes=2, wp=PAPER_DROP_TOL ** 2, max_sweeps=MAX_SWEEPS):
    """Algorithm 1 (passes=1) or 2 (passes=2): (U, S, V, rank, status).
    mix = (theta1, theta2, perm1, perm2), each of length h = ceil(n / 2)."""
    A = _c(A)
    m, n = A.shape
    t1, t2 = _c(mix[0]), _c(mix[1])
    p1 = np.ascontiguousarray(mix[2], dtype=np.int64)
    p2 = np.ascontiguousarray(mix[3], dtype=np.int64)
    U = np.zeros((m, n)); S = np.zeros(n); V = np.zeros((n, n))
    r = ctypes.c_int64(0)
    st = lib().or_ts_svd_tsqr(_p(A), m, n, n, int(passes), float(wp), _p(t1), _p(t2), _ip(p1),
                              _ip(p2), int(max_sweeps), _p(U), n, _p(S), _p(V), n,
                              ctypes.byref(r))
    return U, S, V, r.value, st


def lowrank_svd_tsqr(A, k, l, iters, Omega, mix, wp=PAPER_DROP_TOL ** 2,
                     max_sweeps=MAX_SWEEPS):
    """Algorithm 7: (U m x k, S k, V n x k, rank, status); mix is the mixing
    draw for l columns (length ceil(l / 2) each)."""
    A, Omega = _c(A), _c(Omega)
    m, n = A.shape
    t1, t2 = _c(mix[0]), _c(mix[1])
    p1 = np.ascontiguousarray(mix[2], dtype=np.int64)
    p2 = np.ascontiguousarray(mix[3], dtype=np.int64)
    U = np.zeros((m, k)); S = np.zeros(k); V = np.zeros((n, k))
    r = ctypes.c_int64(0)
    st = lib().or_lowrank_svd_tsqr(_p(A), m, n, n, int(k), int(l), int(iters), _p(Omega), _p(t1),
                                   _p(t2), _ip(p1), _ip(p2), float(wp), int(max_sweeps), _p(U), k,
                                   _p(S), _p(V), k, ctypes.byref(r))
    return U, S, V, r.value, st


def col_means(A):
    A = _c(A)
    m, n = A.shape
    mu = np.zeros(n)
    lib().or_col_means(_p(A), m, n, n, _p(mu))
    return mu


def pca(A, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, max_sweeps=MAX_SWEEPS):
    """PCA of the rows of A: (mu n, U m x n, S n, V n x n, rank, status) of
    the SVD of A - 1 mu^T."""
    A = _c(A)
    m, n = A.shape
    mu = np.zeros(n); U = np.zeros((m, n)); S = np.zeros(n); V = np.zeros((n, n))
    r = ctypes.c_int64(0)
    st = lib().or_pca(_p(A), m, n, n, int(passes), int(bool(scale)), float(drop_tol),
                      int(max_sweeps), _p(mu), _p(U), n, _p(S), _p(V), n, ctypes.byref(r))
    return mu, U, S, V, r.value, st


def lowrank_svd(A, k, l, iters, Omega, drop_tol=PAPER_DROP_TOL, max_sweeps=MAX_SWEEPS,
                return_ranks=False):
    """Algorithm 8: returns (U m x k, S k, V n x k, rank, status)."""
    A, Omega = _c(A), _c(Omega)
    m, n = A.shape
    assert Omega.shape == (n, l)
    U = np.zeros((m, k)); S = np.zeros(k); V = np.zeros((n, k))
    r = ctypes.c_int64(0)
    ranks = (ctypes.c_int64 * (2 * iters + 2))()
    st = lib().or_lowrank_svd(_p(A), m, n, n, int(k), int(l), int(iters), _p(Omega),
                              float(drop_tol), int(max_sweeps), _p(U), k, _p(S), _p(V), k,
                              ctypes.byref(r), ranks)
    out = (U, S, V, r.value, st)
    if return_ranks:
        return out + (list(ranks),)
    return out


def ts_svd_backward(A, S, V, dU=None, dS=None, dV=None):
    """Thin-SVD adjoint: dA for full-rank A (m x n) with SVD (A V S^-1, S, V)."""
    A, S, V = _c(A), _c(S), _c(V)
    m, n = A.shape
    dU = np.zeros((m, n)) if dU is None else _c(dU)
    dS = np.zeros(n) if dS is None else _c(dS)
    dV = np.zeros((n, n)) if dV is None else _c(dV)
    dA = np.zeros((m, n))
    lib().or_ts_svd_backward(_p(A), m, n, n, _p(S), _p(V), n, _p(dU), n, _p(dS),
                             _p(dV), n, _p(dA), n)
    return dA


def lowrank_svd_backward(U, S, V, dU=None, dS=None, dV=None):
    """Adjoint of a rank-k SVD (U m x k, S k, V n x k): dA (m x n)."""
    U, S, V = _c(U), _c(S), _c(V)
    m, k = U.shape
    n = V.shape[0]
    nul = ctypes.POINTER(ctypes.c_double)()
    dU = _c(dU) if dU is not None else None
    dS = _c(dS) if dS is not None else None
    dV = _c(dV) if dV is not None else None
    pdU = _p(dU) if dU is not None else nul
    pdS = _p(dS) if dS is not None else nul
    pdV = _p(dV) if dV is not None else nul
    dA = np.zeros((m, n))
    lib().or_lowrank_svd_backward(_p(U), m, k, k, _p(S), _p(V), n, k, pdU, k, pdS, pdV, k,
                                  _p(dA), n)
    return dA


def orth_error(U):
    U = _c(U)
    return lib().or_orth_error(_p(U), U.shape[0], U.shape[1], U.shape[1])


def spectral_error(A, U, S, V, iters=20, seed=12345):
    """||A - U diag(S) V^T||_2 by `iters` power-method steps (Table "heads")."""
    A, U, S, V = _c(A), _c(U), _c(S), _c(V)
    m, n = A.shape
    r = S.shape[0]
    return lib().or_spectral_error(_p(A), m, n, n, _p(U), U.shape[1], _p(S), _p(V),
                                   V.shape[1], r, int(iters), int(seed))
