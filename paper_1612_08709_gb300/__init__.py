"""GB300-native Gram-based tall-skinny SVD and randomized low-rank SVD.

Implements the hot path of Li, Kluger & Tygert, "Randomized algorithms for
distributed computation of PCA and SVD" (arXiv:1612.08709): Algorithms 3
and 4 (Gram-based TS-SVD with one or two orthonormalisation passes) and
Algorithm 8 (randomized subspace iteration, Algorithm 5, feeding the direct
SVD, Algorithm 6), plus the thin-SVD adjoint.

Every step runs in the CUDA library libtssvd.so (include/tssvd.h); this
module only marshals torch tensors into its C ABI.  There is no CPU
fallback: if the library is missing, importing the binding raises.
"""
from ._binding import (  # noqa: F401
    TSSVD_OK, TSSVD_ENOCONV, TSSVD_RANKDEF, TSSVD_ETIMEOUT, TSSVD_ECUDA, TSSVD_ENOMEM,
    PAPER_DROP_TOL, TsSvdError, lib, library_path, ts_svd, lowrank_svd, ts_svd_backward, ts_gram,
    ts_matmul, ts_svd_batched, ts_svd_batched_workspace_size,
    ts_svd_workspace_size, lowrank_svd_workspace_size, TSSVD, exported_symbols,
    ts_pca, ts_pca_workspace_size, lowrank_svd_backward, LowRankSVD, ts_svd_tsqr,
    lowrank_svd_tsqr, TSSVD_ECOMM, ts_svd_host, ts_svd_host_workspace_size,
)
from ._rowshard import (  # noqa: F401
    ts_svd_rowshard, DistComm, row_block, reduce_fixed_order,
)
