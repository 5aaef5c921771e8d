"""FP64 oracle of the E4M3 range finder: the sketch and power iterations of
the randomized SVD (Sec. 2.2, q power steps) with every product of the
operand X taken on FP8 e4m3 codes as a quantised product of Algorithm 2.

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Readings (the paper runs its RSVD in full precision and names low-precision
range finders only as future work; each reading is listed in the design
notes):
  * Every product X B or X^T B of the range finder (the sketch X Omega,
    X^T Q and X Z^ of the power iterations) is QM(L R, e4m3) of Algorithm 2
    with the left operand (X, or X^T) quantised per row and the right
    operand (the l-column matrix) per column: fp32(fp32(acc) fp32(sL sR))
    with acc the exact code sum (oracle.quant.qm).  Codes are decided in
    FP32 on the FP32 values of X and of the l-column matrix.
  * The orthonormalisations, the projection B = Q^T X (unquantised) and the
    small SVD are those of oracle.lramm.
"""
import numpy as np

from . import lramm
from . import philox
from . import quant

F64 = np.float64
F32 = np.float32


def qproduct_e4m3(L, R):
    """QM(L R, e4m3) with L per row and R per column, as FP64 values of the FP32 result."""
    return quant.qm(np.asarray(L, F32), np.asarray(R, F32), quant.PREC_E4M3, quant.SCALE_ROWCOL).astype(F64)


def range_finder_e4m3(X, l, q, seed, stream, product=qproduct_e4m3):
    """Q (rows x l) orthonormal: the range finder of oracle.lramm with `product`
    in place of every product of X (np.matmul gives lramm.range_finder back)."""
    X = np.asarray(X, dtype=F64)
    Omega = philox.gaussian_matrix(seed, stream, X.shape[1], l).astype(F64)
    Q = lramm.orth(product(X, Omega))
    for _ in range(q):
        Zh = lramm.orth(product(X.T, Q))
        Q = lramm.orth(product(X, Zh))
    return Q


def rsvd_e4m3(X, r, p, q, seed, stream):
    """Algorithm 1 on the e4m3 range finder's basis, truncated to rank r."""
    return lramm.rsvd(X, r, p, q, seed, stream, rf=range_finder_e4m3)
