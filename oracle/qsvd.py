"""FP64 oracle of the quantised SVD approximation of a single matrix
(Algorithm 4; Theorem 4.4 bounds its error).

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Algorithm 4: {U_k, Sigma_k, V_k} = SVD(A, k); U~_k = U_k Sigma_k; quantise
U~_k with d1 bits and V_k with d2 bits; the approximation is
A' = deq(U~_k') deq(V_k')^T.

Readings (listed in the design notes):
  * SVD(A, k) is the framework's randomized SVD (Sec. 2.2, Algorithm 1: l =
    k + p sketch columns, q power iterations, truncated to k), as everywhere
    else in LRAMM.
  * The quantiser is that of Sec. 3.1 (oracle.quant): U~_k by rows and V_k by
    rows (the columns of V_k^T), both per row (ROWCOL) or per tensor (the
    paper's a_max per matrix); MXFP4 blocks run along the rank index.
  * The paper's Theorem 4.4 is stated in expectation over an unbiased
    (dithered) quantiser; the deterministic round-to-nearest quantiser here
    satisfies its per-entry worst case |r| <= 1 / (2 lambda), so the pins use
    the triangle-inequality form
        |A' - A|_F <= |A - A_k|_F + |R_U V_k^T|_F + |U~_k R_V^T|_F + |R_U R_V^T|_F
    with |R_U V_k^T|_F = |R_U|_F (V_k orthonormal) and the per-entry bounds.
"""
import numpy as np

from . import lramm
from . import mixed
from . import quant

F64 = np.float64
F32 = np.float32


def factors(X, k, p, q, seed, stream):
    """U~_k = U_k Sigma_k (rows x k) and V_k (cols x k), FP32 storage, and sigma (FP64)."""
    U, s, V = lramm.rsvd(X, k, p, q, seed, stream)
    return (U * s[None, :]).astype(F32), V.astype(F32), s


def quantise(M, prec, scale):
    """Codes and dequantised values of M (rows quantised along the rank index)."""
    if prec == quant.PREC_F32:
        return None, np.asarray(M, F64)
    if prec == mixed.PREC_MXFP4:
        c, e = mixed.quantize_mxfp4(M)
        return (c, e), mixed.dequantize_mxfp4(c, e)
    axis = 1 if scale == quant.SCALE_ROWCOL else None
    c, _, s = quant.quantize(M, prec, axis)
    return (c, s), quant.dequantize(c, s, axis).astype(F64)


def qsvd(X, k, p, q, seed, stream, prec_u, prec_v, scale=quant.SCALE_ROWCOL):
    """Algorithm 4: returns (codes of U~_k', codes of V_k', A' in FP64, sigma)."""
    Ut, V, s = factors(X, k, p, q, seed, stream)
    cu, du = quantise(Ut, prec_u, scale)
    cv, dv = quantise(V, prec_v, scale)
    return cu, cv, du @ dv.T, s
