"""FP64 oracle of LRAMM: randomized SVD of both operands, then the quantised
factor chain of Algorithm 3.

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Passages followed (paper section / equation / algorithm):
  * Sec. 2.1: truncated SVD A' = U_r Sigma_r V_r^T.
  * Sec. 2.2: two-stage randomized scheme -- find Q with orthonormal columns
    and A ~ Q Q^* A, then factorise; Gaussian sampling for Q.
  * Algorithm 1: B = Q^* A; SVD(B) = U' Sigma V^*; U = Q U'.
  * Eq. (rsvderror_z) and the text after it: q power iterations.
  * Sec. 3.2 (LRAMM product form) and Algorithm 3: RSVD(A), RSVD(B);
    U~ = U_r Sigma_r, Z~ = Gamma_r Z_r^T; E1 = QM(V_r^T W_r, d1),
    E2 = QM(E1 Z~, d2), E3 = QM(U~ E2, d3); D = alpha E3 + beta C.

Readings (listed in the design notes):
  * The sketch has l = r + p columns (oversampling p, which the paper does
    not name); the l x cols SVD of B is truncated to r afterwards.
  * Power iterations follow Halko-Martinsson-Tropp's randomized subspace
    iteration: Q <- orth(A orth(A^T Q)), q times, every product
    re-orthonormalised.
  * orth() is the thin QR factor with a positive diagonal in R (the unique
    thin QR); it is computed here by Householder QR (LAPACK) with a sign fix.
  * The random test matrix for A is Philox stream 0 of the seed, the one for
    B stream 1; Omega is cols x l, row-major element order.
  * d_i applies to both operands of E_i.  The quantisation decisions use the
    FP32-rounded factors (the precision the factors are stored in).
"""
import numpy as np

from . import philox
from . import quant

F64 = np.float64


def orth(Y):
    """Orthonormal basis of range(Y): thin QR, sign-fixed so diag(R) > 0."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=F64), mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def range_finder(X, l, q, seed, stream):
    """Q (rows x l) with orthonormal columns, X ~ Q Q^T X (Sec. 2.2, q power steps)."""
    X = np.asarray(X, dtype=F64)
    cols = X.shape[1]
    Omega = philox.gaussian_matrix(seed, stream, cols, l).astype(F64)
    Q = orth(X @ Omega)
    for _ in range(q):
        Zh = orth(X.T @ Q)
        Q = orth(X @ Zh)
    return Q


def rsvd(X, r, p, q, seed, stream, rf=None):
    """Algorithm 1 on the range-finder basis, truncated to rank r.

    Returns U (rows x r), s (r), V (cols x r) in FP64 with X ~ U diag(s) V^T.
    rf: the range finder (default `range_finder`; oracle.sketch8 supplies
    the e4m3 one).
    """
    X = np.asarray(X, dtype=F64)
    l = r + p
    if not (1 <= r and l <= min(X.shape)):
        raise ValueError("rsvd: need 1 <= r and r + p <= min(rows, cols)")
    Q = (rf or range_finder)(X, l, q, seed, stream)
    B = Q.T @ X                                    # Algorithm 1: B = Q^* A
    Ub, s, Vbt = np.linalg.svd(B, full_matrices=False)   # SVD(B) = U' S V^*
    U = Q @ Ub[:, :r]                              # U = Q U'
    return U, s[:r], Vbt[:r, :].T


def factors(A, B, r, p, q, seed, rf=None):
    """The four Alg. 3 factors in FP32 storage: U~ (m x r), V (k x r), W (k x r),
    Z~ (r x n), with A ~ U~ V^T and B ~ W Z~."""
    U, s, V = rsvd(A, r, p, q, seed, 0, rf)
    W, g, Z = rsvd(B, r, p, q, seed, 1, rf)
    Ut = (U * s[None, :]).astype(np.float32)        # U~ = U_r Sigma_r
    Zt = (Z * g[None, :]).T.astype(np.float32)       # Z~ = Gamma_r Z_r^T
    return Ut, V.astype(np.float32), W.astype(np.float32), Zt


def chain(Ut, V, W, Zt, prec, scale=quant.SCALE_ROWCOL, alpha=1.0, beta=0.0, C=None):
    """Quantised factor chain of Algorithm 3 on given FP32 factors.

    prec = (d1, d2, d3) as quant.PREC_* codes.  Returns D in FP64.
    """
    E1 = quant.qm(np.asarray(V, np.float32).T, W, prec[0], scale)   # E1 = QM(V^T W, d1)
    E2 = quant.qm(E1, Zt, prec[1], scale)                            # E2 = QM(E1 Z~, d2)
    E3 = quant.qm(Ut, E2, prec[2], scale)                            # E3 = QM(U~ E2, d3)
    D = alpha * E3.astype(F64)
    if beta != 0.0:
        D = D + beta * np.asarray(C, dtype=F64)
    return D


def lramm(A, B, r, p, q, seed, prec, scale=quant.SCALE_ROWCOL, alpha=1.0, beta=0.0, C=None, rf=None):
    """LRAMM (Algorithm 3): D = alpha * E3 + beta * C, D ~ alpha * A B + beta * C."""
    Ut, V, W, Zt = factors(A, B, r, p, q, seed, rf)
    return chain(Ut, V, W, Zt, prec, scale, alpha, beta, C)


def exact_product(A, B):
    """C = A B in FP64 (the reference the approximation error is measured against)."""
    return np.asarray(A, dtype=F64) @ np.asarray(B, dtype=F64)


def rel_fro(X, Ref):
    """||X - Ref||_F / ||Ref||_F in FP64 (the E_r measure of Eq. (er_qgemm))."""
    X = np.asarray(X, dtype=F64)
    Ref = np.asarray(Ref, dtype=F64)
    den = np.linalg.norm(Ref)
    return float(np.linalg.norm(X - Ref) / den) if den > 0 else float(np.linalg.norm(X))
