"""FP64 oracle of the range-finder form of LRAMM, used as a linear layer.

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Forward.  C ~ X W (X m x k, W k x n) is computed as (X Q)(Q^T W), where Q
(k x l, l = r + p) is the orthonormal range-finder basis of W: the
two-stage randomized scheme of Sec. 2.2 applied to the right operand
(Gaussian sketch Y = W Omega, Omega = Philox stream 1 of the seed, q power
iterations as in the text after Eq. (rsvderror_z), every product
re-orthonormalised).  With T = X Q (m x l) and P = Q^T W (l x n) the output
is C = QM(T P, d) (Algorithm 2: T quantised per row, P per column) or the
plain product T P when d is FP32.

Backward.  Gradients of L = <G, C> with respect to X and W for a fixed
Omega, straight-through (identity) through the quantisers -- i.e. the
gradients of the unquantised C = X Q Q^T W:
    dT = G P^T,  dP = T^T G,  dX = dT Q^T,
    dW = Q dP  +  (the path through Q),   dQ = X^T dT + W dP^T,
and dQ is carried back through the range finder: each thin QR Y = Q R
(diag R > 0) passes dY = (dQ + Q copyltu(M)) R^-T with M = -dQ^T Q (no
gradient reaches R), copyltu(M) the symmetric matrix that copies M's lower
triangle onto its upper; each product Y = W Z adds dY Z^T to dW and passes
W^T dY to Z, each product Y' = W^T Q adds Q dY'^T to dW and passes W dY'
to Q; the sketch Y0 = W Omega adds dY0 Omega^T.
"""
import numpy as np

from . import mixed
from . import philox
from . import quant

F64 = np.float64


def qr_pos(Y):
    """Thin QR with a positive diagonal in R (the unique thin QR of a full-rank Y)."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=F64), mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], R * d[:, None]


def copyltu(M):
    """Symmetric matrix with M's lower triangle (diagonal included) on both sides."""
    L = np.tril(M)
    return L + np.tril(M, -1).T


def qr_adjoint(Q, R, dQ):
    """Gradient with respect to Y of a loss that depends on Y = Q R through Q only."""
    M = -dQ.T @ Q
    B = dQ + Q @ copyltu(M)
    # B R^-T: solve  X R^T = B  for X
    return np.linalg.solve(R, B.T).T


def range_finder_chain(W, l, q, seed):
    """Q of the range finder of W (k x n) with the intermediates the backward needs.

    Returns (Q, chain) with chain = dict(Om, Q0, R0, steps=[(Zi, Rpi, Qi, Ri)]).
    """
    W = np.asarray(W, dtype=F64)
    n = W.shape[1]
    Om = philox.gaussian_matrix(seed, 1, n, l).astype(F64)
    Q0, R0 = qr_pos(W @ Om)
    Q = Q0
    steps = []
    for _ in range(q):
        Z, Rp = qr_pos(W.T @ Q)
        Qn, Rn = qr_pos(W @ Z)
        steps.append((Z, Rp, Qn, Rn))
        Q = Qn
    return Q, dict(Om=Om, Q0=Q0, R0=R0, steps=steps)


def rf_factors(X, W, r, p, q, seed):
    """T = X Q (m x l), P = Q^T W (l x n) and Q (k x l), FP64."""
    X = np.asarray(X, dtype=F64)
    W = np.asarray(W, dtype=F64)
    Q, _ = range_finder_chain(W, r + p, q, seed)
    return X @ Q, Q.T @ W, Q


def rf_forward(X, W, r, p, q, seed, prec=quant.PREC_F32, scale=quant.SCALE_ROWCOL, alpha=1.0, beta=0.0, C=None):
    """C = alpha QM(T P, prec) + beta C (FP64 result)."""
    T, P, _ = rf_factors(X, W, r, p, q, seed)
    if prec == quant.PREC_F32:
        D = T @ P
    else:
        D = mixed.qm_any(T.astype(np.float32), P.astype(np.float32), prec, scale).astype(F64)
    D = alpha * D
    if beta != 0.0:
        D = D + beta * np.asarray(C, dtype=F64)
    return D


def rf_backward(X, W, G, r, p, q, seed, alpha=1.0):
    """(dX, dW) of L = <G, alpha X Q Q^T W> (straight-through quantisers), FP64."""
    X = np.asarray(X, dtype=F64)
    W = np.asarray(W, dtype=F64)
    G = alpha * np.asarray(G, dtype=F64)
    Q, ch = range_finder_chain(W, r + p, q, seed)
    T = X @ Q
    P = Q.T @ W
    dT = G @ P.T
    dP = T.T @ G
    dX = dT @ Q.T
    dW = Q @ dP
    dQ = X.T @ dT + W @ dP.T
    Qprev = [ch["Q0"]] + [s[2] for s in ch["steps"][:-1]]
    for (Z, Rp, Qi, Ri), Qp in zip(reversed(ch["steps"]), reversed(Qprev)):
        dY = qr_adjoint(Qi, Ri, dQ)          # Y_i = W Z_i
        dW += dY @ Z.T
        dZ = W.T @ dY
        dYp = qr_adjoint(Z, Rp, dZ)          # Y'_i = W^T Q_{i-1}
        dW += Qp @ dYp.T
        dQ = W @ dYp
    dY0 = qr_adjoint(ch["Q0"], ch["R0"], dQ)  # Y_0 = W Omega
    dW += dY0 @ ch["Om"].T
    return dX, dW
