"""The algebra behind the M-only small SVD of the quantised chains, in FP64.

With B^T = P R (thin QR by two CholeskyQR passes: B^T = P1 R1, P1 = P R2,
R = R2 R1) and R^T = U_s Sigma V_s^T, the right singular factors satisfy
P V_s = B^T U_s Sigma^-1 = P1 (R1 U_s Sigma^-1), so the library forms them
from P1 and an l x r factor without accumulating V_s or forming P.  These
tests check that identity, that the rank-r products agree, and that the
plausible slip of pairing P1 with R instead of R1 is caught.
"""
import numpy as np
import pytest


def _chol_qr_pass(X):
    L = np.linalg.cholesky(X.T @ X)
    return np.linalg.solve(L, X.T).T, L.T          # X = Q R with R = L^T


def _setup(k=300, l=40, r=32, seed=5):
    """B^T (k x l, graded spectrum) split as B^T = P1 R1 with P1 far from
    orthonormal (P1 = P R2, R2 an upper-triangular factor a few percent
    from I, as one FP32 CholeskyQR pass leaves it at kappa ~ 10^3), the
    second pass P1 = P R2, and R = R2 R1."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((k, l)))
    V, _ = np.linalg.qr(rng.standard_normal((l, l)))
    sig = (1.0 + np.arange(l)) ** -1.0
    Bt = (U * sig) @ V.T
    Q, Rq = _chol_qr_pass(Bt)
    E = np.eye(l) + 0.05 * np.triu(rng.standard_normal((l, l)))
    P1, R1 = Q @ E, np.linalg.solve(E, Rq)            # B^T = P1 R1 exactly
    P, R2 = _chol_qr_pass(P1)
    R = R2 @ R1
    Us, S, Vst = np.linalg.svd(R.T)
    return Bt, P1, R1, P, R, Us, S, Vst.T, r


def test_right_factors_from_p1():
    Bt, P1, R1, P, R, Us, S, Vs, r = _setup()
    ref = P @ Vs[:, :r]
    via_p1 = P1 @ (R1 @ (Us[:, :r] / S[:r]))
    via_bt = Bt @ (Us[:, :r] / S[:r])
    assert np.linalg.norm(via_p1 - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(via_bt - ref) <= 1e-10 * np.linalg.norm(ref)


def test_rank_r_products_agree():
    """B = U_s Sigma (P V_s)^T: the truncated products of both forms agree."""
    Bt, P1, R1, P, R, Us, S, Vs, r = _setup()
    left = Us[:, :r] * S[:r]
    ref = left @ (P @ Vs[:, :r]).T
    mo = left @ (P1 @ (R1 @ (Us[:, :r] / S[:r]))).T
    assert np.linalg.norm(mo - ref) <= 1e-10 * np.linalg.norm(ref)
    # the full-rank product reproduces B = (B^T)^T
    full = (Us * S) @ (P1 @ (R1 @ (Us / S))).T
    assert np.linalg.norm(full - Bt.T) <= 1e-10 * np.linalg.norm(Bt)


def test_pairing_p1_with_r_is_caught():
    Bt, P1, R1, P, R, Us, S, Vs, r = _setup()
    ref = P @ Vs[:, :r]
    wrong = P1 @ (R @ (Us[:, :r] / S[:r]))
    assert np.linalg.norm(wrong - ref) > 1e-6 * np.linalg.norm(ref)
