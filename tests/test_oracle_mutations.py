"""Plausible mistakes planted in the oracle (on the CPU) must fail a pin.

Each case monkeypatches one oracle function with a broken copy and runs the
pin that is meant to catch it.  A pin that passed on a broken oracle would
mean the oracle is not really pinned.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import philox as P
from oracle import quant as Qn
from oracle import lramm as Lr
from tests import pins


def _philox_rounds(n_rounds, bump=True, swap=False):
    def f(counters, key):
        c = np.asarray(counters, dtype=np.uint32).astype(np.uint64)
        c0, c1, c2, c3 = c[:, 0], c[:, 1], c[:, 2], c[:, 3]
        k0, k1 = int(key[0]), int(key[1])
        m0, m1 = (P.M1, P.M0) if swap else (P.M0, P.M1)
        for rnd in range(n_rounds):
            if rnd > 0 and bump:
                k0 = (k0 + P.W0) & 0xFFFFFFFF
                k1 = (k1 + P.W1) & 0xFFFFFFFF
            p0, p1 = m0 * c0, m1 * c2
            c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0), p1 & P.MASK32,
                              (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1), p0 & P.MASK32)
        return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)
    return f


@pytest.mark.parametrize("mut", [dict(n_rounds=9), dict(n_rounds=10, bump=False),
                                 dict(n_rounds=10, swap=True)])
def test_philox_mutations_caught(monkeypatch, mut):
    monkeypatch.setattr(P, "philox4x32_10", _philox_rounds(**mut))
    try:
        with pytest.raises(AssertionError):
            pins.pin_philox_curand(P)
    except RuntimeError as e:
        pytest.skip(str(e))


def test_box_muller_missing_factor_two_caught(monkeypatch):
    def bad(x, y):
        x = np.asarray(x, dtype=np.uint64)
        y = np.asarray(y, dtype=np.uint64)
        u1 = ((x >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
        u2 = (2.0 * (y >> np.uint64(9)).astype(np.float64) + 1.0) * 2.0 ** -24
        rad = np.sqrt(-np.log(u1))                      # dropped factor 2
        return rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)
    monkeypatch.setattr(P, "box_muller", bad)
    with pytest.raises(AssertionError):
        pins.pin_gaussian_stats(P)


def _quantize_variant(rounding="rne", dmax=None, scale_inv=False):
    def f(X, prec, axis):
        X = np.asarray(X, dtype=np.float32)
        amax = Qn.absmax_groups(X, axis)
        D = np.float32(dmax if dmax is not None else (127 if prec == Qn.PREC_INT8 else 7))
        with np.errstate(divide="ignore", invalid="ignore"):
            lam = np.where(amax > 0, D / amax, np.float32(0)).astype(np.float32)
        s = (lam if scale_inv else amax / D).astype(np.float32)
        lb = lam[:, None] if axis == 1 else (lam[None, :] if axis == 0 else lam[0])
        y = (X * lb).astype(np.float64)
        if rounding == "floor":
            c = np.floor(y)
        elif rounding == "away":
            c = np.sign(y) * np.floor(np.abs(y) + 0.5)
        else:
            c = np.rint(y)
        return np.clip(c, -float(D), float(D)), lam, s
    return f


@pytest.mark.parametrize("mut", [dict(rounding="floor"), dict(rounding="away"), dict(dmax=128)])
def test_quantiser_mutations_caught_by_golden(monkeypatch, mut):
    monkeypatch.setattr(Qn, "quantize", _quantize_variant(**mut))
    with pytest.raises(AssertionError):
        pins.pin_quant_golden(Qn)


def test_dequant_scale_inverted_caught(monkeypatch):
    monkeypatch.setattr(Qn, "quantize", _quantize_variant(scale_inv=True))
    with pytest.raises(AssertionError):
        pins.pin_quant_bounds(Qn)


def test_qm_right_scale_mode_ignored_caught(monkeypatch):
    real = Qn.quantize

    def bad_qm(L, R, prec, scale=Qn.SCALE_ROWCOL):
        # right operand always quantised with one per-tensor scale
        cl, _, sl = real(L, prec, 1 if scale == Qn.SCALE_ROWCOL else None)
        cr, _, sr = real(R, prec, None)
        acc = Qn.code_product(cl, cr)
        sl_b = sl[:, None] if scale == Qn.SCALE_ROWCOL else sl[0]
        return (acc.astype(np.float32) * (sl_b * sr[0]).astype(np.float32)).astype(np.float32)
    monkeypatch.setattr(Qn, "qm", bad_qm)
    with pytest.raises(AssertionError):
        pins.pin_qm_bruteforce(Qn)


def test_qm_dequant_by_lambda_caught(monkeypatch):
    real = Qn.quantize

    def bad_qm(L, R, prec, scale=Qn.SCALE_ROWCOL):
        cl, ll, _ = real(L, prec, 1)
        cr, lr_, _ = real(R, prec, 0)
        acc = Qn.code_product(cl, cr)
        return (acc.astype(np.float32) * (ll[:, None] * lr_[None, :]).astype(np.float32)).astype(np.float32)
    monkeypatch.setattr(Qn, "qm", bad_qm)
    with pytest.raises(AssertionError):
        pins.pin_qm_bruteforce(Qn)


def test_e4m3_truncation_caught(monkeypatch):
    def trunc(v):
        v = np.asarray(v, dtype=np.float64)
        a = np.abs(v)
        with np.errstate(divide="ignore"):
            e = np.clip(np.floor(np.log2(np.where(a > 0, a, 1.0))), -6, 8)
        q = np.exp2(e - 3)
        return np.sign(v) * np.minimum(np.floor(a / q) * q, 448.0)
    monkeypatch.setattr(Qn, "round_e4m3", trunc)
    with pytest.raises(AssertionError):
        pins.pin_e4m3(Qn)


def test_orth_without_sign_fix_caught(monkeypatch):
    def bad(Y):
        Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
        return -Q
    monkeypatch.setattr(Lr, "orth", bad)
    with pytest.raises(AssertionError):
        pins.pin_orth(Lr)


def test_rsvd_skipping_small_svd_caught(monkeypatch):
    def bad(X, r, p, q, seed, stream):
        Q = Lr.range_finder(X, r + p, q, seed, stream)
        B = Q.T @ X
        Ub, s, Vbt = np.linalg.svd(B, full_matrices=False)
        return Q[:, :r], s[:r], Vbt[:r].T                # U' dropped
    monkeypatch.setattr(Lr, "rsvd", bad)
    with pytest.raises(AssertionError):
        pins.pin_rsvd_exact_rank(Lr, workloads)


def test_rsvd_wrong_power_step_caught(monkeypatch):
    real_rf = Lr.range_finder

    def bad_rf(X, l, q, seed, stream):
        Q = real_rf(X, l, 0, seed, stream)
        for _ in range(q):
            Q = Lr.orth(X @ (X.T @ X) @ Q[: X.shape[1]] if X.shape[0] >= X.shape[1] else X @ Q[: X.shape[1]])
        return Q
    monkeypatch.setattr(Lr, "range_finder", bad_rf)
    with pytest.raises((AssertionError, ValueError)):
        pins.pin_rsvd_bounds(Lr, workloads, trials=20)


def test_chain_missing_sigma_caught(monkeypatch):
    def bad_factors(A, B, r, p, q, seed):
        U, s, V = Lr.rsvd(A, r, p, q, seed, 0)
        W, g, Z = Lr.rsvd(B, r, p, q, seed, 1)
        return U.astype(np.float32), V.astype(np.float32), W.astype(np.float32), (Z * g).T.astype(np.float32)
    monkeypatch.setattr(Lr, "factors", bad_factors)
    with pytest.raises(AssertionError):
        pins.pin_lramm_factor_identity(Lr, workloads, Qn)


def test_chain_transposed_e1_caught(monkeypatch):
    def bad_chain(Ut, V, W, Zt, prec, scale=Qn.SCALE_ROWCOL, alpha=1.0, beta=0.0, C=None):
        E1 = Qn.qm(np.asarray(W, np.float32).T, V, prec[0], scale)   # W^T V instead of V^T W
        E2 = Qn.qm(E1, Zt, prec[1], scale)
        return alpha * Qn.qm(Ut, E2, prec[2], scale).astype(np.float64)
    monkeypatch.setattr(Lr, "chain", bad_chain)
    with pytest.raises(AssertionError):
        pins.pin_lramm_factor_identity(Lr, workloads, Qn)


# ---------------------------------------------------------------- range-finder form
from oracle import rf as Rf


def _qr_adjoint_variant(kind):
    def f(Q, R, dQ):
        M = -dQ.T @ Q
        if kind == "no_copyltu":
            B = dQ
        elif kind == "upper":
            B = dQ + Q @ (np.triu(M) + np.triu(M, 1).T)
        else:  # sign of M
            B = dQ - Q @ Rf.copyltu(M)
        return np.linalg.solve(R, B.T).T
    return f


@pytest.mark.parametrize("kind", ["no_copyltu", "upper", "sign"])
def test_qr_adjoint_mutations_caught(monkeypatch, kind):
    monkeypatch.setattr(Rf, "qr_adjoint", _qr_adjoint_variant(kind))
    with pytest.raises(AssertionError):
        pins.pin_qr_adjoint_fd(Rf)


def test_rf_backward_missing_direct_term_caught(monkeypatch):
    orig = Rf.rf_backward

    def bad(X, W, G, r, p, q, seed, alpha=1.0):
        dX, dW = orig(X, W, G, r, p, q, seed, alpha)
        Q, _ = Rf.range_finder_chain(W, r + p, q, seed)
        return dX, dW - Q @ ((X @ Q).T @ (alpha * G))    # drop dW's term through P = Q^T W
    monkeypatch.setattr(Rf, "rf_backward", bad)
    with pytest.raises(AssertionError):
        pins.pin_rf_gradients_fd(Rf)


def test_rf_backward_missing_dq_term_caught(monkeypatch):
    """dQ without the W dP^T term (the dependence of P = Q^T W on Q)."""
    src_qr_adjoint = Rf.qr_adjoint

    def bad(X, W, G, r, p, q, seed, alpha=1.0):
        X = np.asarray(X, dtype=float); W = np.asarray(W, dtype=float); G = alpha * np.asarray(G, dtype=float)
        Q, ch = Rf.range_finder_chain(W, r + p, q, seed)
        T = X @ Q; P = Q.T @ W
        dT = G @ P.T; dP = T.T @ G
        dX = dT @ Q.T
        dW = Q @ dP
        dQ = X.T @ dT                      # missing + W @ dP.T
        Qprev = [ch["Q0"]] + [st[2] for st in ch["steps"][:-1]]
        for (Z, Rp, Qi, Ri), Qp in zip(reversed(ch["steps"]), reversed(Qprev)):
            dY = src_qr_adjoint(Qi, Ri, dQ)
            dW += dY @ Z.T
            dYp = src_qr_adjoint(Z, Rp, W.T @ dY)
            dW += Qp @ dYp.T
            dQ = W @ dYp
        dW += src_qr_adjoint(ch["Q0"], ch["R0"], dQ) @ ch["Om"].T
        return dX, dW
    monkeypatch.setattr(Rf, "rf_backward", bad)
    with pytest.raises(AssertionError):
        pins.pin_rf_gradients_fd(Rf)


# ---------------------------------------------------------------- MXFP4, residuals, lead / tail
from oracle import mixed as Mx  # noqa: E402


def test_e2m1_ties_away_caught(monkeypatch):
    def bad(v):
        v = np.asarray(v, dtype=np.float64)
        a = np.abs(v)
        with np.errstate(divide="ignore"):
            e = np.clip(np.floor(np.log2(np.where(a > 0, a, 1.0))), 0, 2)
        q = np.exp2(e - 1)
        return np.sign(v) * np.minimum(np.floor(a / q + 0.5) * q, 6.0)     # ties away from zero
    monkeypatch.setattr(Mx, "round_e2m1", bad)
    with pytest.raises(AssertionError):
        pins.pin_e2m1(Mx)


def test_mx_floor_exponent_caught(monkeypatch):
    def bad(amax):
        amax = np.asarray(amax, dtype=np.float32)
        y = (amax / np.float32(6.0)).astype(np.float32)
        m, E = np.frexp(y.astype(np.float64))
        e = np.where(amax > 0, E - 1, -127)                                # floor(log2 y)
        return np.clip(e, -127, 127).astype(np.int64)
    monkeypatch.setattr(Mx, "mx_exponent", bad)
    with pytest.raises(AssertionError):
        pins.pin_mx_scale_rule(Mx)


def test_mx_product_wrong_block_scale_caught(monkeypatch):
    good = Mx.mx_product

    def bad(cl, el, cr, er):
        return good(cl, el, cr, np.roll(er, 1, axis=1))                   # right scales one block off
    monkeypatch.setattr(Mx, "mx_product", bad)
    with pytest.raises(AssertionError):
        pins.pin_mx_product_bruteforce(Mx)


def test_hilo_without_residual_caught(monkeypatch):
    def bad(X, prec, axis):
        X = np.asarray(X, dtype=np.float32)
        c_hi, _, s_hi = Qn.quantize(X, prec, axis)
        c_lo, _, s_lo = Qn.quantize(X, prec, axis)                         # quantises x again, not x - deq(hi)
        return (c_hi, s_hi), (c_lo, s_lo)
    monkeypatch.setattr(Mx, "quantize_hilo", bad)
    with pytest.raises(AssertionError):
        pins.pin_hilo_residual(Mx, Qn)


def test_lead_tail_missing_residual_term_caught(monkeypatch):
    good = Mx._qm_codes
    calls = {"n": 0}

    def bad(cl, sl, cr, sr, ax_l, ax_r):
        calls["n"] += 1
        out = good(cl, sl, cr, sr, ax_l, ax_r)
        return out * 0 if calls["n"] % 3 == 2 else out                     # the lo.hi term lost
    monkeypatch.setattr(Mx, "_qm_codes", bad)
    with pytest.raises(AssertionError):
        pins.pin_lead_tail(Mx, Qn)


# Algorithm 4
def test_qsvd_missing_sigma_caught(monkeypatch):
    from oracle import qsvd as Qs

    def bad(X, k, p, q, seed, stream):
        U, s, V = Lr.rsvd(X, k, p, q, seed, stream)
        return U.astype(np.float32), V.astype(np.float32), s     # U_k instead of U_k Sigma_k
    monkeypatch.setattr(Qs, "factors", bad)
    with pytest.raises(AssertionError):
        pins.pin_qsvd_unquantised(Qs, Lr, workloads, Qn)


def test_qsvd_v_scaled_by_columns_caught(monkeypatch):
    from oracle import qsvd as Qs
    orig = Qs.quantise

    def bad(M, prec, scale):
        if prec in (Qn.PREC_INT8, Qn.PREC_INT4) and scale == Qn.SCALE_ROWCOL and M.shape[0] == 17:
            c, _, s = Qn.quantize(M, prec, 0)                     # one scale per rank index
            return (c, s), Qn.dequantize(c, s, 0).astype(np.float64)
        return orig(M, prec, scale)
    monkeypatch.setattr(Qs, "quantise", bad)
    with pytest.raises(AssertionError):
        pins.pin_qsvd_codes_bruteforce(Qs, Qn)


def test_qsvd_bit_widths_swapped_caught(monkeypatch):
    from oracle import qsvd as Qs
    orig = Qs.qsvd

    def bad(X, k, p, q, seed, stream, prec_u, prec_v, scale=Qn.SCALE_ROWCOL):
        return orig(X, k, p, q, seed, stream, prec_v, prec_u, scale)
    monkeypatch.setattr(Qs, "qsvd", bad)
    with pytest.raises(AssertionError):
        pins.pin_qsvd_codes_bruteforce(Qs, Qn)


def test_qsvd_floor_rounding_caught(monkeypatch):
    from oracle import qsvd as Qs

    def bad(M, prec, scale):
        if prec == Qn.PREC_F32:
            return None, np.asarray(M, np.float64)
        M = np.asarray(M, np.float32)
        D = np.float32(Qn.qmax(prec))
        amax = np.max(np.abs(M), axis=1).astype(np.float32)
        lam = (D / amax).astype(np.float32)
        c = np.clip(np.floor((M * lam[:, None]).astype(np.float64)), -D, D)   # truncation, not nearest
        s = (amax / D).astype(np.float32)
        return (c, s), (c * s[:, None]).astype(np.float32).astype(np.float64)
    monkeypatch.setattr(Qs, "quantise", bad)
    with pytest.raises(AssertionError):
        pins.pin_qsvd_error_bounds(Qs, workloads, Qn)


# E4M3 range finder
def test_rf_e4m3_left_per_column_caught(monkeypatch):
    from oracle import sketch8 as S8

    def bad(L, R):
        Lq = np.asarray(L, np.float32)
        c, _, s = Qn.quantize(Lq, Qn.PREC_E4M3, 0)                 # left operand per column
        cr, _, sr = Qn.quantize(np.asarray(R, np.float32), Qn.PREC_E4M3, 0)
        deq = Qn.dequantize(c, s, 0).astype(np.float64)
        return (deq @ Qn.dequantize(cr, sr, 0).astype(np.float64)).astype(np.float32).astype(np.float64)
    monkeypatch.setattr(S8, "qproduct_e4m3", bad)
    with pytest.raises(AssertionError):
        pins.pin_rf_e4m3_product(S8, Qn)


def test_rf_e4m3_power_step_on_x_caught(monkeypatch):
    from oracle import sketch8 as S8
    from oracle import philox as Ph

    def bad(X, l, q, seed, stream, product=S8.qproduct_e4m3):
        X = np.asarray(X, dtype=np.float64)
        Om = Ph.gaussian_matrix(seed, stream, X.shape[1], l).astype(np.float64)
        Q = Lr.orth(product(X, Om))
        for _ in range(q):
            Q = Lr.orth(product(X, Om))          # the power step re-sketches instead of using X^T Q
        return Q
    monkeypatch.setattr(S8, "range_finder_e4m3", bad)
    with pytest.raises(AssertionError):
        pins.pin_rf_e4m3_structure(S8, Lr, workloads)
