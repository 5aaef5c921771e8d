"""Element-wise error bounds for GPU products formed from the same codes as
the oracle's (test helper; imports the oracle, never the CUDA path).

Both sides quantise identical FP32 inputs with the same FP32 decisions
(Eqs. get_lambda, Quantization), so their codes and scales agree bit for
bit; they differ only in how code products and terms are summed: FP32 on
the GPU (tensor-core or SIMT accumulation, FP32 adds of the terms of a lead /
tail E3), exact or FP64 in the oracle.  With u = 2^-24, a sum of K terms
accumulated in FP32 in any order is within (K - 1) u sum |terms| of the
exact sum, and a later FP32 rounding adds u |value|.

A chain requantises its intermediate results (E1, E2; Algorithm 3), so the
GPU's FP32 rounding of E1 could move one of E2's codes across a rounding
boundary.  `assert_same_codes` proves that it cannot for the inputs at hand:
every pre-rounding value y = fp32(x lambda) of the oracle sits farther from
its nearest boundary than the GPU's value can be away from it.
"""
import numpy as np

import oracle

U = 2.0 ** -24
F32 = np.float32
F64 = np.float64
Q = oracle.quant


def _axis(side, scale):
    """Scale groups: the left operand per row, the right per column (ROWCOL), else per tensor."""
    if scale == Q.SCALE_TENSOR:
        return None
    return 1 if side == "left" else 0


def _bcast(v, axis):
    v = np.asarray(v, dtype=F64)
    if axis is None:
        return v[0]
    return v[:, None] if axis == 1 else v[None, :]


def prerounding(X, prec, axis):
    """(y, lam, s): y = fp32(x * lambda) as the quantiser forms it before rounding."""
    X = np.asarray(X, dtype=F32)
    _, lam, s = Q.quantize(X, prec, axis)
    lam_b = np.asarray(lam, F32)[0] if axis is None else (
        np.asarray(lam, F32)[:, None] if axis == 1 else np.asarray(lam, F32)[None, :])
    return (X * lam_b).astype(F32).astype(F64), np.asarray(lam, F64), np.asarray(s, F64)


def boundary_distance(y, prec):
    """Distance of each y to the nearest rounding boundary of its code grid
    (half-integers for INT8 / INT4, midpoints of the e4m3 grid for E4M3);
    entries past the saturation point are never near one (inf)."""
    a = np.abs(np.asarray(y, dtype=F64))
    if prec in (Q.PREC_INT8, Q.PREC_INT4):
        d = np.abs(a - (np.floor(a) + 0.5))
        return np.where(a >= Q.qmax(prec) + 0.5, np.inf, d)
    # the grid value g that a rounds to and its two neighbours; the rounding
    # boundaries are the midpoints between them
    g = np.abs(Q.round_e4m3(a))
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(g > 0, g, 1.0)))
    e = np.clip(e, -6, 8)
    q = np.exp2(e - 3)                                  # spacing above g
    q_dn = np.where((g == np.exp2(e)) & (e > -6), q / 2, q)   # spacing below a binade's first value
    q = np.where(g > 0, q, 2.0 ** -9)
    q_dn = np.where(g > 0, q_dn, 2.0 ** -9)
    d = np.minimum(g + q / 2 - a, a - (g - q_dn / 2))
    # saturation: every value from 448 up rounds to 448
    return np.where(a >= Q.E4M3_MAX, np.inf, d)


def assert_same_codes(X_ref, err, prec, axis, what):
    """X_ref (the oracle's FP32 values) and a GPU copy within `err`
    (element-wise) quantise to the same codes: the GPU's a_max moves lambda by
    at most (max err in the group) / a_max relative (+ one rounding), so y
    moves by at most lambda err + |y| (that + 2u); every boundary distance of
    y_ref must exceed that."""
    X_ref = np.asarray(X_ref, dtype=F32)
    err = np.broadcast_to(np.asarray(err, dtype=F64), X_ref.shape)
    y, lam, s = prerounding(X_ref, prec, axis)
    amax = Q.absmax_groups(X_ref, axis).astype(F64)
    if axis is None:
        rel = err.max() / max(amax[0], 1e-300) + 2 * U
        lam_b, rel_b = lam[0], rel
    else:
        emax = err.max(axis=axis)
        rel = emax / np.where(amax > 0, amax, 1e-300) + 2 * U
        lam_b = _bcast(lam, axis)
        rel_b = _bcast(rel, axis)
    move = lam_b * err + np.abs(y) * rel_b + 2 * U * np.abs(y)
    dist = boundary_distance(y, prec)
    bad = ~(dist > move)
    assert not bad.any(), "%s: %d values could round to another code (min margin %.3g code units)" % (
        what, int(bad.sum()), float(np.min(dist - move)))


def qm_terms(L, R, prec, scale=Q.SCALE_ROWCOL):
    """(value, magnitude) of the oracle's QM(L R, prec): value = fp32(fp32(acc) *
    fp32(sL sR)) as in oracle.quant.qm, magnitude = sum_k |cL||cR| sL sR (FP64)."""
    L = np.asarray(L, dtype=F32)
    R = np.asarray(R, dtype=F32)
    ax_l, ax_r = _axis("left", scale), _axis("right", scale)
    cl, _, sl = Q.quantize(L, prec, ax_l)
    cr, _, sr = Q.quantize(R, prec, ax_r)
    sprod = (np.asarray(_bcast(sl, ax_l), F32) * np.asarray(_bcast(sr, ax_r), F32)).astype(F32).astype(F64)
    mag = (np.abs(cl) @ np.abs(cr)) * sprod
    return Q.qm(L, R, prec, scale).astype(F64), mag


def qm_bound(mag, ref, K):
    """|GPU - oracle| for one QM on identical codes: the FP32 sum of K code
    products (K u magnitude), one rounding of the accumulator and one of the
    dequantised product (2u |value|), plus the tiniest subnormal step."""
    return K * U * mag + 2.0 * U * np.abs(ref) + 1e-38


def f32_product_bound(A, B):
    """|fp32 product - exact| <= K u |A||B| (+ one rounding) for FP32 A (M x K), B (K x N)."""
    A = np.abs(np.asarray(A, dtype=F64))
    B = np.abs(np.asarray(B, dtype=F64))
    return (A.shape[1] + 1) * U * (A @ B)


def _group_rel(err, X, axis):
    """Relative bound on the change of each scale group's a_max (hence its
    scale) when X moves by at most err element-wise, broadcast over X."""
    X = np.asarray(X, dtype=F32)
    err = np.broadcast_to(np.asarray(err, dtype=F64), X.shape)
    amax = Q.absmax_groups(X, axis).astype(F64)
    safe = np.where(amax > 0, amax, np.inf)
    if axis is None:
        return err.max() / safe[0] + 2 * U
    return _bcast(err.max(axis=axis) / safe + 2 * U, axis)


def stage(Lref, Lerr, Rref, Rerr, prec, scale=Q.SCALE_ROWCOL):
    """One product of a chain, (oracle value, element-wise bound on the GPU's
    distance from it) given inputs the GPU holds within Lerr / Rerr of the
    oracle's.  prec 0: FP32 product; else QM(L R, prec) (Algorithm 2) after
    proving that both operands quantise to the oracle's codes."""
    Lref = np.asarray(Lref, dtype=F32)
    Rref = np.asarray(Rref, dtype=F32)
    K = Lref.shape[1]
    aL, aR = np.abs(Lref.astype(F64)), np.abs(Rref.astype(F64))
    Lerr_b = np.broadcast_to(np.asarray(Lerr, dtype=F64), Lref.shape)
    Rerr_b = np.broadcast_to(np.asarray(Rerr, dtype=F64), Rref.shape)
    if prec == Q.PREC_F32:
        # |Lg Rg - L R| <= |L||dR| + |dL||R| + |dL||dR|, plus the FP32 sum of
        # K products of the GPU's inputs and one rounding
        val = Q.qm(Lref, Rref, prec).astype(F64)
        err = (aL @ Rerr_b + Lerr_b @ aR + Lerr_b @ Rerr_b
               + (K + 1) * U * ((aL + Lerr_b) @ (aR + Rerr_b)) + U * np.abs(val))
        return val, err
    ax_l, ax_r = _axis("left", scale), _axis("right", scale)
    if np.any(Lerr_b > 0):
        assert_same_codes(Lref, Lerr_b, prec, ax_l, "left operand")
    if np.any(Rerr_b > 0):
        assert_same_codes(Rref, Rerr_b, prec, ax_r, "right operand")
    val, mag = qm_terms(Lref, Rref, prec, scale)
    rel = 0.0
    if np.any(Lerr_b > 0):
        rel = rel + _group_rel(Lerr_b, Lref, ax_l)
    if np.any(Rerr_b > 0):
        rel = rel + _group_rel(Rerr_b, Rref, ax_r)
    # integer codes: exact sums on both sides, so identical codes and scales
    # give identical values; E4M3 codes: the FP32 accumulation bound
    acc = 0.0 if prec in (Q.PREC_INT8, Q.PREC_INT4) else qm_bound(mag, val, K)
    err = acc + np.abs(val) * (rel * 1.0001 + (2 * U if np.any(rel) else 0.0))
    return val, err


def chain_bound(Ut, Vt, Wt, Zt, prec, scale=Q.SCALE_ROWCOL):
    """Algorithm 3's chain E1 = QM(V^T W), E2 = QM(E1 Z~), E3 = QM(U~ E2) on
    FP32 factors given as the GPU takes them (Ut m x r, Vt r x k, Wt r x k,
    Zt n x r): (the oracle's E3, its element-wise bound for the GPU)."""
    Vt = np.asarray(Vt, dtype=F32)
    Wt = np.asarray(Wt, dtype=F32)
    Zt = np.asarray(Zt, dtype=F32)
    E1, e1 = stage(Vt, 0.0, Wt.T, 0.0, prec[0], scale)
    E2, e2 = stage(E1.astype(F32), e1, Zt.T, 0.0, prec[1], scale)
    E3, e3 = stage(np.asarray(Ut, F32), 0.0, E2.astype(F32), e2, prec[2], scale)
    return E3, e3


def lead_tail_bound(Ut, Vt, Wt, Zt, prec, lead, lead_prec, lead_split, scale=Q.SCALE_ROWCOL, alpha=1.0, beta=0.0,
                    C=None):
    """Element-wise bound for the GPU's lead / tail chain (E3 = the lead's
    8-bit terms with split-precision residuals + the tail in prec[2]; the
    lead / tail reading of the 8192 recipe) on the oracle's value, for
    integer E1 and E2 (bit-identical on both sides, so every lead code is
    too).  Lead terms: exact integer sums, identical FP32 values.  Tail:
    MXFP4 (FP32 accumulation of the exact element products), E4M3 (FP32
    accumulation), FP32 (FP32 product) or integer (exact).  The terms are
    added in FP32 on the GPU, in FP64 by the oracle."""
    MX = oracle.mixed
    Ut = np.asarray(Ut, dtype=F32)
    E1, e1 = stage(np.asarray(Vt, F32), 0.0, np.asarray(Wt, F32).T, 0.0, prec[0], scale)
    E2, e2 = stage(E1.astype(F32), e1, np.asarray(Zt, F32).T, 0.0, prec[1], scale)
    assert not np.any(e2), "lead_tail_bound needs integer E1 and E2"
    E2 = E2.astype(F32)
    r = Ut.shape[1]
    lead = min(lead, r)
    ax_l, ax_r = _axis("left", scale), _axis("right", scale)
    mags, err = [], 0.0
    if lead > 0:
        (uh, suh), (ul, sul) = MX.quantize_hilo(Ut[:, :lead], lead_prec, ax_l)
        (eh, seh), (el, sel) = MX.quantize_hilo(E2[:lead, :], lead_prec, ax_r)
        pairs = [(uh, suh, eh, seh)]
        if lead_split >= 1:
            pairs.append((ul, sul, eh, seh))
        if lead_split >= 2:
            pairs.append((uh, suh, el, sel))
        for cl, sl, cr, sr in pairs:
            sprod = (np.asarray(_bcast(sl, ax_l), F32) * np.asarray(_bcast(sr, ax_r), F32)).astype(F32)
            mag = (np.abs(cl) @ np.abs(cr)) * sprod.astype(F64)
            mags.append(mag)
            if lead_prec not in (Q.PREC_INT8, Q.PREC_INT4):
                err = err + qm_bound(mag, mag, lead)
    if lead < r:
        Ut_t, E2_t = Ut[:, lead:], E2[lead:, :]
        Kt = r - lead
        if prec[2] == MX.PREC_MXFP4:
            # the GPU sums the tail's Kt element products (exact BF16 values
            # code x 2^e) in FP32 on the tensor cores; the oracle sums each
            # 32-block exactly and the blocks in FP64, then rounds once
            cl, el_ = MX.quantize_mxfp4(Ut_t)
            cr, er = MX.quantize_mxfp4(E2_t.T)
            mag = MX.mx_product(np.abs(cl), el_, np.abs(cr), er)
            err = err + (Kt + 1) * U * mag + U * mag
        elif prec[2] == Q.PREC_F32:
            mag = np.abs(Ut_t.astype(F64)) @ np.abs(E2_t.astype(F64))
            err = err + (Kt + 2) * U * mag
        else:
            _, mag = qm_terms(Ut_t, E2_t, prec[2], scale)
            if prec[2] not in (Q.PREC_INT8, Q.PREC_INT4):
                err = err + qm_bound(mag, mag, Kt)
        mags.append(mag)
    total = sum(mags) if mags else 0.0
    # D = alpha E3 + beta C: each term scaled by alpha (one rounding), beta C
    # joined by one FMA, the terms added in FP32
    bc = abs(beta) * np.abs(np.asarray(C, dtype=F64)) if beta != 0.0 else 0.0
    return abs(alpha) * err + (len(mags) + 1) * U * (abs(alpha) * total + bc) + 1e-38
