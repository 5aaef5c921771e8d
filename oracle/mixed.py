"""Mixed-precision E3 of the 8192-size workload: a lead block of the rank
dimension in 8 bits with a split-precision residual, the tail in 4 bits
(unpacked INT4 or MXFP4 with 32-element block scales).

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Passages followed:
  * Algorithm 3: E3 = QM(U~ E2, d3), the largest product of the chain; U~ =
    U_r Sigma_r holds the singular directions in decreasing sigma order.
  * Sec. 3.1 / Algorithm 2: the symmetric quantiser and QM (oracle.quant).
  * Sec. 3.5 / Sec. 4.2: mixed bit widths across the chain ("884").

Readings (the paper states no lead/tail split, residual or block format;
each is listed in the design notes):
  * E3's contraction index (the rank index, K = r) is split into the first
    `lead` directions and the rest:
        E3 = sum_terms QM8(U~_lead^a, E2_lead^b) + QM4(U~_tail, E2_tail).
  * Split-precision residual of a factor x quantised to codes c with scales
    s: x^hi = (c, s), x^lo = quantise(fp32(x - fp32(c * s))) with its own
    scales.  lead_split = 0: hi.hi only; 1: + lo.hi (the left factor's
    residual); 2: + lo.hi + hi.lo (lo.lo dropped).
  * Every term is a QM of Algorithm 2 (its own scales, its exact integer
    sum, fp32(fp32(acc) * fp32(sL * sR))); the terms are added in FP64.
  * MXFP4 (OCP Microscaling v1.0 e2m1 elements with an 8-bit power-of-two
    scale per 32 consecutive elements along K): scale exponent
    e = ceil(log2(fp32(amax / 6))) (no element saturates), clamped to
    [-127, 127] (e = -127 for an all-zero block); element = x * 2^-e rounded
    to nearest, ties to even, on the e2m1 grid (saturating at 6).  A block
    product sum_k cL cR is exact (multiples of 1/4 below 2^11); blocks are
    added with their factors 2^(eL + eR) (FP64, exact here), then rounded to
    FP32.
"""
import numpy as np

from . import quant

F32 = np.float32
F64 = np.float64

PREC_MXFP4 = 4
MX_BLOCK = 32
E2M1_MAX = 6.0


def round_e2m1(v):
    """Round to nearest-even on the e2m1 grid, saturating at +-6.

    e2m1: 1 sign, 2 exponent bits (bias 1), 1 mantissa bit; normal values
    (1 + m/2) 2^(e-1) for e = 1..3, subnormals m/2 for e = 0: the magnitudes
    0, 0.5, 1, 1.5, 2, 3, 4, 6.  The spacing in the binade [2^E, 2^(E+1)) is
    2^(E-1) for E = 0..2, and 0.5 below 1.  Computed in FP64 (exact).
    """
    v = np.asarray(v, dtype=F64)
    a = np.abs(v)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, 0, 2)
    quantum = np.exp2(e - 1)
    r = np.minimum(np.rint(a / quantum) * quantum, E2M1_MAX)
    return np.sign(v) * r


def mx_exponent(amax):
    """e = ceil(log2(fp32(amax / 6))) per block, clamped to [-127, 127]; -127 for amax = 0."""
    amax = np.asarray(amax, dtype=F32)
    y = (amax / F32(E2M1_MAX)).astype(F32)             # one IEEE FP32 division
    m, E = np.frexp(y.astype(F64))                      # y = m 2^E, m in [0.5, 1): exact
    e = np.where(m > 0.5, E, E - 1)                     # ceil(log2 y); y a power of two: E - 1
    e = np.where(amax > 0, e, -127)
    return np.clip(e, -127, 127).astype(np.int64)


def quantize_mxfp4(X):
    """Rows of X (M x K) in MXFP4 with blocks of 32 along K.

    Returns (codes: e2m1 values as FP64, M x K; exps: M x ceil(K/32) ints).
    """
    X = np.asarray(X, dtype=F32)
    M, K = X.shape
    nb = -(-K // MX_BLOCK)
    Xp = np.zeros((M, nb * MX_BLOCK), dtype=F32)
    Xp[:, :K] = X
    blocks = Xp.reshape(M, nb, MX_BLOCK)
    exps = mx_exponent(np.max(np.abs(blocks), axis=2))
    scaled = blocks.astype(F64) * np.exp2(-exps.astype(F64))[:, :, None]    # exact
    codes = round_e2m1(scaled).reshape(M, nb * MX_BLOCK)[:, :K]
    return codes, exps


def dequantize_mxfp4(codes, exps):
    codes = np.asarray(codes, dtype=F64)
    M, K = codes.shape
    f = np.repeat(np.exp2(np.asarray(exps, dtype=F64)), MX_BLOCK, axis=1)[:, :K]
    return codes * f


def mx_product(cl, el, cr, er):
    """sum_b 2^(el[i,b] + er[j,b]) sum_{k in b} cl[i,k] cr[j,k] (FP64; both K-major)."""
    cl = np.asarray(cl, dtype=F64)
    cr = np.asarray(cr, dtype=F64)
    M, K = cl.shape
    N = cr.shape[0]
    acc = np.zeros((M, N), dtype=F64)
    for b in range(-(-K // MX_BLOCK)):
        k0, k1 = b * MX_BLOCK, min(K, (b + 1) * MX_BLOCK)
        part = cl[:, k0:k1] @ cr[:, k0:k1].T                  # exact: multiples of 1/4, < 2^11
        acc += part * np.exp2(el[:, b][:, None] + er[:, b][None, :].astype(F64))
    return acc


def qm_mxfp4(L, R):
    """QM with MXFP4 operands: L (M x K) by rows, R (K x N) by columns, blocks along K.  FP32 result."""
    cl, el = quantize_mxfp4(L)
    cr, er = quantize_mxfp4(np.asarray(R, dtype=F32).T)
    return mx_product(cl, el, cr, er).astype(F32)


def quantize_hilo(X, prec, axis):
    """Split-precision quantisation: (c_hi, s_hi), (c_lo, s_lo) with the
    residual fp32(X - fp32(c_hi * s_hi)) quantised in the same format and
    grouping."""
    X = np.asarray(X, dtype=F32)
    c_hi, _, s_hi = quant.quantize(X, prec, axis)
    resid = (X - quant.dequantize(c_hi, s_hi, axis)).astype(F32)
    c_lo, _, s_lo = quant.quantize(resid, prec, axis)
    return (c_hi, s_hi), (c_lo, s_lo)


def _qm_codes(cl, sl, cr, sr, ax_l, ax_r):
    """One QM term on given codes: fp32(fp32(acc) * fp32(sL * sR))."""
    acc = quant.code_product(cl, cr)
    sl_b = np.asarray(sl, F32)[:, None] if ax_l == 1 else np.asarray(sl, F32)[0]
    sr_b = np.asarray(sr, F32)[None, :] if ax_r == 0 else np.asarray(sr, F32)[0]
    return (acc.astype(F32) * (sl_b * sr_b).astype(F32)).astype(F32)


def qm_any(L, R, prec, scale):
    """QM in any chain precision: MXFP4 here, the rest in oracle.quant."""
    if prec == PREC_MXFP4:
        return qm_mxfp4(L, R)
    return quant.qm(L, R, prec, scale)


def e3_lead_tail(Ut, E2, prec_tail, lead, lead_prec, lead_split, scale=quant.SCALE_ROWCOL):
    """E3 (FP64) = lead terms + tail term.  Ut: m x r, E2: r x n (FP32)."""
    Ut = np.asarray(Ut, dtype=F32)
    E2 = np.asarray(E2, dtype=F32)
    r = Ut.shape[1]
    lead = min(lead, r)
    ax_l, ax_r = (1, 0) if scale == quant.SCALE_ROWCOL else (None, None)
    out = np.zeros((Ut.shape[0], E2.shape[1]), dtype=F64)
    if lead > 0:
        (uh, suh), (ul, sul) = quantize_hilo(Ut[:, :lead], lead_prec, ax_l)
        (eh, seh), (el, sel) = quantize_hilo(E2[:lead, :], lead_prec, ax_r)
        out += _qm_codes(uh, suh, eh, seh, ax_l, ax_r)
        if lead_split >= 1:
            out += _qm_codes(ul, sul, eh, seh, ax_l, ax_r)
        if lead_split >= 2:
            out += _qm_codes(uh, suh, el, sel, ax_l, ax_r)
    if lead < r:
        out += qm_any(Ut[:, lead:], E2[lead:, :], prec_tail, scale)
    return out


def chain_lead_tail(Ut, V, W, Zt, prec, lead, lead_prec, lead_split, scale=quant.SCALE_ROWCOL,
                    alpha=1.0, beta=0.0, C=None):
    """Algorithm 3's chain with the lead/tail E3: E1 = QM(V^T W, d1), E2 =
    QM(E1 Z~, d2) as in oracle.lramm.chain, E3 as e3_lead_tail with the
    tail in d3.  Returns D = alpha E3 + beta C in FP64."""
    E1 = qm_any(np.asarray(V, F32).T, W, prec[0], scale)
    E2 = qm_any(E1, Zt, prec[1], scale)
    D = alpha * e3_lead_tail(Ut, E2, prec[2], lead, lead_prec, lead_split, scale)
    if beta != 0.0:
        D = D + beta * np.asarray(C, dtype=F64)
    return D
