"""Symmetric linear quantiser, dequantiser and the quantised GEMM "QM".

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Paper passages followed:
  * Eq. (Quantization), Sec. 3.1: a_int = TypeCast(lambda * a_fp, intN).
  * Eq. (get_lambda), Sec. 3.1: lambda = (2^(N-1) - 1) / a_max, a_max the
    largest absolute value of the scale group.
  * Eq. (Dequantization), Sec. 3.1: a_fp = a_int / lambda.
  * Algorithm 2 (quantised GEMM): quantise A and B, integer GEMM, dequantise
    the integer product, D = alpha * D_F + beta * C.

Readings where the paper is silent (each is listed in the design notes):
  * TypeCast rounds to nearest, ties to even, then clamps to +-(2^(N-1)-1);
    the symmetric range never produces -2^(N-1).
  * The arithmetic that decides a code is FP32 (the precision the factors are
    stored in on the device): a_max exact, lambda = fp32(D) / fp32(a_max)
    (IEEE division), code = rint(fp32(x * lambda)).  A group whose a_max is 0
    gets lambda = 0, codes 0 and scale 0.
  * The dequantisation scale is s = fp32(a_max / D) (= 1/lambda in exact
    arithmetic); the product of a left code row i and right code column j is
    dequantised as fp32( fp32(acc) * fp32(s_left[i] * s_right[j]) ), acc being
    the exact integer (or exact FP8-product) sum.
  * Scale groups: ROWCOL gives the left operand one scale per row and the
    right operand one scale per column (so both factor out of the K sum);
    TENSOR gives each operand a single scale.
  * FP8 e4m3 (OCP OFP8): lambda = 448 / a_max, the code is fp32(x * lambda)
    rounded to nearest-even onto the e4m3 grid, saturating at +-448; the
    scale is s = fp32(a_max / 448).
"""
import numpy as np

F32 = np.float32

PREC_F32, PREC_INT8, PREC_INT4, PREC_E4M3 = 0, 1, 2, 3
SCALE_ROWCOL, SCALE_TENSOR = 0, 1

E4M3_MAX = 448.0


def qmax(prec):
    """D = 2^(N-1) - 1 of Eq. (get_lambda) for the integer formats."""
    return {PREC_INT8: 127, PREC_INT4: 7}[prec]


def round_e4m3(v):
    """Round FP32 values to nearest-even on the OCP e4m3 grid, saturating.

    e4m3: 1 sign, 4 exponent (bias 7), 3 mantissa bits; normal numbers
    (1 + m/8) * 2^(e-7) for e = 1..15 (e = 15, m = 7 is NaN, so the largest
    finite is 1.75 * 2^8 = 448); subnormals m/8 * 2^-6.  Grid spacing in the
    binade [2^E, 2^(E+1)) is 2^(E-3) for E >= -6 and 2^-9 below 2^-6.
    Computed in FP64, where every step is exact for FP32 inputs.
    """
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.clip(e, -6, 8)
    quantum = np.exp2(e - 3)
    r = np.rint(a / quantum) * quantum          # a/quantum exact (power of 2)
    r = np.minimum(r, E4M3_MAX)
    return np.sign(v) * r


def absmax_groups(X, axis):
    """a_max per row (axis=1), per column (axis=0) or whole tensor (axis=None)."""
    X = np.asarray(X, dtype=F32)
    if axis is None:
        return np.array([np.max(np.abs(X))], dtype=F32) if X.size else np.zeros(1, F32)
    return np.max(np.abs(X), axis=axis).astype(F32)


def quantize(X, prec, axis):
    """Quantise an FP32 matrix with one scale per group along `axis`.

    axis=1: one group per row; axis=0: one group per column; axis=None: one
    group for the whole matrix.  Returns (codes as float64 holding the code
    values, lam (FP32, per group), s (FP32 dequant scale, per group)).
    Codes are integers for INT8/INT4 and e4m3 values for E4M3.
    """
    X = np.asarray(X, dtype=F32)
    amax = absmax_groups(X, axis)
    if prec in (PREC_INT8, PREC_INT4):
        D = F32(qmax(prec))
    elif prec == PREC_E4M3:
        D = F32(E4M3_MAX)
    else:
        raise ValueError("quantize: unsupported precision %r" % prec)
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = np.where(amax > 0, D / amax, F32(0)).astype(F32)
    s = (amax / D).astype(F32)
    if axis is None:
        lam_b = lam[0]
    elif axis == 1:
        lam_b = lam[:, None]
    else:
        lam_b = lam[None, :]
    y = (X * lam_b).astype(F32)                     # one FP32 multiply
    if prec == PREC_E4M3:
        codes = round_e4m3(y)
    else:
        codes = np.clip(np.rint(y.astype(np.float64)), -float(D), float(D))
    return codes.astype(np.float64), lam, s


def dequantize(codes, s, axis):
    """Elementwise dequantisation a_fp = code * s (Eq. Dequantization)."""
    s = np.asarray(s, dtype=F32)
    if axis is None:
        sb = s[0]
    elif axis == 1:
        sb = s[:, None]
    else:
        sb = s[None, :]
    return (np.asarray(codes, dtype=F32) * sb).astype(F32)


def code_product(codes_l, codes_r):
    """Exact sum over K of code products (int or e4m3 values).

    Integer codes are at most 127 in magnitude and e4m3 codes carry 4
    significant bits, so every product and every partial sum of the shapes
    used here is an integer multiple of 2^-18 below 2^53 * 2^-18: an FP64
    matrix product is exact.  (Checked against a brute-force loop in tests.)
    """
    return np.asarray(codes_l, dtype=np.float64) @ np.asarray(codes_r, dtype=np.float64)


def qm(L, R, prec, scale=SCALE_ROWCOL):
    """QM(L * R, d) of Algorithm 2 / Algorithm 3, returned in FP32.

    L: M x K, R: K x N (FP32).  The left operand is scaled per row, the
    right per column (ROWCOL) or both per tensor (TENSOR).  For PREC_F32 the
    product is the plain FP64 product (no quantisation), rounded to FP32.
    """
    L = np.asarray(L, dtype=F32)
    R = np.asarray(R, dtype=F32)
    if prec == PREC_F32:
        return (L.astype(np.float64) @ R.astype(np.float64)).astype(F32)
    ax_l, ax_r = (1, 0) if scale == SCALE_ROWCOL else (None, None)
    cl, _, sl = quantize(L, prec, ax_l)
    cr, _, sr = quantize(R, prec, ax_r)
    acc = code_product(cl, cr)
    sl_b = sl[:, None] if ax_l == 1 else sl[0]
    sr_b = sr[None, :] if ax_r == 0 else sr[0]
    sprod = (sl_b * sr_b).astype(F32)               # FP32 product of scales
    return (acc.astype(F32) * sprod).astype(F32)    # one rounding of acc, one multiply
