"""The tensor-core QM products (tcgen05) against the oracle.

INT8 codes as BF16 (kind::f16): the integer sum must be exact (FP32
partials of at most 1024 products are exact integers; longer K is split and
added as 32-bit integers), so with unit scales the output is fp32(exact
sum), compared bit for bit; with real scales the dequantised value is
fp32(fp32(acc) * fp32(sL * sR)) as the oracle computes it.  INT4 codes as
e4m3 bytes (kind::f8f6f4): exact in the same sense.  E4M3 codes: FP32
accumulation, within the FP32 summation bound.  FP32 operands as TF32
(kind::tf32): within the TF32 rounding bound.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def np_(t):
    return t.detach().cpu().numpy()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def codes(vals):
    return dev(vals.astype(np.float32)).to(torch.bfloat16)


def ones(n):
    return torch.ones(n, dtype=torch.float32, device="cuda")


# (M, N, K): ragged tiles, K not a multiple of the 64-wide stage, one and several
# K chunks, the shapes of E1 (r x r, K = k), E2 (n x r, K = r) and E3 (m x n, K = r)
SHAPES = [(70, 45, 48), (129, 65, 4096), (64, 200, 1040), (1, 1, 16), (300, 260, 256), (256, 256, 4096),
          (4096, 256, 256), (1000, 1100, 272), (128, 4096, 2048)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_integer_sum_exact(L, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = rng.integers(-127, 128, (M, K))
    b = rng.integers(-127, 128, (N, K))
    D = np_(L.qgemm_tc(codes(a), codes(b), ones(M), ones(N)))
    exact = oracle.quant.code_product(a, b.T)
    assert np.array_equal(D, exact.astype(np.float32))


@pytest.mark.parametrize("K", [1024, 1040, 4096, 16384])
def test_worst_case_codes(L, K):
    """All-extreme codes: |acc| up to 127^2 K, far above 2^24 for K > 1024."""
    a = np.full((3, K), 127.0)
    a[1] = -127.0
    a[2, ::2] = -127.0
    b = np.full((2, K), 127.0)
    b[1, 1::2] = -127.0
    D = np_(L.qgemm_tc(codes(a), codes(b), ones(3), ones(2)))
    assert np.array_equal(D, oracle.quant.code_product(a, b.T).astype(np.float32))


@pytest.mark.parametrize("per_row", [True, False])
@pytest.mark.parametrize("M,K,N", [(150, 200, 90), (4096, 256, 300), (256, 4096, 256)])
def test_dequantised_matches_oracle(L, per_row, M, K, N):
    rng = np.random.default_rng(M + K + N + per_row)
    Lm = (rng.standard_normal((M, K)) * np.exp(rng.uniform(-2, 2, (M, 1)))).astype(np.float32)
    R = (rng.standard_normal((K, N)) * np.exp(rng.uniform(-2, 2, (1, N)))).astype(np.float32)
    Kp = K + (-K) % 16
    cL, sL = L.quantize(dev(Lm), 1, per_row, ldcodes=Kp)
    cR, sR = L.quantize(dev(np.ascontiguousarray(R.T)), 1, per_row, ldcodes=Kp)
    D = np_(L.qgemm_tc(cL, cR, sL, sR, per_row=per_row))
    ref = oracle.quant.qm(Lm, R, 1, 0 if per_row else 1)
    assert np.array_equal(D, ref)


# Many output tiles (at least four 128 x 256 tiles per SM): the persistent
# kernel (one CTA per SM, double-buffered TMEM accumulators).  Ragged M, N
# and K (a multiple of 16, as the entry point requires); its results must be those of the per-tile kernel bit for bit.
PERSIST_SHAPES = [(5000, 5000, 128), (4999, 4100, 208), (8192, 4864, 64)]


@pytest.mark.parametrize("M,N,K", PERSIST_SHAPES)
def test_integer_sum_exact_persistent(L, M, N, K):
    rng = np.random.default_rng(M + 5 * N + 9 * K)
    a = rng.integers(-127, 128, (M, K))
    b = rng.integers(-127, 128, (N, K))
    D = np_(L.qgemm_tc(codes(a), codes(b), ones(M), ones(N)))
    assert np.array_equal(D, oracle.quant.code_product(a, b.T).astype(np.float32))


@pytest.mark.parametrize("per_row", [True, False])
def test_dequantised_matches_oracle_persistent(L, per_row):
    rng = np.random.default_rng(41 + per_row)
    M, K, N = 4100, 130, 4864
    Lm = (rng.standard_normal((M, K)) * np.exp(rng.uniform(-2, 2, (M, 1)))).astype(np.float32)
    R = (rng.standard_normal((K, N)) * np.exp(rng.uniform(-2, 2, (1, N)))).astype(np.float32)
    Kp = K + (-K) % 16
    cL, sL = L.quantize(dev(Lm), 1, per_row, ldcodes=Kp)
    cR, sR = L.quantize(dev(np.ascontiguousarray(R.T)), 1, per_row, ldcodes=Kp)
    D = np_(L.qgemm_tc(cL, cR, sL, sR, per_row=per_row, alpha=0.5))
    ref = (np.float32(0.5) * oracle.quant.qm(Lm, R, 1, 0 if per_row else 1)).astype(np.float32)
    assert np.array_equal(D, ref)


def test_int4_codes_exact_persistent(L):
    rng = np.random.default_rng(17)
    M, N, K = 5000, 4100, 256
    a = rng.integers(-7, 8, (M, K))
    b = rng.integers(-7, 8, (N, K))
    D = np_(L.qgemm_tc(e4m3(a), e4m3(b), ones(M), ones(N), prec=L.P_INT4))
    assert np.array_equal(D, oracle.quant.code_product(a, b.T).astype(np.float32))


def test_alpha_beta(L):
    """D = alpha QM + beta C: one FP32 multiply and one FMA after the dequantisation."""
    rng = np.random.default_rng(5)
    M, K, N = 300, 256, 280
    Lm = rng.standard_normal((M, K)).astype(np.float32)
    R = rng.standard_normal((K, N)).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    cL, sL = L.quantize(dev(Lm), 1, True, ldcodes=K)
    cR, sR = L.quantize(dev(np.ascontiguousarray(R.T)), 1, True, ldcodes=K)
    D = np_(L.qgemm_tc(cL, cR, sL, sR, alpha=0.75, beta=-1.5, C=dev(C)))
    qm = oracle.quant.qm(Lm, R, 1, 0)
    v = (np.float32(0.75) * qm).astype(np.float32)
    ref = np.float64(-1.5) * C.astype(np.float64) + v.astype(np.float64)   # exact FMA, one rounding below
    assert np.all(np.abs(D - ref) <= 2.0 ** -24 * np.abs(ref) + 1e-30)


# ---------------------------------------------------------------- FP8 kinds
from tests import pins  # noqa: E402


def e4m3(vals):
    return dev(np.asarray(vals, dtype=np.float32)).to(torch.float8_e4m3fn)


FP8_SHAPES = [(70, 45, 48), (129, 65, 4096), (1, 1, 16), (300, 260, 400), (4096, 256, 128), (1000, 1100, 400),
              (256, 256, 8192)]


@pytest.mark.parametrize("M,N,K", FP8_SHAPES)
def test_int4_codes_exact(L, M, N, K):
    """INT4 codes |c| <= 7 are exact e4m3 values; sums of products <= 49 are exact in FP32."""
    rng = np.random.default_rng(M + 3 * N + 5 * K)
    a = rng.integers(-7, 8, (M, K))
    b = rng.integers(-7, 8, (N, K))
    D = np_(L.qgemm_tc(e4m3(a), e4m3(b), ones(M), ones(N), prec=L.P_INT4))
    assert np.array_equal(D, oracle.quant.code_product(a, b.T).astype(np.float32))


def test_int4_worst_case(L):
    K = 65536
    a = np.full((2, K), 7.0)
    a[1, ::2] = -7.0
    b = np.full((2, K), -7.0)
    D = np_(L.qgemm_tc(e4m3(a), e4m3(b), ones(2), ones(2), prec=L.P_INT4))
    assert np.array_equal(D, oracle.quant.code_product(a, b.T).astype(np.float32))


@pytest.mark.parametrize("M,N,K", [(96, 80, 2048), (300, 260, 400), (1000, 1100, 400)])
def test_e4m3_codes_within_fp32_sum_bound(L, M, N, K):
    rng = np.random.default_rng(M + N + K)
    grid = pins.e4m3_decode_all()
    a = rng.choice(grid, (M, K))
    b = rng.choice(grid, (N, K))
    D = np_(L.qgemm_tc(e4m3(a), e4m3(b), ones(M), ones(N), prec=L.P_E4M3)).astype(np.float64)
    ref = oracle.quant.code_product(a, b.T)
    mag = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(D - ref) <= K * 2.0 ** -24 * mag + 2.0 ** -24 * np.abs(ref))


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("per_row", [True, False])
def test_fp8_dequantised_matches_oracle(L, prec, per_row):
    rng = np.random.default_rng(30 + prec + per_row)
    M, K, N = 300, 400, 280
    Lm = (rng.standard_normal((M, K)) * np.exp(rng.uniform(-2, 2, (M, 1)))).astype(np.float32)
    R = (rng.standard_normal((K, N)) * np.exp(rng.uniform(-2, 2, (1, N)))).astype(np.float32)
    cL, sL = L.quantize(dev(Lm), prec, per_row, ldcodes=K)
    cR, sR = L.quantize(dev(np.ascontiguousarray(R.T)), prec, per_row, ldcodes=K)
    D = np_(L.qgemm_tc(cL, cR, sL, sR, per_row=per_row, prec=prec))
    ref = oracle.quant.qm(Lm, R, prec, 0 if per_row else 1)
    if prec == 2:
        assert np.array_equal(D, ref)
    else:
        assert oracle.lramm.rel_fro(D, ref) < 1e-6


# ---------------------------------------------------------------- TF32 products
@pytest.mark.parametrize("M,N,K", [(70, 45, 40), (512, 1000, 400), (4096, 4096, 400), (64, 64, 4096), (1, 300, 8)])
@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_tgemm_within_tf32_bound(L, M, N, K, beta):
    """C = alpha A B^T + beta C with operands as TF32 (10 explicit mantissa
    bits): |error| <= 2^-9 (|A| |B|^T) + FP32 summation, elementwise."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    C = L.tgemm_tc(dev(A), dev(B), alpha=0.5, beta=beta, C=dev(C0.copy()))
    ref = 0.5 * (A.astype(np.float64) @ B.astype(np.float64).T) + beta * C0
    mag = 0.5 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T) + abs(beta) * np.abs(C0)
    assert np.all(np.abs(np_(C) - ref) <= (2.0 ** -9 + K * 2.0 ** -23) * mag)
