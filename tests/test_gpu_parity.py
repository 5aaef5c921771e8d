"""CUDA path (through the C ABI) against the CPU oracle on seeded inputs.

Bars: bit-exact for integer work (Philox words, integer codes, integer
accumulators, and every FP32 value that is decided by FP32 operations on
identical inputs: quantisation scales, dequantised QM outputs, the whole
integer chain); tolerances written per test for floating point.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import elementwise as EW
from tests import pins

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


def codes_np(c):
    return c.float().cpu().numpy().astype(np.float64)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ---------------------------------------------------------------- Philox / Omega
@pytest.mark.parametrize("seed,sid,n", [(7, 0, 1000), (7, 1, 4099), (0x123456789ABCDEF, 65535, 17),
                                        (0xFFFFFFFF00000001, 3, 1)])
def test_philox_words_bit_exact(L, seed, sid, n):
    g = np_(L.philox_words(seed, sid, n)).view(np.uint32)
    assert np.array_equal(g, oracle.philox.philox_words(seed, sid, n))


@pytest.mark.parametrize("rows,cols", [(512, 74), (37, 13), (1, 1), (4097, 272), (3, 5)])
def test_gaussian_matches_oracle(L, rows, cols):
    g = np_(L.gaussian(7, 1, rows, cols)).astype(np.float64)
    o = oracle.philox.gaussian_matrix(7, 1, rows, cols).astype(np.float64)
    # FP32 logf / log1pf / sincospif against FP64 then rounded: a few ulp
    assert np.all(np.abs(g - o) <= 2e-6 + 1e-6 * np.abs(o))


# ---------------------------------------------------------------- quantiser
PRECS = [1, 2, 3]  # INT8, INT4, E4M3


def _qinput(rows, cols, seed):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((rows, cols)) * np.exp(rng.uniform(-6, 6, (rows, 1)))).astype(np.float32)
    X[min(5, rows - 1)] = 0.0
    return X


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("per_row", [True, False])
@pytest.mark.parametrize("rows,cols,ldc", [(133, 77, 80), (1, 16, 16), (64, 4096, 4096), (7, 3, 16)])
def test_quantize_bit_exact(L, prec, per_row, rows, cols, ldc):
    X = _qinput(rows, cols, rows * 7 + cols)
    codes, scales = L.quantize(dev(X), prec, per_row, ldcodes=ldc)
    c = codes_np(codes)
    oc, lam, s = oracle.quant.quantize(X, prec, 1 if per_row else None)
    assert np.array_equal(c[:, :cols], oc)
    assert np.all(c[:, cols:] == 0)
    assert np.array_equal(np_(scales), s)


def test_quantize_worked_examples_on_gpu(L):
    """The hand-worked examples of Eqs. (get_lambda), (Quantization) on the CUDA quantiser."""
    for bits, xs, codes in pins._read_golden("quant_worked_example.txt"):
        prec = 1 if int(bits) == 8 else 2
        x = np.array([[float(v) for v in xs.split()]], dtype=np.float32)
        want = np.array([float(v) for v in codes.split()])
        c, s = L.quantize(dev(x), prec, True, ldcodes=16)
        assert np.array_equal(codes_np(c)[0, : x.shape[1]], want), (bits, xs)


def test_e4m3_rounding_on_gpu(L):
    """lambda = 448 / a_max = 1 on rows whose a_max is 448: codes are the plain
    RNE-satfinite e4m3 rounding of the inputs (grid values, midpoints, goldens)."""
    grid = pins.e4m3_decode_all()
    pos = grid[grid >= 0]
    mids = (pos[:-1] + pos[1:]) / 2.0
    gold = [float(x) for x, _ in pins._read_golden("e4m3_rounding.txt") if abs(float(x)) <= 448.0]
    vals = np.concatenate([grid, mids, -mids, gold]).astype(np.float32)
    n = len(vals)
    cols = 1 + n
    X = np.zeros((1, cols), dtype=np.float32)
    X[0, 0] = 448.0
    X[0, 1:] = vals
    c, s = L.quantize(dev(X), 3, True, ldcodes=cols + (-cols) % 16)
    got = codes_np(c)[0, 1:cols]
    assert np.array_equal(got, oracle.quant.round_e4m3(vals))
    assert np_(s)[0] == np.float32(1.0)


# ---------------------------------------------------------------- QM products
def _codes(vals, prec):
    t = torch.from_numpy(np.ascontiguousarray(vals.astype(np.float32))).cuda()
    return t.to(torch.bfloat16) if prec == 1 else t.to(torch.float8_e4m3fn)


@pytest.mark.parametrize("M,N,K", [(70, 45, 48), (129, 65, 4096), (64, 200, 1040), (1, 1, 16)])
@pytest.mark.parametrize("prec,D", [(1, 127), (2, 7)])
def test_qgemm_integer_accumulator_bit_exact(L, M, N, K, prec, D):
    rng = np.random.default_rng(M + N + K)
    a = rng.integers(-D, D + 1, (M, K))
    b = rng.integers(-D, D + 1, (N, K))
    acc = np_(L.qgemm(_codes(a, prec), _codes(b, prec), prec, raw=True)).astype(np.float64)
    assert np.array_equal(acc, oracle.quant.code_product(a, b.T))


@pytest.mark.parametrize("K", [1024, 1040, 4096, 16384])
def test_qgemm_int8_worst_case(L, K):
    """All-extreme codes: |acc| up to 127^2 K, far above 2^24 (FP32 integers)."""
    a = np.full((3, K), 127.0)
    a[1] = -127.0
    a[2, ::2] = -127.0
    b = np.full((2, K), 127.0)
    b[1, 1::2] = -127.0
    acc = np_(L.qgemm(_codes(a, 1), _codes(b, 1), 1, raw=True)).astype(np.float64)
    assert np.array_equal(acc, oracle.quant.code_product(a, b.T))


def test_qgemm_e4m3_accumulator(L):
    rng = np.random.default_rng(4)
    grid = pins.e4m3_decode_all()
    M, N, K = 96, 80, 2048
    a = rng.choice(grid, (M, K))
    b = rng.choice(grid, (N, K))
    acc = np_(L.qgemm(_codes(a, 3), _codes(b, 3), 3, raw=True)).astype(np.float64)
    ref = oracle.quant.code_product(a, b.T)
    mag = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(acc - ref) <= K * 2.0 ** -24 * mag)          # FP32 accumulation bound


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("per_row", [True, False])
def test_qm_dequantised_matches_oracle(L, prec, per_row):
    rng = np.random.default_rng(10 + prec)
    M, K, N = 150, 200, 90
    Lm = (rng.standard_normal((M, K)) * np.exp(rng.uniform(-2, 2, (M, 1)))).astype(np.float32)
    R = (rng.standard_normal((K, N)) * np.exp(rng.uniform(-2, 2, (1, N)))).astype(np.float32)
    Kp = K + (-K) % 16
    cL, sL = L.quantize(dev(Lm), prec, per_row, ldcodes=Kp)
    cR, sR = L.quantize(dev(np.ascontiguousarray(R.T)), prec, per_row, ldcodes=Kp)
    D = np_(L.qgemm(cL, cR, prec, sL, sR, per_row=per_row))
    ref = oracle.quant.qm(Lm, R, prec, 0 if per_row else 1)
    if prec in (1, 2):
        assert np.array_equal(D, ref)
    else:
        # identical e4m3 codes, FP32 accumulation of K products on the GPU
        _, mag = EW.qm_terms(Lm, R, prec, 0 if per_row else 1)
        assert np.all(np.abs(D.astype(np.float64) - ref) <= EW.qm_bound(mag, ref, K))


def test_qm_alpha_beta_epilogue(L):
    rng = np.random.default_rng(12)
    M, K, N = 64, 48, 40
    Lm = rng.standard_normal((M, K)).astype(np.float32)
    R = rng.standard_normal((K, N)).astype(np.float32)
    C = rng.standard_normal((M, N)).astype(np.float32)
    cL, sL = L.quantize(dev(Lm), 1, True)
    cR, sR = L.quantize(dev(np.ascontiguousarray(R.T)), 1, True)
    D = np_(L.qgemm(cL, cR, 1, sL, sR, alpha=0.75, beta=-1.5, C=dev(C))).astype(np.float64)
    ref = 0.75 * oracle.quant.qm(Lm, R, 1).astype(np.float64) - 1.5 * C
    assert np.allclose(D, ref, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- factor chain
def _factors(m, n, k, r, seed):
    rng = np.random.default_rng(seed)
    Ut = (rng.standard_normal((m, r)) * np.exp(-np.arange(r) / 8.0)).astype(np.float32)
    Vt = (rng.standard_normal((r, k)) / np.sqrt(k)).astype(np.float32)
    Wt = (rng.standard_normal((r, k)) / np.sqrt(k)).astype(np.float32)
    Zt = (rng.standard_normal((n, r)) * np.exp(-np.arange(r) / 8.0)).astype(np.float32)
    return Ut, Vt, Wt, Zt


@pytest.mark.parametrize("prec", [(1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)])
@pytest.mark.parametrize("scale", [0, 1])
def test_chain_integer_bit_exact(L, prec, scale):
    """Identical FP32 factors in: E1, E2 (requantised) and E3 are decided by
    the same FP32 operations on both sides, so D is bit-identical."""
    m, n, k, r = 300, 260, 333, 40
    Ut, Vt, Wt, Zt = _factors(m, n, k, r, 21)
    plan = L.Plan(m, n, k, r, 0, 0, prec=prec, scale=scale)
    D = np_(L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt)))
    ref = oracle.lramm.chain(Ut, Vt.T, Wt.T, Zt.T, prec, scale)
    assert np.array_equal(D.astype(np.float64), ref)


def _positive_factors(m, n, k, r, seed):
    """Factors with entries of one sign (no cancellation in any product), so
    that every sum's FP32 bound is close to its value."""
    rng = np.random.default_rng(seed)
    Ut = (rng.uniform(0.5, 1.5, (m, r)) * np.exp(-np.arange(r) / 8.0)).astype(np.float32)
    Vt = (rng.uniform(0.5, 1.5, (r, k)) / np.sqrt(k)).astype(np.float32)
    Wt = (rng.uniform(0.5, 1.5, (r, k)) / np.sqrt(k)).astype(np.float32)
    Zt = (rng.uniform(0.5, 1.5, (n, r)) * np.exp(-np.arange(r) / 8.0)).astype(np.float32)
    return Ut, Vt, Wt, Zt


@pytest.mark.parametrize("prec", [(3, 3, 3), (3, 1, 3), (1, 1, 3), (1, 0, 3)])
@pytest.mark.parametrize("scale", [0, 1])
def test_chain_fp8_elementwise(L, prec, scale):
    """Chains with E4M3 (and FP32) stages, element by element.  An E4M3 QM
    sums its code products in FP32 on the GPU, so on identical codes it is
    within K u sum |cL cR| sL sR (+ 2u) of the oracle's exact sum (Algorithm
    2); a requantised intermediate (E1 for E2, E2 for E3; Algorithm 3) then
    has the oracle's codes wherever its pre-rounding value lies farther from
    a rounding boundary than that bound moves it.  The inputs are the first
    seed of a fixed list for which this holds at every stage
    (tests/elementwise.py proves it), so D is compared entry by entry against
    the propagated bound."""
    m, n, k, r = 300, 260, 160, 16
    for seed in range(22, 102):
        Ut, Vt, Wt, Zt = _positive_factors(m, n, k, r, seed)
        try:
            ref, bound = EW.chain_bound(Ut, Vt, Wt, Zt, prec, scale)
            break
        except AssertionError:
            continue
    else:
        pytest.fail("no seed in the list has provably identical codes at every stage")
    assert np.array_equal(ref, oracle.lramm.chain(Ut, Vt.T, Wt.T, Zt.T, prec, scale))
    plan = L.Plan(m, n, k, r, 0, 0, prec=prec, scale=scale)
    D = np_(L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt))).astype(np.float64)
    bad = np.abs(D - ref) > bound
    assert not bad.any(), "seed %d: %d entries outside the bound, worst %.3g x bound" % (
        seed, int(bad.sum()), float(np.max(np.abs(D - ref) / bound)))


def test_chain_f32_elementwise(L):
    """The FP32 chain (no quantisation): every product within its FP32
    forward-error bound, propagated element by element through E1, E2, E3."""
    m, n, k, r = 200, 180, 260, 32
    Ut, Vt, Wt, Zt = _factors(m, n, k, r, 22)
    plan = L.Plan(m, n, k, r, 0, 0, prec=(0, 0, 0))
    D = np_(L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt))).astype(np.float64)
    ref, bound = EW.chain_bound(Ut, Vt, Wt, Zt, (0, 0, 0))
    assert np.all(np.abs(D - ref) <= bound)
    assert oracle.lramm.rel_fro(D, ref) < 2e-6


def test_chain_e4m3_random_signs(L):
    """E4M3 chains on factors with random signs and K = 260: cancellation
    puts some intermediates within their FP32 bound of a rounding boundary,
    so a code may differ between the sides; the whole chain is compared by
    its relative Frobenius error (a code step is 2^-4 relative)."""
    m, n, k, r = 200, 180, 260, 32
    Ut, Vt, Wt, Zt = _factors(m, n, k, r, 22)
    for prec in ((3, 3, 3), (1, 0, 3)):
        plan = L.Plan(m, n, k, r, 0, 0, prec=prec)
        D = np_(L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt)))
        ref = oracle.lramm.chain(Ut, Vt.T, Wt.T, Zt.T, prec)
        assert oracle.lramm.rel_fro(D, ref) < 2e-3, prec


# ---------------------------------------------------------------- randomized SVD
@pytest.mark.parametrize("m,k,r,p,q", [(512, 512, 64, 10, 1), (300, 260, 20, 8, 2), (133, 97, 7, 5, 0),
                                       (700, 520, 48, 16, 1)])
@pytest.mark.parametrize("which", [0, 1])
def test_rsvd_matches_oracle(L, m, k, r, p, q, which):
    sig = workloads.spectrum("exp32", min(m, k))
    X = workloads.lowrank(m, k, sig, 500 + m).astype(np.float32)
    # plan: which=0 treats X as A (m x k); which=1 as B (k' x n') = X
    plan = L.Plan(m, m, k, r, p, q, seed=7) if which == 0 else L.Plan(k, k, m, r, p, q, seed=7)
    U, S, V = (np_(t) for t in L.rsvd(plan, which, dev(X)))
    Uo, so, Vo = oracle.lramm.rsvd(X, r, p, q, 7, which)
    assert np.allclose(S, so, rtol=1e-5, atol=1e-6 * so[0])
    assert oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T) < 1e-5
    # FP32 CholeskyQR2 orthogonality: ~sqrt(rows * l) u typical
    tol = 4.0 * np.sqrt(max(m, k) * (r + p)) * 2.0 ** -24
    assert np.abs(U.T @ U - np.eye(r)).max() < tol
    assert np.abs(V.T @ V - np.eye(r)).max() < tol


@pytest.mark.parametrize("m,k,r,p,q", [(900, 800, 200, 16, 1), (1100, 1024, 256, 16, 2), (1100, 1024, 272, 16, 1),
                                       (1100, 1024, 300, 20, 1), (1300, 1100, 380, 20, 1), (1500, 1300, 512, 32, 1)])
def test_rsvd_wide_sketch_matches_oracle(L, m, k, r, p, q):
    """l = 216, 272, 288, 320, 400, 544: the small SVD runs on 14- and 16-CTA
    clusters; l = 288 is the largest single-CTA blocked Cholesky, l = 320
    takes the column-panel Cholesky, l = 400 and 544 the two-level
    Cholesky (blocks of 224 + 176 and 288 + 256)."""
    X = workloads.lowrank(m, k, workloads.spectrum("poly1", min(m, k)), 600 + m).astype(np.float32)
    plan = L.Plan(m, m, k, r, p, q, seed=7)
    ws = plan.workspace()
    U, S, V = (np_(t) for t in L.rsvd(plan, 0, dev(X), ws=ws))
    assert L.status_read(ws) == 0
    Uo, so, Vo = oracle.lramm.rsvd(X, r, p, q, 7, 0)
    assert np.allclose(S, so, rtol=2e-5, atol=2e-6 * so[0])
    assert oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T) < 2e-5
    tol = 4.0 * np.sqrt(max(m, k) * (r + p)) * 2.0 ** -24
    assert np.abs(U.T @ U - np.eye(r)).max() < tol
    assert np.abs(V.T @ V - np.eye(r)).max() < tol


def test_rsvd_rank_deficient_sketch(L):
    """rank(X) = 10 < l = 18: the sketch is rank-deficient, the shifted first
    CholeskyQR pass still factors it, X is reproduced and the trailing singular
    values vanish."""
    m, k, rank, r, p = 300, 200, 10, 12, 6
    X = workloads.exact_rank(m, k, rank, 77).astype(np.float32)
    plan = L.Plan(m, m, k, r, p, 1, seed=7)
    ws = plan.workspace()
    U, S, V = (np_(t) for t in L.rsvd(plan, 0, dev(X), ws=ws))
    st = L.status_read(ws)
    assert st in (0, 7)
    assert oracle.lramm.rel_fro((U[:, :rank] * S[:rank]) @ V[:, :rank].T, X) < 1e-5
    assert np.all(S[rank:] < 1e-5 * S[0])


# ---------------------------------------------------------------- end to end
def _e2e(L, name, prec, scale=None, **kw):
    c = workloads.CONFIGS[name]
    A, B = workloads.operands(name, scale=scale)
    m, k = A.shape
    n = B.shape[1]
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    plan = L.Plan(m, n, k, c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=prec, **kw)
    ws = plan.workspace()
    D = L.matmul(plan, dev(A32), dev(B32), ws=ws)
    st = L.status_read(ws)
    assert st == 0, st
    ref = oracle.lramm.lramm(A32, B32, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, prec)
    return np_(D).astype(np.float64), ref, A32, B32


def test_matmul_fp32_path_lramm_512(L):
    """Plain LRAMM (FP32 factors), m=n=k=512, r=64, p=10, q=1: <= 1e-5."""
    D, ref, A, B = _e2e(L, "lramm_512", (0, 0, 0))
    assert oracle.lramm.rel_fro(D, ref) <= 1e-5


def quantised_agreement(D, ref_q, ref_f, exact):
    """The GPU's FP32 RSVD and the oracle's FP64 RSVD give factors that differ
    by ~u / (relative singular-value gap) per singular vector (up to ~1e-3
    here), so many codes land on different sides of a rounding boundary: the
    two quantised outputs are two draws of the same quantisation noise.
    Bars: they differ by at most 1.5x that noise (the noise being the
    oracle's quantised-minus-unquantised chain), and their errors against
    the exact product agree to 10%."""
    noise = oracle.lramm.rel_fro(ref_q, ref_f)
    assert oracle.lramm.rel_fro(D, ref_q) <= 1.5 * noise
    err_gpu = oracle.lramm.rel_fro(D, exact)
    err_orc = oracle.lramm.rel_fro(ref_q, exact)
    assert abs(err_gpu - err_orc) <= 0.10 * err_orc


def test_matmul_per_tensor_scales_lramm_512(L):
    """Per-tensor scales through lramm_matmul: each operand's factors are
    quantised on its own stream (the second stream with its own amax word)
    before the chain; the result against the oracle's per-tensor chain by
    the same noise criterion as the per-row case."""
    c = workloads.CONFIGS["lramm_512"]
    A, B = workloads.operands("lramm_512")
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    m, k = A32.shape
    n = B32.shape[1]
    prec = (1, 1, 1)
    plan = L.Plan(m, n, k, c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=prec, scale=L.S_TENSOR)
    ws = plan.workspace()
    D1 = np_(L.matmul(plan, dev(A32), dev(B32), ws=ws)).astype(np.float64)
    D2 = np_(L.matmul(plan, dev(A32), dev(B32), ws=ws)).astype(np.float64)
    assert L.status_read(ws) == 0
    assert np.array_equal(D1, D2)   # the per-tensor amax words start from zero on every call
    ref = oracle.lramm.lramm(A32, B32, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, prec,
                             scale=oracle.quant.SCALE_TENSOR)
    ref_f = oracle.lramm.lramm(A32, B32, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (0, 0, 0))
    quantised_agreement(D1, ref, ref_f, oracle.lramm.exact_product(A32, B32))


@pytest.mark.parametrize("prec", [(1, 1, 1), (1, 1, 2), (3, 3, 3)])
def test_matmul_quantised_lramm_512(L, prec):
    D, ref, A, B = _e2e(L, "lramm_512", prec)
    c = workloads.CONFIGS["lramm_512"]
    ref_f = oracle.lramm.lramm(A, B, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (0, 0, 0))
    quantised_agreement(D, ref, ref_f, oracle.lramm.exact_product(A, B))


def test_matmul_alpha_beta_c(L):
    m, n, k = 256, 192, 224
    A, B = workloads.operands("lramm_512", scale=(m, n, k))
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    C = np.random.default_rng(2).standard_normal((m, n)).astype(np.float32)
    plan = L.Plan(m, n, k, 24, 8, 1, seed=7, prec=(1, 1, 1), alpha=0.5, beta=2.0)
    D = np_(L.matmul(plan, dev(A32), dev(B32), C=dev(C))).astype(np.float64)
    ref = oracle.lramm.lramm(A32, B32, 24, 8, 1, 7, (1, 1, 1), alpha=0.5, beta=2.0, C=C)
    ref_f = oracle.lramm.lramm(A32, B32, 24, 8, 1, 7, (0, 0, 0), alpha=0.5, beta=2.0, C=C)
    quantised_agreement(D, ref, ref_f, 0.5 * oracle.lramm.exact_product(A32, B32) + 2.0 * C)
    plan0 = L.Plan(m, n, k, 24, 8, 1, seed=7, prec=(0, 0, 0), alpha=0.5, beta=2.0)
    D0 = np_(L.matmul(plan0, dev(A32), dev(B32), C=dev(C))).astype(np.float64)
    assert oracle.lramm.rel_fro(D0, ref_f) <= 1e-5


def test_matmul_graph_replay_bit_identical(L):
    """LRAMM_FLAG_GRAPH: the first call on a (non-default) stream captures the
    call into a CUDA graph, later calls with the same buffers replay it; the
    output is bit-identical to the uncaptured call, a new output buffer is
    captured anew, and the launch counter counts the replayed kernels."""
    m = n = k = 512
    A, B = workloads.operands("lramm_512", scale=(m, n, k))
    A32, B32 = dev(A.astype(np.float32)), dev(B.astype(np.float32))
    ref_plan = L.Plan(m, n, k, 64, 10, 1, seed=7, prec=(1, 1, 1), sketch=L.SKETCH_TF32)
    ref = np_(L.matmul(ref_plan, A32, B32))
    plan = L.Plan(m, n, k, 64, 10, 1, seed=7, prec=(1, 1, 1), sketch=L.SKETCH_TF32, graph=True)
    ws = plan.workspace()
    s = torch.cuda.Stream()
    D1 = torch.empty((m, n), dtype=torch.float32, device="cuda")
    D2 = torch.empty_like(D1)
    with torch.cuda.stream(s):
        L.matmul(plan, A32, B32, out=D1, ws=ws)           # capture + launch
        c0 = L.launch_count()
        D1.zero_()
        L.matmul(plan, A32, B32, out=D1, ws=ws)           # replay
        per_call = L.launch_count() - c0
        L.matmul(plan, A32, B32, out=D2, ws=ws)           # other output: capture again
    s.synchronize()
    assert L.status_read(ws, stream=s) == 0
    assert np.array_equal(np_(D1), ref) and np.array_equal(np_(D2), ref)
    assert per_call > 50


@pytest.mark.parametrize("which", ["A", "B", "both"])
def test_matmul_zero_operand(L, which):
    """Degenerate input: a zero operand. Its sketch, Gram and R factor are
    zero (the Cholesky meets zero pivots: status 0 or LRAMM_ERR_NUMERIC), the
    singular values vanish and D is exactly zero -- no NaN or Inf anywhere."""
    m, n, k = 200, 180, 160
    rng = np.random.default_rng(5)
    A = rng.standard_normal((m, k)).astype(np.float32)
    B = rng.standard_normal((k, n)).astype(np.float32)
    if which in ("A", "both"):
        A[:] = 0
    if which in ("B", "both"):
        B[:] = 0
    for prec in ((0, 0, 0), (1, 1, 1)):
        plan = L.Plan(m, n, k, 16, 4, 1, seed=7, prec=prec)
        ws = plan.workspace()
        D = np_(L.matmul(plan, dev(A), dev(B), ws=ws))
        assert L.status_read(ws) in (0, 5)
        assert np.all(D == 0), prec
