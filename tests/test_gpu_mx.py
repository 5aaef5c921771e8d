"""MXFP4 operands, split-precision residuals and the lead / tail E3 through
the C ABI against the oracle (oracle/mixed.py).

* MXFP4 codes and block exponents: bit-exact (the decisions are FP32 a_max,
  one FP32 division and the binary exponent on both sides).
* Block-scaled product: exact block sums; the sum over blocks is FP32 on the
  GPU, so |D - ref| <= nb 2^-24 sum_b |term_b| (+ one rounding).
* Lead / tail chain on identical FP32 factors: every QM term is formed
  exactly as the oracle forms it (integer E1, E2 and lead terms are
  bit-identical); the MXFP4 tail sums its blocks and the terms are added in
  FP32 (GPU) vs FP64 (oracle): element by element within those sums' FP32
  bounds (tests/elementwise.py).
* End to end (RSVD in FP32 on the GPU, FP64 in the oracle): the
  quantisation-noise criterion of the other end-to-end tests.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import elementwise as EW
from tests.test_gpu_parity import _factors, quantised_agreement

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
MX = oracle.mixed


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _mx_input(rows, cols, seed):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((rows, cols)) * np.exp(rng.uniform(-6, 6, (rows, cols)))).astype(np.float32)
    X[0, :] = 0.0                      # all-zero blocks
    if rows > 2 and cols > 40:
        X[2, 33] = 3.0e7               # one large entry in one block only
        X[1, :32] = 6.0                # exact-power edge: e = 0, codes 6
    return X


@pytest.mark.parametrize("rows,cols", [(37, 77), (300, 256), (5, 32), (129, 1000)])
def test_quantize_mx_bit_exact(L, rows, cols):
    X = _mx_input(rows, cols, rows + cols)
    c, e = L.quantize_mx(dev(X))
    c, e = c.cpu().numpy(), e.cpu().numpy()
    rc, re = MX.quantize_mxfp4(X)
    K = c.shape[1]
    want = np.zeros((rows, K))
    want[:, :cols] = 2.0 * rc
    assert np.array_equal(c.astype(np.float64), want)
    assert np.array_equal(e.astype(np.int64), re)


@pytest.mark.parametrize("M,N,K", [(70, 45, 64), (129, 65, 800), (1, 1, 32), (300, 260, 448)])
def test_qgemm_mx_within_fp32_block_sum(L, M, N, K):
    rng = np.random.default_rng(M + N + K)
    Lm = (rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, K)))).astype(np.float32)
    Rm = (rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, K)))).astype(np.float32)
    cl, el = L.quantize_mx(dev(Lm))
    cr, er = L.quantize_mx(dev(Rm))
    D = L.qgemm_mx(cl, el, cr, er).cpu().numpy().astype(np.float64)
    ocl, oel = MX.quantize_mxfp4(Lm)
    ocr, oer = MX.quantize_mxfp4(Rm)
    ref = MX.mx_product(ocl, oel, ocr, oer)
    mag = MX.mx_product(np.abs(ocl), oel, np.abs(ocr), oer)
    nb = K // 32
    assert np.all(np.abs(D - ref) <= nb * 2.0 ** -24 * mag + 2.0 ** -24 * np.abs(ref))


LEAD_CASES = [(8, 2, 2), (8, 1, 4), (8, 0, 3), (40, 2, 2), (16, 2, 4), (0, 0, 4), (12, 2, 0)]


@pytest.mark.parametrize("lead,split,tail", LEAD_CASES)
@pytest.mark.parametrize("scale", [0, 1])
def test_chain_lead_tail_matches_oracle(L, lead, split, tail, scale):
    m, n, k, r = 300, 260, 333, 40
    Ut, Vt, Wt, Zt = _factors(m, n, k, r, 61)
    prec = (1, 1, tail)
    plan = L.Plan(m, n, k, r, 0, 0, prec=prec, scale=scale, lead=lead, lead_prec=1, lead_split=split)
    D = L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt)).cpu().numpy().astype(np.float64)
    ref = MX.chain_lead_tail(Ut, Vt.T, Wt.T, Zt.T, prec, lead, 1, split, scale)
    bound = EW.lead_tail_bound(Ut, Vt, Wt, Zt, prec, lead, 1, split, scale)
    bad = np.abs(D - ref) > bound
    assert not bad.any(), "%d entries outside the bound, worst %.3g x bound" % (
        int(bad.sum()), float(np.max(np.abs(D - ref) / bound)))


@pytest.mark.parametrize("tail", [4, 1])
def test_chain_lead_tail_alpha_beta(L, tail):
    """D = alpha E3 + beta C with the lead / tail E3 in one tensor-core pass
    (INT8 lead with both residuals; MXFP4 or INT8 tail): beta C joins the
    first term, as when every term is its own pass."""
    m, n, k, r, lead = 260, 300, 200, 48, 16
    Ut, Vt, Wt, Zt = _factors(m, n, k, r, 63)
    C = np.random.default_rng(64).standard_normal((m, n)).astype(np.float32)
    prec = (1, 1, tail)
    plan = L.Plan(m, n, k, r, 0, 0, prec=prec, lead=lead, lead_prec=1, lead_split=2, alpha=0.75, beta=-1.5)
    D = L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt), C=dev(C)).cpu().numpy().astype(np.float64)
    ref = MX.chain_lead_tail(Ut, Vt.T, Wt.T, Zt.T, prec, lead, 1, 2, alpha=0.75, beta=-1.5, C=C)
    bound = EW.lead_tail_bound(Ut, Vt, Wt, Zt, prec, lead, 1, 2, alpha=0.75, beta=-1.5, C=C)
    assert np.all(np.abs(D - ref) <= bound), float(np.max(np.abs(D - ref) / bound))


def test_chain_mxfp4_everywhere(L):
    m, n, k, r = 200, 180, 260, 64
    Ut, Vt, Wt, Zt = _factors(m, n, k, r, 62)
    plan = L.Plan(m, n, k, r, 0, 0, prec=(4, 4, 4))
    D = L.chain(plan, dev(Ut), dev(Vt), dev(Wt), dev(Zt)).cpu().numpy().astype(np.float64)
    ref = MX.chain_lead_tail(Ut, Vt.T, Wt.T, Zt.T, (4, 4, 4), 0, 1, 0)
    assert oracle.lramm.rel_fro(D, ref) <= 1e-5


@pytest.mark.parametrize("sketch", ["f32", "tf32"])
def test_lead_tail_end_to_end_bf16(L, sketch):
    """The 8192 workload's recipe at 512: BF16 operands, INT8 lead with both
    residuals, MXFP4 tail; the lead split cuts the error of the all-4-bit E3.
    With tensor-core products (the bench's mode: BF16 operands on kind::f16
    and the factors assembled in TF32, info word 3) and without."""
    m = n = k = 512
    A, B = workloads.operands("lramm_8192", scale=(m, n, k))
    Ab = torch.from_numpy(A.astype(np.float32)).to(torch.bfloat16)
    Bb = torch.from_numpy(B.astype(np.float32)).to(torch.bfloat16)
    A32, B32 = Ab.float().numpy(), Bb.float().numpy()
    r, p, q, lead = 64, 8, 1, 16
    sk = L.SKETCH_TF32 if sketch == "tf32" else L.SKETCH_F32
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(1, 1, 4), a_type=L.BF16, b_type=L.BF16, lead=lead, lead_prec=1,
                  lead_split=2, sketch=sk)
    ws = plan.workspace()
    D = L.matmul(plan, Ab.cuda(), Bb.cuda(), ws=ws).cpu().numpy().astype(np.float64)
    assert (int(L.info_read(ws, 4)[3]) & 1) == (1 if sketch == "tf32" else 0)
    assert L.status_read(ws) == 0
    fac = oracle.lramm.factors(A32, B32, r, p, q, 7)
    ref_q = MX.chain_lead_tail(*fac, (1, 1, 4), lead, 1, 2)
    ref_f = oracle.lramm.chain(*fac, (0, 0, 0))
    exact = oracle.lramm.exact_product(A32, B32)
    quantised_agreement(D, ref_q, ref_f, exact)
    all4 = MX.chain_lead_tail(*fac, (1, 1, 4), 0, 1, 0)
    assert oracle.lramm.rel_fro(ref_q, ref_f) < oracle.lramm.rel_fro(all4, ref_f)


def test_rf_forward_mxfp4(L):
    m, k, n, r, p, q = 256, 192, 224, 24, 8, 1
    rng = np.random.default_rng(71)
    X = rng.standard_normal((m, k)).astype(np.float32)
    W = workloads.lowrank(k, n, workloads.spectrum("exp32", min(k, n)), 72).astype(np.float32)
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, 4))
    C = L.rf_forward(plan, dev(X), dev(W)).cpu().numpy().astype(np.float64)
    ref_q = oracle.rf.rf_forward(X, W, r, p, q, 7, prec=4)
    ref_f = oracle.rf.rf_forward(X, W, r, p, q, 7)
    quantised_agreement(C, ref_q, ref_f, oracle.lramm.exact_product(X, W))
