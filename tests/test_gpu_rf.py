"""Range-finder form C ~ (X Q)(Q^T W) and its hand-written backward, through
the C ABI, against the FP64 oracle (oracle/rf.py, whose gradients are pinned
to central finite differences).

Bars: FP32 forward <= 1e-5 relative Frobenius; gradients dX, dW <= 1e-4
relative Frobenius (FP32 arithmetic through the QR adjoints and the power
chain); quantised (FP8 e4m3) forward within the quantisation-noise criterion
of the other end-to-end tests.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import quantised_agreement

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _case(m, k, n, seed, spectrum="exp32"):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, k)).astype(np.float32)
    W = workloads.lowrank(k, n, workloads.spectrum(spectrum, min(k, n)), seed + 1).astype(np.float32)
    G = rng.standard_normal((m, n)).astype(np.float32)
    return X, W, G


SHAPES = [(96, 80, 112, 10, 4, 0), (200, 160, 150, 12, 4, 1), (128, 256, 192, 20, 8, 2), (64, 300, 257, 28, 4, 1),
          (512, 900, 1000, 380, 20, 1)]


def _spectrum(l):
    """exp(-i/32) for the small sketches; for l = 400 the linear-layer weight's
    spectrum exp(-i/128) + 1e-3 (with exp(-i/32), sigma_400 / sigma_0 = 4e-6:
    the sketch is numerically rank-deficient in FP32 and CholeskyQR breaks
    down)."""
    return "exp128" if l > 64 else "exp32"


@pytest.mark.parametrize("m,k,n,r,p,q", SHAPES)
def test_rf_forward_fp32(L, m, k, n, r, p, q):
    X, W, _ = _case(m, k, n, m + k + n, _spectrum(r + p))
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, 0))
    ws = plan.workspace()
    C = L.rf_forward(plan, dev(X), dev(W), ws=ws).cpu().numpy().astype(np.float64)
    assert L.status_read(ws) == 0
    ref = oracle.rf.rf_forward(X, W, r, p, q, 7)
    assert oracle.lramm.rel_fro(C, ref) <= 1e-5


@pytest.mark.parametrize("m,k,n,r,p,q", SHAPES)
def test_rf_backward_fp32(L, m, k, n, r, p, q):
    X, W, G = _case(m, k, n, 3 * m + k, _spectrum(r + p))
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, 0))
    ws = plan.workspace()
    dX, dW = (t.cpu().numpy().astype(np.float64) for t in L.rf_backward(plan, dev(X), dev(W), dev(G), ws=ws))
    assert L.status_read(ws) == 0
    rX, rW = oracle.rf.rf_backward(X, W, G, r, p, q, 7)
    assert oracle.lramm.rel_fro(dX, rX) <= 1e-4
    assert oracle.lramm.rel_fro(dW, rW) <= 1e-4


def test_rf_gradients_at_32_match_finite_differences(L):
    """m = n = k = 32: the GPU gradients against FP64 central differences of
    the oracle's forward (directional derivatives)."""
    m = n = k = 32
    X, W, G = _case(m, k, n, 11)
    r, p, q = 6, 2, 1
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, 0))
    dX, dW = (t.cpu().numpy().astype(np.float64) for t in L.rf_backward(plan, dev(X), dev(W), dev(G)))
    X64, W64, G64 = X.astype(np.float64), W.astype(np.float64), G.astype(np.float64)
    rng = np.random.default_rng(12)
    h = 1e-6

    def loss(Xv, Wv):
        return np.sum(G64 * oracle.rf.rf_forward(Xv, Wv, r, p, q, 7))
    for _ in range(4):
        EX, EW = rng.standard_normal(X.shape), rng.standard_normal(W.shape)
        fdx = (loss(X64 + h * EX, W64) - loss(X64 - h * EX, W64)) / (2 * h)
        fdw = (loss(X64, W64 + h * EW) - loss(X64, W64 - h * EW)) / (2 * h)
        assert abs(np.sum(dX * EX) - fdx) <= 1e-4 * (abs(fdx) + np.linalg.norm(dX) * np.linalg.norm(EX) * 1e-3)
        assert abs(np.sum(dW * EW) - fdw) <= 1e-4 * (abs(fdw) + np.linalg.norm(dW) * np.linalg.norm(EW) * 1e-3)


@pytest.mark.parametrize("prec", [1, 3])
def test_rf_forward_quantised(L, prec):
    m, k, n, r, p, q = 256, 192, 224, 24, 8, 1
    X, W, _ = _case(m, k, n, 21)
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, prec))
    C = L.rf_forward(plan, dev(X), dev(W)).cpu().numpy().astype(np.float64)
    ref_q = oracle.rf.rf_forward(X, W, r, p, q, 7, prec=prec)
    ref_f = oracle.rf.rf_forward(X, W, r, p, q, 7)
    quantised_agreement(C, ref_q, ref_f, oracle.lramm.exact_product(X, W))


def test_rf_bf16_activations(L):
    """X stored in BF16 (the linear-layer configuration): the oracle sees the same BF16 values."""
    m, k, n, r, p, q = 160, 128, 144, 16, 4, 1
    X, W, _ = _case(m, k, n, 31)
    Xb = torch.from_numpy(X).to(torch.bfloat16)
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, 0), a_type=L.BF16)
    C = L.rf_forward(plan, Xb.cuda(), dev(W)).cpu().numpy().astype(np.float64)
    ref = oracle.rf.rf_forward(Xb.float().numpy(), W, r, p, q, 7)
    assert oracle.lramm.rel_fro(C, ref) <= 1e-5


def test_rf_autograd(L):
    m, k, n, r, p, q = 96, 128, 112, 12, 4, 1
    X, W, G = _case(m, k, n, 41)
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(0, 0, 0))
    Xt = dev(X).requires_grad_(True)
    Wt = dev(W).requires_grad_(True)
    C = L.rf_matmul(Xt, Wt, plan)
    (C * dev(G)).sum().backward()
    rX, rW = oracle.rf.rf_backward(X, W, G, r, p, q, 7)
    assert oracle.lramm.rel_fro(Xt.grad.cpu().numpy().astype(np.float64), rX) <= 1e-4
    assert oracle.lramm.rel_fro(Wt.grad.cpu().numpy().astype(np.float64), rW) <= 1e-4
